// Host-side pieces of the three-dimensional variant shared by its
// translation units (the step in sim3d.cu, the observables in
// observables3d.cu).
#pragma once
#include <cstddef>

#include "dpd.h"
#include "sim_host.h"

namespace dpd {

struct Sys3 {
    Sys b;                      // geometry scalars, physics, keys, scan/thermo/error words
    uint4 *S_p, *U_p, *C_p;
    float4 *S_v, *U_v, *C_v, *C_f;
    long long *F;               // pair-force sums per sorted slot: x, y, z counts of 2^-24
                                // force units and a pad word (zero between steps)
    float4 *S_off;              // offset from the own cell's corner (length units) + id bits, sorted
    const uint32_t *corner;     // fixed-point corner ceil(c 2^32 / n_c) of cell coordinate c
    float rc2f;                 // r_c^2 (1 + 1e-5): candidate filter, never narrower than the exact test
    uint32_t *U_rank, *slot;
};

}  // namespace dpd

struct dpd3_ctx {
    dpd_params p{};
    dpd::Sys3 s{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int nscan = 1;
    void *pool = nullptr;
    char *stage = nullptr;     // 48 B/bead staging for host state transfers
    double *h_pin = nullptr;
    long long step = 0;
    bool have_state = false;
    void *obs = nullptr;       // observables scratch (observables3d.cu), grown on demand
    size_t obs_bytes = 0;
};

int dpd3_internal_latched(dpd3_ctx *c);
