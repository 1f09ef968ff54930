// Host-side pieces shared by the translation units of libdpd.
#pragma once
#include <cstddef>

#include "dpd.h"
#include "dpd_device.cuh"

namespace dpd {
int n_cells_side(double L, double rc);
int validate(const dpd_params *p);
void fill_physics(Sys &d, const dpd_params *p);
void fill_geometry(Sys &d, const dpd_params *p, int B);
int tile_capacity(const dpd_params *p, int B);
size_t force_smem(int B, int var, int cap, bool count);
void launch_iteration(const Sys &d, int B, int var, cudaStream_t st, int nscan, size_t smem, int flags, bool count);
void launch_force_only(const Sys &d, int B, int var, cudaStream_t st, size_t smem, int flags, bool count);
void launch_scatter(const Sys &d, int B, cudaStream_t st);
int set_force_smem(int B, int var, int cap);
int max_dynamic_smem();
void launch_bin(const Sys &d, int B, cudaStream_t st);
void launch_kick_bin(const Sys &d, int B, cudaStream_t st);
int host_cell_of(int B, int nc, int cx, int cy);
bool tuned_shape(const dpd_params *p, int R, int *tile, int *variant);
constexpr int DEFAULT_TILE = 8, DEFAULT_VARIANT = 2;
}  // namespace dpd

struct dpd_ctx {
    dpd_params p{};
    dpd::Sys d{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int B = 8, var = 2, nscan = 1;
    size_t smem = 0;
    void *pool = nullptr;
    size_t pool_bytes = 0;
    uint32_t *pcnt_buf = nullptr;
    cudaGraphExec_t g1 = nullptr, g8 = nullptr, gfin = nullptr;
    long long step = 0;
    bool have_state = false;
    bool sorted_canonical = false;  // S / cstart hold the canonical positions
    bool batch_owned = false;       // a replica of a dpd_batch (destroyed with it)
    double *h_pin = nullptr;        // small pinned staging (thermo, scalars)
    void *obs = nullptr;            // observables scratch (observables.cu)
    void *stage = nullptr;          // 32 B/bead staging for host state transfers
    unsigned long long ovf_seen = 0;  // overflowed tiles already answered by a larger capacity
    int dev = -1;                   // CUDA device current at creation (owns every buffer)
};

int dpd_internal_latched(dpd_ctx *c);
void dpd_internal_free_obs(dpd_ctx *c);
