// Kernel-shape autotuner (include/dpd.h, dpd_autotune / dpd_batch_autotune).
//
// The paper ran a CPU molecular-dynamics code and has no counterpart of this:
// on the GPU the cell-block side B (cells per tile side) and the pair-walk
// variant only change how the work is cut into CTAs and lanes.  Every shape
// produces the same trajectory bits (integer pair separations, fixed-point
// force sums), so the tuner times each shape on the caller's workload, keeps
// the fastest in a process-wide cache, and dpd_create / dpd_batch_create take
// the cached shape when a caller leaves both tile and variant at 0.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dpd.h"
#include "sim_host.h"

namespace {

struct TuneEntry {
    bool batch;
    int64_t n_beads;     // single system: N; batch: sum of N
    double L, rc;        // single system: L, r_c; batch: sum of L^2, sum of N^2 (a mix fingerprint)
    int R;               // batch: replica count
    int tile, variant;
};

std::mutex g_mu;
std::vector<TuneEntry> g_cache;

bool same_key(const TuneEntry &a, const TuneEntry &b)
{
    return a.batch == b.batch && a.n_beads == b.n_beads && a.L == b.L && a.rc == b.rc && a.R == b.R;
}

TuneEntry single_key(const dpd_params *p)
{
    TuneEntry e{};
    e.batch = false;
    e.n_beads = p->n_beads;
    e.L = p->L;
    e.rc = p->rc;
    e.R = 1;
    return e;
}

TuneEntry batch_key(const dpd_params *p, int R)
{
    TuneEntry e{};
    e.batch = true;
    e.R = R;
    for (int r = 0; r < R; ++r) {
        e.n_beads += p[r].n_beads;
        e.L += p[r].L * p[r].L;
        e.rc += (double)p[r].n_beads * (double)p[r].n_beads;
    }
    return e;
}

void store(const TuneEntry &k)
{
    std::lock_guard<std::mutex> g(g_mu);
    for (auto &e : g_cache)
        if (same_key(e, k)) { e.tile = k.tile; e.variant = k.variant; return; }
    g_cache.push_back(k);
}

bool lookup(const TuneEntry &k, int *tile, int *variant)
{
    std::lock_guard<std::mutex> g(g_mu);
    for (const auto &e : g_cache)
        if (same_key(e, k)) { *tile = e.tile; *variant = e.variant; return true; }
    return false;
}

const int TILES[3] = {4, 8, 16};

// Fastest measured shape of a report (ties keep the earlier shape).
void pick(dpd_tune_report *rep)
{
    int best = -1;
    for (int i = 0; i < rep->n_shapes; ++i)
        if (rep->ms_per_step[i] > 0 && (best < 0 || rep->ms_per_step[i] < rep->ms_per_step[best])) best = i;
    rep->best_tile = best >= 0 ? rep->tile[best] : 0;
    rep->best_variant = best >= 0 ? rep->variant[best] : 0;
    rep->best_ms_per_step = best >= 0 ? rep->ms_per_step[best] : -1.0;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~Events() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
};

}  // namespace

namespace dpd {
// Shape that dpd_create (R = 1) or dpd_batch_create (R replicas) uses when
// the caller leaves tile and variant at 0: the tuned one if cached.
bool tuned_shape(const dpd_params *p, int R, int *tile, int *variant)
{
    return lookup(R == 1 ? single_key(p) : batch_key(p, R), tile, variant);
}
}  // namespace dpd

// Time n steps of a context on its own stream (best of two runs).
static int time_steps(dpd_ctx *c, int steps, Events &ev, double *ms_per_step)
{
    double best = -1.0;
    for (int rep = 0; rep < 2; ++rep) {
        if (cudaEventRecord(ev.a, c->st) != cudaSuccess) return DPD_ERR_CUDA;
        int rc = dpd_step(c, steps);
        if (rc) return rc;
        if (cudaEventRecord(ev.b, c->st) != cudaSuccess) return DPD_ERR_CUDA;
        rc = dpd_sync(c);
        if (rc) return rc;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) return DPD_ERR_CUDA;
        const double per = (double)ms / steps;
        if (best < 0 || per < best) best = per;
    }
    *ms_per_step = best;
    return DPD_OK;
}

extern "C" {

int dpd_autotune(const dpd_params *p, const double *x, const float *v, int where, int steps, void *stream,
                 dpd_tune_report *rep)
{
    if (!p || !rep || steps < 1 || steps > 100000 || (x && !v) || (where != DPD_HOST && where != DPD_DEVICE))
        return DPD_ERR_INVALID_ARG;
    int rc = dpd::validate(p);
    if (rc) return rc;
    std::memset(rep, 0, sizeof(*rep));
    Events ev;
    if (!ev.a || !ev.b) return DPD_ERR_CUDA;
    for (int ti = 0; ti < 3; ++ti)
        for (int var = 1; var <= 5; ++var) {
            const int i = rep->n_shapes++;
            rep->tile[i] = TILES[ti];
            rep->variant[i] = var;
            rep->ms_per_step[i] = -1.0;
            dpd_params q = *p;
            q.tile = TILES[ti];
            q.variant = var;
            dpd_ctx *c = nullptr;
            rc = dpd_create(&q, stream, &c);
            if (rc == DPD_ERR_INVALID_ARG) continue;   // shape does not fit in shared memory
            if (rc) return rc;
            rc = x ? dpd_set_state(c, x, v, nullptr, 0, where) : dpd_init_random(c, p->seed);
            if (!rc) rc = dpd_step(c, 2);
            if (!rc) rc = dpd_sync(c);
            if (!rc) rc = time_steps(c, steps, ev, &rep->ms_per_step[i]);
            dpd_destroy(c);
            if (rc) return rc;
        }
    pick(rep);
    if (rep->best_tile == 0) return DPD_ERR_INVALID_ARG;
    TuneEntry k = single_key(p);
    k.tile = rep->best_tile;
    k.variant = rep->best_variant;
    store(k);
    return DPD_OK;
}

int dpd_batch_autotune(const dpd_params *p, int R, int steps, void *stream, dpd_tune_report *rep)
{
    if (!p || !rep || R < 1 || R > 1023 || steps < 1 || steps > 100000) return DPD_ERR_INVALID_ARG;
    for (int r = 0; r < R; ++r) {
        const int rc = dpd::validate(&p[r]);
        if (rc) return rc;
    }
    std::memset(rep, 0, sizeof(*rep));
    Events ev;
    if (!ev.a || !ev.b) return DPD_ERR_CUDA;
    std::vector<dpd_params> q(p, p + R);
    for (int ti = 0; ti < 3; ++ti)
        for (int var = 2; var <= 5; ++var) {
            const int i = rep->n_shapes++;
            rep->tile[i] = TILES[ti];
            rep->variant[i] = var;
            rep->ms_per_step[i] = -1.0;
            for (auto &e : q) { e.tile = TILES[ti]; e.variant = var; }
            dpd_batch *b = nullptr;
            int rc = dpd_batch_create(q.data(), R, stream, &b);
            if (rc == DPD_ERR_INVALID_ARG) continue;
            if (rc) return rc;
            dpd_ctx *view = nullptr;
            rc = dpd_batch_replica(b, 0, &view);
            if (!rc) rc = dpd_batch_init_random(b, p[0].seed);
            if (!rc) rc = dpd_batch_step(b, steps);   // captures the graph for `steps`
            if (!rc) rc = dpd_batch_sync(b);
            double best = -1.0;
            for (int k = 0; k < 2 && !rc; ++k) {
                if (cudaEventRecord(ev.a, view->st) != cudaSuccess) { rc = DPD_ERR_CUDA; break; }
                rc = dpd_batch_step(b, steps);
                if (rc) break;
                if (cudaEventRecord(ev.b, view->st) != cudaSuccess) { rc = DPD_ERR_CUDA; break; }
                rc = dpd_batch_sync(b);
                float ms = 0.f;
                if (!rc && cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) rc = DPD_ERR_CUDA;
                if (!rc && (best < 0 || ms / steps < best)) best = (double)ms / steps;
            }
            dpd_batch_destroy(b);
            if (rc) return rc;
            rep->ms_per_step[i] = best;
        }
    pick(rep);
    if (rep->best_tile == 0) return DPD_ERR_INVALID_ARG;
    TuneEntry k = batch_key(p, R);
    k.tile = rep->best_tile;
    k.variant = rep->best_variant;
    store(k);
    return DPD_OK;
}

int dpd_tune_store(const dpd_params *p, int R, int tile, int variant)
{
    if (!p || R < 1 || R > 1023 || !(tile == 4 || tile == 8 || tile == 16) || variant < 1 || variant > 5)
        return DPD_ERR_INVALID_ARG;
    TuneEntry k = R == 1 ? single_key(p) : batch_key(p, R);
    k.tile = tile;
    k.variant = variant;
    store(k);
    return DPD_OK;
}

int dpd_tune_lookup(const dpd_params *p, int R, int *tile, int *variant)
{
    if (!p || !tile || !variant || R < 1 || R > 1023) return DPD_ERR_INVALID_ARG;
    return lookup(R == 1 ? single_key(p) : batch_key(p, R), tile, variant) ? DPD_OK : DPD_ERR_STATE;
}

void dpd_tune_clear(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_cache.clear();
}

}  // extern "C"
