// Batched ensemble: R replicas of uneven size and parameters advanced by one
// persistent kernel (include/dpd.h, dpd_batch_*).
//
// Each replica is an ordinary context (its own buffers, cell list, thermo log
// and canonical state), so every single-system call also works on it through
// dpd_batch_replica.  The batch adds a device table of the replicas' Sys
// descriptors, three work lists and one kernel that runs n whole steps for all
// replicas: per step three phases (cell scan, scatter, fused force/integrate)
// separated by grid-wide barriers.  In the scan phase block b takes work
// items b, b + G, b + 2G, ... (G blocks) of the list of 4096-cell chunks of
// the replicas' decoupled look-back scans.  The scatter phase's items
// (1024-bead chunks, shuffled once with a fixed seed so that a replica's
// chunks spread out) and the force phase's items (replica, cell block),
// ordered by estimated cost, largest first, are handed out by two counters
// that are cleared before each launch and never reset inside it (every
// block's last, failing take of a step keeps the count per step fixed),
// which balances uneven items across blocks.  The kernel is
// launched with no more blocks than can be resident at once and every
// barrier wait is bounded: a block that gives up latches DPD_ERR_TIMEOUT in
// the batch's error word instead of hanging.  The launch for a given step
// count is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "dpd.h"
#include "sim_host.h"
#include "sim_kernels.cuh"

namespace dpd {

constexpr int ENS_CHUNK = 1024;   // beads per scatter work item

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over the resident blocks: an arrival counter and a
// generation word.  The wait is bounded; on timeout the block sets the error
// word and proceeds.  skip != 0 makes this block not arrive (self-test).
__device__ void grid_barrier(unsigned *bar, unsigned nblocks, int *err, int skip)
{
    __syncthreads();
    if (threadIdx.x == 0 && !skip) {
        unsigned *count = bar, *gen = bar + 1;
        const unsigned g = ld_acquire_u32(gen);
        __threadfence();
        const unsigned t = atomicAdd(count, 1u);
        if (t == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_u32(gen) == g) {
                if (++spins > SPIN_LIMIT) { atomicOr(err, ERR_TIMEOUT); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Scatter U -> S of the beads [k0, k1) of one replica, four beads per thread
// in flight (their loads issued before any store), which a latency-bound
// phase of a few warps per SM needs.  Same result as scatter_one per bead.
template <int B>
__device__ __forceinline__ void scatter_chunk(const Sys &d, int k0, int k1)
{
    constexpr int U = 4;
    const int bd = blockDim.x;
    for (int kb = k0 + (int)threadIdx.x; kb < k1; kb += U * bd) {
        uint4 xv[U];
        uint32_t id[U], dst[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = kb + u * bd;
            if (k < k1) {
                xv[u] = d.U_xv[k];
                id[u] = d.U_id[k];
                dst[u] = d.U_rank[k];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (kb + u * bd < k1) dst[u] += d.cstart[cell_of<B>(d, cell_coord(d, xv[u].x), cell_coord(d, xv[u].y))];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = kb + u * bd;
            if (k >= k1) continue;
            if (dst[u] >= (uint32_t)d.n || id[u] >= (uint32_t)d.n) {
                set_err_at(d, ERR_INTERNAL, 1, k, dst[u], id[u]);
                continue;
            }
            d.S_xv[dst[u]] = xv[u];
            d.S_id[dst[u]] = id[u];
            d.slot[id[u]] = dst[u];
        }
    }
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Optional phase log (tlog != NULL, a profiling launch): per step s and phase
// p (scan, scatter, force), block b writes the nanoseconds from the start of
// the phase to its arrival at the barrier into tlog[(3 s + p) gridDim + b],
// and block 0 writes the global timer at each barrier release into
// tlog[3 nsteps gridDim + 4 s + i] (i = 0 at the step's start).
// 16 x 16 blocks: five CTAs per SM fit in shared memory, so the register
// budget of five is used (no spills); smaller blocks keep eight.
template <int B, int VAR>
__global__ void __launch_bounds__(TILE_THREADS, B == 16 ? 5 : 8)
    k_ensemble(const Sys *__restrict__ sys, const uint32_t *__restrict__ scan_items, int n_scan,
               const uint32_t *__restrict__ scat, int n_scat, const uint32_t *__restrict__ tiles, int n_tiles,
               unsigned *bar, int *berr, int nsteps, int final_last, unsigned long long *ctr,
               unsigned long long *tlog)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_item;
    const unsigned nb = gridDim.x;
    const bool lg = tlog != nullptr && threadIdx.x == 0;
    unsigned long long *rel = tlog ? tlog + 3ull * nsteps * nb : nullptr;
    unsigned long long t0 = 0;
    for (int s = 0; s < nsteps; ++s) {
        if (lg) { t0 = gtimer(); if (blockIdx.x == 0) rel[4 * s] = t0; }
        // phase 1: cell scans; a replica of n cells contributes
        // ceil(n / SCAN_TILE) items, each one chunk of its decoupled
        // look-back scan (the chunk comes from the replica's ticket)
        for (int it = blockIdx.x; it < n_scan; it += nb) {
            const Sys &d = sys[scan_items[it]];
            scan_decoupled_t<TILE_THREADS>(d, (d.ncells + SCAN_TILE - 1) / SCAN_TILE, (uint32_t *)smem);
        }
        if (lg) tlog[(3ull * s + 0) * nb + blockIdx.x] = gtimer() - t0;
        grid_barrier(bar, nb, berr, 0);
        if (lg) { t0 = gtimer(); if (blockIdx.x == 0) rel[4 * s + 1] = t0; }
        // phase 2: scatter U -> S in chunks of ENS_CHUNK beads, the chunks
        // taken from the second counter (step s starts at s (n_scat + G),
        // as in the force phase below)
        const unsigned long long sbase = (unsigned long long)s * (unsigned long long)(n_scat + nb);
        while (true) {
            if (threadIdx.x == 0) s_item = atomicAdd(ctr + 1, 1ull) - sbase;
            __syncthreads();
            const unsigned long long it = s_item;
            __syncthreads();
            if (it >= (unsigned long long)n_scat) break;
            const uint32_t w = scat[it];
            const Sys &d = sys[w >> 22];
            const int k0 = (int)(w & 0x3fffffu) * ENS_CHUNK;
            scatter_chunk<B>(d, k0, min(d.n, k0 + ENS_CHUNK));
        }
        if (lg) tlog[(3ull * s + 1) * nb + blockIdx.x] = gtimer() - t0;
        grid_barrier(bar, nb, berr, 0);
        if (lg) { t0 = gtimer(); if (blockIdx.x == 0) rel[4 * s + 2] = t0; }
        // phase 3: fused force / integrate / re-bin per (replica, cell block),
        // the blocks taking items from a counter (the list is ordered by
        // estimated cost, largest first).  The counter is cleared before the
        // launch and never reset inside it: in step s every block takes items
        // until one lies past the list, so the step consumes exactly
        // n_tiles + gridDim.x values and step s starts at s (n_tiles + gridDim.x).
        const int flags = F_ADVANCE | ((final_last && s == nsteps - 1) ? F_FINAL : 0);
        const unsigned long long base = (unsigned long long)s * (unsigned long long)(n_tiles + nb);
        while (true) {
            if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1ull) - base;
            __syncthreads();
            const unsigned long long it = s_item;
            __syncthreads();
            if (it >= (unsigned long long)n_tiles) break;
            const uint32_t w = tiles[it];
            const Sys &d = sys[w >> 22];
            Thermo3 th{0.0, 0.0, 0.0};
            force_tile<B, false, VAR>(d, (int)(w & 0x3fffffu), flags, smem, th);
            __syncthreads();
            thermo_flush_tile(d, th, (double *)(smem + tile_flush_off<B, VAR>()));
            __syncthreads();
        }
        if (lg) tlog[(3ull * s + 2) * nb + blockIdx.x] = gtimer() - t0;
        grid_barrier(bar, nb, berr, 0);
        if (lg && blockIdx.x == 0) rel[4 * s + 3] = gtimer();
    }
}

// Self-test of the bounded barrier: block 0 never arrives, every other block
// must give up after the spin limit and latch DPD_ERR_TIMEOUT.
__global__ void k_barrier_selftest(unsigned *bar, int *berr)
{
    grid_barrier(bar, gridDim.x, berr, blockIdx.x == 0);
}

}  // namespace dpd

using namespace dpd;

struct dpd_batch {
    int R = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<dpd_ctx *> reps;
    void *pool = nullptr;
    Sys *d_sys = nullptr;
    uint32_t *d_scan = nullptr, *d_scat = nullptr, *d_tiles = nullptr;
    unsigned *d_bar = nullptr;
    int *d_err = nullptr;
    unsigned long long *d_ctr = nullptr;   // work counters: [0] force phase, [1] scatter phase
    int n_scan = 0, n_scat = 0, n_tiles = 0, B = 8, var = 2, cap = 0, grid = 0;
    size_t smem = 0;
    cudaGraphExec_t g = nullptr;
    int64_t g_steps = -1;
    int *h_pin = nullptr;
};

#define CUB(x)                                                                      \
    do {                                                                            \
        const cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

template <int B, int VAR>
static int ens_prepare(dpd_batch *b)
{
    // the opt-in limit covers static plus dynamic shared memory
    cudaFuncAttributes fa;
    CUB(cudaFuncGetAttributes(&fa, k_ensemble<B, VAR>));
    if (b->smem + fa.sharedSizeBytes > (size_t)max_dynamic_smem()) return DPD_ERR_INVALID_ARG;
    CUB(cudaFuncSetAttribute(k_ensemble<B, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_dynamic_smem() - (int)fa.sharedSizeBytes));
    int dev = 0, nsm = 0, occ = 0;
    CUB(cudaGetDevice(&dev));
    CUB(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ensemble<B, VAR>, TILE_THREADS, b->smem));
    if (occ < 1) return DPD_ERR_INVALID_ARG;
    b->grid = nsm * occ;
    return DPD_OK;
}

template <int B, int VAR>
static void ens_launch(dpd_batch *b, int nsteps, int final_last, unsigned long long *tlog)
{
    k_ensemble<B, VAR><<<b->grid, TILE_THREADS, b->smem, b->st>>>(b->d_sys, b->d_scan, b->n_scan, b->d_scat, b->n_scat,
                                                                  b->d_tiles, b->n_tiles, b->d_bar, b->d_err, nsteps,
                                                                  final_last, b->d_ctr, tlog);
}

static int ens_dispatch_prepare(dpd_batch *b)
{
    if (b->var == 1) return b->B == 4 ? ens_prepare<4, 1>(b) : b->B == 8 ? ens_prepare<8, 1>(b) : ens_prepare<16, 1>(b);
    if (b->var == 3) return b->B == 4 ? ens_prepare<4, 3>(b) : b->B == 8 ? ens_prepare<8, 3>(b) : ens_prepare<16, 3>(b);
    if (b->var == 4) return b->B == 4 ? ens_prepare<4, 4>(b) : b->B == 8 ? ens_prepare<8, 4>(b) : ens_prepare<16, 4>(b);
    if (b->var == 5) return b->B == 4 ? ens_prepare<4, 5>(b) : b->B == 8 ? ens_prepare<8, 5>(b) : ens_prepare<16, 5>(b);
    return b->B == 4 ? ens_prepare<4, 2>(b) : b->B == 8 ? ens_prepare<8, 2>(b) : ens_prepare<16, 2>(b);
}

static void ens_dispatch_launch(dpd_batch *b, int nsteps, int final_last, unsigned long long *tlog = nullptr)
{
    if (b->var == 1) {
        if (b->B == 4) ens_launch<4, 1>(b, nsteps, final_last, tlog);
        else if (b->B == 8) ens_launch<8, 1>(b, nsteps, final_last, tlog);
        else ens_launch<16, 1>(b, nsteps, final_last, tlog);
    } else if (b->var == 3) {
        if (b->B == 4) ens_launch<4, 3>(b, nsteps, final_last, tlog);
        else if (b->B == 8) ens_launch<8, 3>(b, nsteps, final_last, tlog);
        else ens_launch<16, 3>(b, nsteps, final_last, tlog);
    } else if (b->var == 4) {
        if (b->B == 4) ens_launch<4, 4>(b, nsteps, final_last, tlog);
        else if (b->B == 8) ens_launch<8, 4>(b, nsteps, final_last, tlog);
        else ens_launch<16, 4>(b, nsteps, final_last, tlog);
    } else if (b->var == 5) {
        if (b->B == 4) ens_launch<4, 5>(b, nsteps, final_last, tlog);
        else if (b->B == 8) ens_launch<8, 5>(b, nsteps, final_last, tlog);
        else ens_launch<16, 5>(b, nsteps, final_last, tlog);
    } else {
        if (b->B == 4) ens_launch<4, 2>(b, nsteps, final_last, tlog);
        else if (b->B == 8) ens_launch<8, 2>(b, nsteps, final_last, tlog);
        else ens_launch<16, 2>(b, nsteps, final_last, tlog);
    }
}

static int ens_build_tables(dpd_batch *b)
{
    std::vector<Sys> sys(b->R);
    std::vector<uint32_t> order(b->R), scan, scat, tiles;
    int cap = 0;
    for (int r = 0; r < b->R; ++r) {
        sys[r] = b->reps[r]->d;
        cap = std::max(cap, sys[r].cap);
        const int nch = (sys[r].n + ENS_CHUNK - 1) / ENS_CHUNK, nt = sys[r].ntx * sys[r].ntx;
        if (nch >= (1 << 22) || nt >= (1 << 22)) return DPD_ERR_INVALID_ARG;
        for (int c = 0; c < nch; ++c) scat.push_back(((uint32_t)r << 22) | (uint32_t)c);
        for (int t = 0; t < nt; ++t) tiles.push_back(((uint32_t)r << 22) | (uint32_t)t);
    }
    // fixed-seed shuffles (xorshift, Fisher-Yates) spread replicas over blocks;
    // the largest replicas are scanned first
    uint64_t rs = 0x9E3779B97F4A7C15ull;
    auto rnd = [&rs]() { rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17; return rs; };
    auto shuffle = [&rnd](std::vector<uint32_t> &v) {
        for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[rnd() % i]);
    };
    shuffle(scat);
    // force items by estimated cost, largest first: pairs per cell grow as the
    // square of the bead density, times the cells of the block
    {
        std::vector<std::pair<double, uint32_t>> cost(tiles.size());
        for (size_t i = 0; i < tiles.size(); ++i) {
            const uint32_t w = tiles[i];
            const Sys &d = sys[w >> 22];
            const int t = (int)(w & 0x3fffffu), ty = t / d.ntx, tx = t - ty * d.ntx;
            const int tw = std::min(b->B, d.nc - tx * b->B), th = std::min(b->B, d.nc - ty * b->B);
            const double rho = (double)d.n / ((double)d.L * d.L);
            cost[i] = {-(rho * rho * tw * th), w};
        }
        std::stable_sort(cost.begin(), cost.end());
        for (size_t i = 0; i < tiles.size(); ++i) tiles[i] = cost[i].second;
    }
    for (int r = 0; r < b->R; ++r) order[r] = (uint32_t)r;
    std::stable_sort(order.begin(), order.end(), [&sys](uint32_t a, uint32_t c) { return sys[a].ncells > sys[c].ncells; });
    for (uint32_t r : order)
        for (int k = 0; k < (sys[r].ncells + SCAN_TILE - 1) / SCAN_TILE; ++k) scan.push_back(r);
    // every replica's tile plan fits the common shared-memory size
    for (int r = 0; r < b->R; ++r) sys[r].cap = cap;
    for (int r = 0; r < b->R; ++r) b->reps[r]->d.cap = cap;
    b->cap = cap;
    // the dynamic buffer also serves the scan phase's transpose
    b->smem = std::max(force_smem(b->B, b->var, cap, false), sizeof(uint32_t) * (size_t)SCAN_BUF);
    b->n_scan = (int)scan.size();
    b->n_scat = (int)scat.size();
    b->n_tiles = (int)tiles.size();
    if (b->pool) cudaFree(b->pool);
    const size_t bytes = sizeof(Sys) * (size_t)b->R + 4 * scan.size() + 4 * scat.size() + 4 * tiles.size() + 256 * 5;
    CUB(cudaMalloc(&b->pool, bytes));
    char *p = (char *)b->pool;
    b->d_sys = (Sys *)p; p += (sizeof(Sys) * (size_t)b->R + 255) & ~size_t(255);
    b->d_scan = (uint32_t *)p; p += (4 * scan.size() + 255) & ~size_t(255);
    b->d_scat = (uint32_t *)p; p += (4 * scat.size() + 255) & ~size_t(255);
    b->d_tiles = (uint32_t *)p; p += (4 * tiles.size() + 255) & ~size_t(255);
    b->d_bar = (unsigned *)p;          // 2 words
    b->d_err = (int *)(b->d_bar + 8);  // 1 word
    b->d_ctr = (unsigned long long *)(b->d_bar + 16);
    CUB(cudaMemcpyAsync(b->d_sys, sys.data(), sizeof(Sys) * (size_t)b->R, cudaMemcpyHostToDevice, b->st));
    CUB(cudaMemcpyAsync(b->d_scan, scan.data(), 4 * scan.size(), cudaMemcpyHostToDevice, b->st));
    CUB(cudaMemcpyAsync(b->d_scat, scat.data(), 4 * scat.size(), cudaMemcpyHostToDevice, b->st));
    CUB(cudaMemcpyAsync(b->d_tiles, tiles.data(), 4 * tiles.size(), cudaMemcpyHostToDevice, b->st));
    CUB(cudaMemsetAsync(b->d_bar, 0, 64, b->st));
    for (int r = 0; r < b->R; ++r) {
        dpd_ctx *c = b->reps[r];
        c->smem = b->smem;
        const int rc = set_force_smem(c->B, b->var, cap);
        if (rc) return rc;
    }
    int rc = ens_dispatch_prepare(b);
    if (rc) return rc;
    CUB(cudaStreamSynchronize(b->st));
    return DPD_OK;
}

extern "C" {

int dpd_batch_create(const dpd_params *p, int R, void *stream, dpd_batch **out)
{
    if (!out || !p || R < 1 || R > 1023) return DPD_ERR_INVALID_ARG;
    *out = nullptr;
    for (int r = 0; r < R; ++r) {
        const int rc = validate(&p[r]);
        if (rc) return rc;
        if (p[r].tile != p[0].tile || p[r].variant != p[0].variant)
            return DPD_ERR_INVALID_ARG;   // one kernel shape for the whole batch
    }
    // one shape for every replica: the caller's, the tuned one, or the default
    std::vector<dpd_params> q(p, p + R);
    {
        int t = p[0].tile ? p[0].tile : DEFAULT_TILE, v = p[0].variant ? p[0].variant : DEFAULT_VARIANT;
        if (!p[0].tile && !p[0].variant) tuned_shape(p, R, &t, &v);
        for (auto &e : q) { e.tile = t; e.variant = v; }
    }
    dpd_batch *b = new (std::nothrow) dpd_batch();
    if (!b) return DPD_ERR_OOM;
    b->R = R;
    if (stream) {
        b->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) { delete b; return DPD_ERR_CUDA; }
        b->own_stream = true;
    }
    b->B = q[0].tile;
    b->var = q[0].variant;
    b->reps.assign(R, nullptr);
    int rc = DPD_OK;
    for (int r = 0; r < R && rc == DPD_OK; ++r) {
        rc = dpd_create(&q[r], b->st, &b->reps[r]);
        if (rc == DPD_OK) b->reps[r]->batch_owned = true;
    }
    if (rc == DPD_OK && cudaMallocHost((void **)&b->h_pin, 64) != cudaSuccess) rc = DPD_ERR_OOM;
    if (rc == DPD_OK) rc = ens_build_tables(b);
    if (rc) {
        dpd_batch_destroy(b);
        return rc;
    }
    *out = b;
    return DPD_OK;
}

void dpd_batch_destroy(dpd_batch *b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->g) cudaGraphExecDestroy(b->g);
    for (dpd_ctx *c : b->reps) {
        if (c) {
            c->batch_owned = false;
            dpd_destroy(c);
        }
    }
    if (b->pool) cudaFree(b->pool);
    if (b->h_pin) cudaFreeHost(b->h_pin);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

int dpd_batch_replica(dpd_batch *b, int r, dpd_ctx **view)
{
    if (!b || !view || r < 0 || r >= b->R) return DPD_ERR_INVALID_ARG;
    *view = b->reps[r];
    return DPD_OK;
}

int dpd_batch_init_random(dpd_batch *b, uint64_t seed)
{
    if (!b) return DPD_ERR_INVALID_ARG;
    for (int r = 0; r < b->R; ++r) {
        const int rc = dpd_init_random(b->reps[r], seed + (uint64_t)r);
        if (rc) return rc;
    }
    return DPD_OK;
}

int dpd_batch_step(dpd_batch *b, int64_t n)
{
    if (!b || n < 0 || n > (1ll << 30)) return DPD_ERR_INVALID_ARG;
    for (dpd_ctx *c : b->reps)
        if (!c->have_state) return DPD_ERR_STATE;
    if (n == 0) return DPD_OK;
    if (!b->g || b->g_steps != n) {
        if (b->g) cudaGraphExecDestroy(b->g);
        b->g = nullptr;
        cudaGraph_t gr = nullptr;
        CUB(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(b->d_ctr, 0, 2 * sizeof(unsigned long long), b->st);
        ens_dispatch_launch(b, (int)n, 1);
        const cudaError_t e = cudaStreamEndCapture(b->st, &gr);
        if (e != cudaSuccess) return DPD_ERR_CUDA;
        const cudaError_t e2 = cudaGraphInstantiate(&b->g, gr, 0);
        cudaGraphDestroy(gr);
        if (e2 != cudaSuccess) return DPD_ERR_CUDA;
        b->g_steps = n;
    }
    CUB(cudaGraphLaunch(b->g, b->st));
    for (dpd_ctx *c : b->reps) {
        c->step += n;
        c->sorted_canonical = true;
    }
    return DPD_OK;
}

int dpd_batch_sync(dpd_batch *b)
{
    if (!b) return DPD_ERR_INVALID_ARG;
    CUB(cudaMemcpyAsync(b->h_pin, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    CUB(cudaStreamSynchronize(b->st));
    int status = DPD_OK;
    if (b->h_pin[0] & ERR_TIMEOUT) status = DPD_ERR_TIMEOUT;
    for (dpd_ctx *c : b->reps) {
        const int rc = dpd_internal_latched(c);
        if (rc && status == DPD_OK) status = rc;
    }
    return status;
}

int dpd_batch_barrier_selftest(dpd_batch *b)
{
    if (!b) return DPD_ERR_INVALID_ARG;
    CUB(cudaMemsetAsync(b->d_bar, 0, 64, b->st));
    int dev = 0, nsm = 0;
    CUB(cudaGetDevice(&dev));
    CUB(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    k_barrier_selftest<<<std::min(nsm, 8), 32, 0, b->st>>>(b->d_bar, b->d_err);
    CUB(cudaGetLastError());
    CUB(cudaMemcpyAsync(b->h_pin, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    CUB(cudaStreamSynchronize(b->st));
    const int seen = b->h_pin[0];
    // leave the batch usable: clear the error word and the barrier state
    CUB(cudaMemsetAsync(b->d_bar, 0, 64, b->st));
    CUB(cudaStreamSynchronize(b->st));
    return (seen & ERR_TIMEOUT) ? DPD_ERR_TIMEOUT : DPD_OK;
}

int dpd_batch_profile(dpd_batch *b, int nsteps, double out[6])
{
    if (!b || !out || nsteps < 1 || nsteps > 64) return DPD_ERR_INVALID_ARG;
    for (dpd_ctx *c : b->reps)
        if (!c->have_state) return DPD_ERR_STATE;
    const size_t n_blk = 3ull * nsteps * (size_t)b->grid, n_rel = 4ull * nsteps;
    unsigned long long *dlog = nullptr;
    CUB(cudaMalloc(&dlog, 8 * (n_blk + n_rel)));
    CUB(cudaMemsetAsync(b->d_ctr, 0, 2 * sizeof(unsigned long long), b->st));
    ens_dispatch_launch(b, nsteps, 1, dlog);
    std::vector<unsigned long long> h(n_blk + n_rel);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dlog, 8 * h.size(), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    cudaFree(dlog);
    if (e != cudaSuccess) return DPD_ERR_CUDA;
    for (dpd_ctx *c : b->reps) {
        c->step += nsteps;
        c->sorted_canonical = true;
    }
    // phase durations between barrier releases, and the mean over blocks of
    // the time a block worked in the phase (the rest is waiting at the barrier)
    double dur[3] = {0, 0, 0}, busy[3] = {0, 0, 0};
    const unsigned long long *rel = h.data() + n_blk;
    for (int s = 0; s < nsteps; ++s)
        for (int p = 0; p < 3; ++p) {
            dur[p] += (double)(rel[4 * s + p + 1] - rel[4 * s + p]);
            double sum = 0;
            for (int blk = 0; blk < b->grid; ++blk) sum += (double)h[(3ull * s + p) * b->grid + blk];
            busy[p] += sum / b->grid;
        }
    for (int p = 0; p < 3; ++p) {
        out[p] = dur[p] / nsteps / 1e6;
        out[3 + p] = busy[p] / nsteps / 1e6;
    }
    return dpd_batch_sync(b);
}

int dpd_batch_info(dpd_batch *b, int *n_replicas, int *grid, int *n_work_tiles)
{
    if (!b) return DPD_ERR_INVALID_ARG;
    if (n_replicas) *n_replicas = b->R;
    if (grid) *grid = b->grid;
    if (n_work_tiles) *n_work_tiles = b->n_tiles;
    return DPD_OK;
}

}  // extern "C"
