// Per-step device work of the DPD dimer simulator, written as device
// functions so that the single-system kernels and the persistent ensemble
// kernel share them.
//
// One step s -> s+1 (standard velocity-Verlet, Sec. 5 of arXiv:1310.0998):
//   scan     cstart = exclusive_scan(counts), counts = 0, step += 1
//   scatter  U (unsorted, with ranks) -> S sorted by cell, slot[id]
//   force    per tile: pair forces (Eqs. DPDf, DPDcdr, weightFunc01), bond
//            (Eq. stiffSpring), propulsion and drag (Eq. DPDnp); then
//            v_s = v* + dt/2m f_s (skipped at set-up), FP64 thermo partials,
//            v_{s+1/2} = v_s + dt/2m f_s, x_{s+1} = wrap(x_s + dt v_{s+1/2}),
//            binning of x_{s+1} into counts (rank = atomic ticket) -> U.
#pragma once
#include "dpd_device.cuh"

namespace dpd {

// ------------------------------------------------------------------ scan ----
// Single-pass exclusive scan with decoupled look-back over blocks of
// SCAN_TILE cells.  Logical block ids come from a monotonically growing
// ticket so predecessors always run first; the epoch (ticket / nblocks) tags
// the status words so nothing needs clearing between launches.  Waits are
// bounded: on timeout the error bit is set and the scan continues.  NT
// threads per block: every block size cuts the cells into the same SCAN_TILE
// chunks, so the ticket epochs of a context stay consistent whichever kernel
// scans it.  Counts are read (and zeroed) and cell starts written with
// consecutive lanes on consecutive cells; the shared buffer s_buf
// (SCAN_BUF words, one pad word per 32 so that a thread's run of consecutive
// cells sits in distinct banks) turns that order into runs of SCAN_TILE / NT
// cells per thread and back.
constexpr int SCAN_BUF = SCAN_TILE + SCAN_TILE / 32;
__device__ __forceinline__ int scan_pad(int e) { return e + (e >> 5); }

template <int NT>
__device__ inline void scan_decoupled_t(const Sys &d, int nblocks, uint32_t *s_buf)
{
    constexpr int IPT = SCAN_TILE / NT;
    static_assert(IPT * NT == SCAN_TILE && NT % 32 == 0 && NT <= 1024, "scan block shape");
    __shared__ uint32_t s_warp[NT / 32];
    __shared__ uint32_t s_excl;
    __shared__ int s_bid;
    __shared__ uint32_t s_epoch;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const unsigned long long t = atomicAdd(d.scan_ticket, 1ull);
        s_bid = (int)(t % (unsigned long long)nblocks);
        s_epoch = (uint32_t)((t / (unsigned long long)nblocks + 1ull) & 0x3fffffffull);
    }
    __syncthreads();
    const int bid = s_bid;
    const unsigned long long ep = s_epoch;
    const int base = bid * SCAN_TILE;
    // batches of eight loads in flight, then the zeroing stores
    static_assert(IPT % 8 == 0, "scan load batches");
#pragma unroll
    for (int k0 = 0; k0 < IPT; k0 += 8) {
        uint32_t c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int idx = base + (k0 + k) * NT + tid;
            c[k] = idx < d.ncells ? d.counts[idx] : 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s_buf[scan_pad((k0 + k) * NT + tid)] = c[k];
    }
#pragma unroll 8
    for (int k = 0; k < IPT; ++k) {
        const int idx = base + k * NT + tid;
        if (idx < d.ncells) d.counts[idx] = 0u;
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll 8
    for (int k = 0; k < IPT; ++k) sum += s_buf[scan_pad(tid * IPT + k)];
    // block exclusive scan of the per-thread sums
    const int lane = tid & 31, wid = tid >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < NT / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NT / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
        const uint32_t total = __shfl_sync(0xffffffffu, wi, NT / 32 - 1);
        uint32_t excl = 0;
        unsigned long long *st = d.scan_status;
        if (bid == 0) {
            if (lane == 0) st_release_u64(&st[0], (ep << 34) | (2ull << 32) | total);
        } else {
            if (lane == 0) st_release_u64(&st[bid], (ep << 34) | (1ull << 32) | total);
            // Warp-wide look-back: lane l reads predecessor top - l.  The
            // window's words up to the nearest inclusive prefix are added
            // once all of them are published (aggregate or inclusive); a
            // window of 32 aggregates is added whole and the window moves
            // back.  A block therefore needs an inclusive prefix from one
            // of its 32 nearest predecessors, not from the next one, which
            // keeps the chain of waits across blocks short.
            int top = bid - 1;
            long long spins = 0;
            while (true) {
                const int j = top - lane;
                const unsigned long long w64 = j >= 0 ? ld_acquire_u64(&st[j]) : (2ull << 32);
                const unsigned long long fl = (w64 >> 32) & 3ull;
                const bool ok = j < 0 || ((w64 >> 34) == ep && fl != 0ull);
                const unsigned okm = __ballot_sync(0xffffffffu, ok);
                const unsigned incm = __ballot_sync(0xffffffffu, ok && fl == 2ull);
                const int m = incm ? __ffs(incm) - 1 : 31;          // last lane to add
                const unsigned need = m == 31 ? 0xffffffffu : ((2u << m) - 1u);
                if ((okm & need) == need) {
                    excl += __reduce_add_sync(0xffffffffu, (lane <= m && j >= 0) ? (uint32_t)w64 : 0u);
                    if (incm) break;
                    top -= 32;
                    continue;
                }
                if (++spins > SPIN_LIMIT) {
                    if (lane == 0) set_err_at(d, ERR_TIMEOUT, 3, bid, top, 0);
                    break;
                }
                __nanosleep(32);
            }
            if (lane == 0) st_release_u64(&st[bid], (ep << 34) | (2ull << 32) | (excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            if (bid == nblocks - 1) d.cstart[d.ncells] = excl + total;
        }
    }
    __syncthreads();
    uint32_t run = s_excl + s_warp[wid] + (incl - sum);
#pragma unroll 8
    for (int k = 0; k < IPT; ++k) {
        const int i = scan_pad(tid * IPT + k);
        const uint32_t c = s_buf[i];
        s_buf[i] = run;
        run += c;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < IPT; ++k) {
        const int e = k * NT + tid, idx = base + e;
        if (idx < d.ncells) d.cstart[idx] = s_buf[scan_pad(e)];
    }
    if (bid == 0 && tid == 0) {
        const long long s1 = *d.step + 1;
        *d.step = s1;
        double *th = d.thermo + 4 * (size_t)(s1 % THERMO_CAP);
        th[0] = 0.0; th[1] = 0.0; th[2] = 0.0; th[3] = 0.0;
    }
    __syncthreads();   // s_buf is free again for the caller
}


// --------------------------------------------------------------- scatter ----
template <int B>
__device__ __forceinline__ void scatter_one(const Sys &d, int k)
{
    const uint4 xv = d.U_xv[k];
    const uint32_t id = d.U_id[k], rank = d.U_rank[k];
    const int c = cell_of<B>(d, cell_coord(d, xv.x), cell_coord(d, xv.y));
    const uint32_t dst = d.cstart[c] + rank;
    if (dst >= (uint32_t)d.n || id >= (uint32_t)d.n) {
        set_err_at(d, ERR_INTERNAL, 1, k, dst, id);
        return;
    }
    d.S_xv[dst] = xv;
    d.S_id[dst] = id;
    d.slot[id] = dst;
}

// Bin a state held in U (uploaded or initial): rank of each bead in its cell.
template <int B>
__device__ __forceinline__ void bin_one(const Sys &d, int k)
{
    const uint4 xv = d.U_xv[k];
    const int c = cell_of<B>(d, cell_coord(d, xv.x), cell_coord(d, xv.y));
    d.U_rank[k] = atomicAdd(&d.counts[c], 1u);
}

// ------------------------------------------------------------- integrate ----
struct Thermo3 { float ke, px, py; };

// Everything after the pair sum for one owned bead at sorted slot g:
// bond + propulsion (partner through slot[id ^ 1]), drag, the two half kicks
// and the drift, canonical output, binning of the new position.
template <int B>
__device__ __forceinline__ void integrate_bead(const Sys &d, int g, uint4 xv, uint32_t id, float fx, float fy,
                                               int flags, Thermo3 &th)
{
    const uint32_t ps = d.slot[id ^ 1u];
    if (ps < (uint32_t)d.n) {
        const uint4 xp = d.S_xv[ps];
        const float dx = mdiff(d, xv.x, xp.x);
        const float dy = mdiff(d, xv.y, xp.y);
        const float r2 = dx * dx + dy * dy;
        if (r2 > 0.f) {
            const float r = sqrtf(r2);
            const float inv = 1.0f / r;
            const float ex = dx * inv, ey = dy * inv;   // from partner to self
            const float fb = -d.kbond * (r - d.r0);
            const float sp = (id & 1u) ? -d.fp : d.fp;  // n_k = head - tail
            fx += (fb + sp) * ex;
            fy += (fb + sp) * ey;
        }
    } else {
        set_err_at(d, ERR_INTERNAL, 2, g, id, ps);
    }
    float vx = vbits(xv.z), vy = vbits(xv.w);
    fx -= d.zeta * vx;
    fy -= d.zeta * vy;
    if (!(flags & F_FIRST)) { vx += d.hdtm * fx; vy += d.hdtm * fy; }
    th.ke += vx * vx + vy * vy;
    th.px += vx;
    th.py += vy;
    if (flags & F_FINAL) {
        d.C_xv[id] = make_uint4(xv.x, xv.y, fbits(vx), fbits(vy));
        d.C_f[id] = make_float2(fx, fy);
    }
    if (flags & F_ADVANCE) {
        vx += d.hdtm * fx;
        vy += d.hdtm * fy;
        const float ddx = d.dt * vx, ddy = d.dt * vy;
        uint32_t nx = xv.x, ny = xv.y;
        if (fabsf(ddx) < 0.25f * d.L && fabsf(ddy) < 0.25f * d.L) {   // false for NaN too
            nx = fx_add(d, xv.x, ddx);
            ny = fx_add(d, xv.y, ddy);
        } else {
            set_err(d, ERR_NONFINITE);
            vx = 0.f; vy = 0.f;
        }
        const int c = cell_of<B>(d, cell_coord(d, nx), cell_coord(d, ny));
        d.U_rank[g] = atomicAdd(&d.counts[c], 1u);
        d.U_xv[g] = make_uint4(nx, ny, fbits(vx), fbits(vy));
        d.U_id[g] = id;
    }
}

// ------------------------------------------------------------ force tile ----
// Shared-memory plan of one tile (B x B owned cells + one-cell halo).
constexpr int TILE_THREADS = 128;
template <int B>
struct TilePlan {
    static constexpr int NCL = (B + 2) * (B + 2);   // local cell table
    static constexpr int NH = 4 * B + 4;            // halo cells
    static constexpr int NINT = 2 * NCL + 5 * (NH + 1) + 2 * (B + 2) + 8;
    static __host__ __device__ size_t red_off() { return ((size_t)NINT * 4 + 7) & ~size_t(7); }
    static __host__ __device__ size_t bead_off(int nthreads)
    {
        return (red_off() + sizeof(double) * 3 * (size_t)(nthreads / 32 + 1) + 15) & ~size_t(15);
    }
    // per staged bead: pos 8, vel 8, id 4, fx 4, fy 4, local cell 1 (+ count 4)
    static __host__ __device__ size_t bead_bytes(bool count) { return count ? 33 : 29; }
    static __host__ __device__ size_t queue_off(int cap, int nthreads, bool count)
    {
        return (bead_off(nthreads) + (size_t)cap * bead_bytes(count) + 15) & ~size_t(15);
    }
    static __host__ __device__ size_t bytes(int cap, int nthreads, bool count)
    {
        return queue_off(cap, nthreads, count) + sizeof(uint32_t) * 128 * (size_t)(nthreads / 32);
    }
};

__device__ __forceinline__ float dpd_pair_scalar(const Sys &d, float dx, float dy, float dvx, float dvy,
                                                 uint32_t idi, uint32_t idj, uint32_t s_lo, uint32_t s_hi,
                                                 float r2, float &ex, float &ey)
{
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float w = 1.0f - r * d.inv_rc;
    ex = dx * rinv;
    ey = dy * rinv;
    const float dve = dvx * ex + dvy * ey;
    const float nz = pair_noise(d, idi, idj, s_lo, s_hi);
    if (!d.gen_w) return w * (d.a - d.gamma * w * dve + d.sig_r * nz);
    // changed exponent of w: w_R = w^(s/2), w_D = w_R^2 (uniform branch)
    const float wr = __powf(w, d.hwexp);
    return d.a * w - d.gamma * (wr * wr) * dve + d.sig_r * wr * nz;
}


// Neighbour offsets packed 2 bits per entry (value + 1), entries in the
// order 0 = own cell, 1-4 ahead (E, NE, N, NW), 5-8 behind (W, SW, S, SE).
constexpr uint32_t NB_DX = 0x1u | (2u << 2) | (2u << 4) | (1u << 6) | (0u << 8) | (0u << 10) | (0u << 12) |
                           (1u << 14) | (2u << 16);
constexpr uint32_t NB_DY = 0x1u | (1u << 2) | (2u << 4) | (2u << 6) | (2u << 8) | (1u << 10) | (0u << 12) |
                           (0u << 14) | (0u << 16);

// Offset of bead i seen from a bead in the cell (dx, dy) away.
__device__ __forceinline__ float shift_off(float o, int dx, float cs)
{
    return dx == 0 ? o : (dx > 0 ? o - cs : o + cs);
}

// Variant 1: one thread per owned bead walks its candidates and evaluates
// each interacting pair in place (divergent; kept as the simple reference
// kernel and for the autotuner).
template <int B, bool COUNT>
__device__ __forceinline__ void pairs_thread(const Sys &d, int n_own, int tw, int th_, const int *s_cbeg,
                                             const int *s_ccnt, const float2 *s_pos, const float2 *s_vel,
                                             const uint32_t *s_id, float *s_fx, float *s_fy, uint32_t *s_cnt,
                                             const unsigned char *s_lc, uint32_t s_lo, uint32_t s_hi)
{
    for (int k = threadIdx.x; k < n_own; k += blockDim.x) {
        const float2 oi = s_pos[k], vi = s_vel[k];
        const uint32_t idi = s_id[k], pid = d.excl ? (idi ^ 1u) : 0xffffffffu;
        const int lx = s_lc[k] & 15, ly = s_lc[k] >> 4;
        float fx = 0.f, fy = 0.f;
        uint32_t cnt = 0;
#pragma unroll 1
        for (int nb = 0; nb < 9; ++nb) {
            const int ox_ = (int)((NB_DX >> (2 * nb)) & 3u) - 1, oy_ = (int)((NB_DY >> (2 * nb)) & 3u) - 1;
            const int nlx = lx + ox_, nly = ly + oy_;
            const bool owned = (nlx >= 0 && nlx < tw && nly >= 0 && nly < th_);
            if (nb >= 5 && owned) continue;    // the other bead's forward sweep takes it
            const bool newton = owned;
            const float pix = shift_off(oi.x, ox_, d.cs), piy = shift_off(oi.y, oy_, d.cs);
            const int lc = (nly + 1) * (B + 2) + nlx + 1;
            int j = s_cbeg[lc];
            const int je = j + s_ccnt[lc];
            if (nb == 0) j = k + 1;
            for (; j < je; ++j) {
                const float2 pj = s_pos[j];
                const float dx = pix - pj.x, dy = piy - pj.y;
                const float r2 = dx * dx + dy * dy;
                if (r2 < d.rc2 && r2 > 0.f) {
                    const uint32_t idj = s_id[j];
                    if (idj == pid) continue;
                    const float2 vj = s_vel[j];
                    float ex, ey;
                    const float F = dpd_pair_scalar(d, dx, dy, vi.x - vj.x, vi.y - vj.y, idi, idj, s_lo, s_hi, r2,
                                                    ex, ey);
                    fx += F * ex;
                    fy += F * ey;
                    if (COUNT) ++cnt;
                    if (newton) {
                        atomicAdd(&s_fx[j], -F * ex);
                        atomicAdd(&s_fy[j], -F * ey);
                        if (COUNT) atomicAdd(&s_cnt[j], 1u);
                    }
                }
            }
        }
        atomicAdd(&s_fx[k], fx);
        atomicAdd(&s_fy[k], fy);
        if (COUNT) atomicAdd(&s_cnt[k], cnt);
    }
}

// Variant 2: pair queue.  Each lane walks the candidates of one owned bead at
// a time (taking the next bead from a block-wide counter when it runs out, so
// warps stay balanced); every candidate inside r_c is pushed, packed as
// (i, j, Newton-3 flag, cell offset), into the warp's 128-entry buffer.
// Whenever 32 pairs are queued the whole warp evaluates them together, so
// the Philox and force arithmetic runs with every lane active.  Forces land
// in shared memory through atomics on both sides of a Newton-3 pair.
template <bool COUNT>
__device__ __forceinline__ void queue_eval(const Sys &d, uint32_t code, const float2 *s_pos, const float2 *s_vel,
                                           const uint32_t *s_id, float *s_fx, float *s_fy, uint32_t *s_cnt,
                                           uint32_t s_lo, uint32_t s_hi)
{
    const int k = code & 0xfffu, j = (code >> 12) & 0xfffu;
    const bool newton = (code >> 24) & 1u;
    const int dcx = (int)((code >> 25) & 3u) - 1, dcy = (int)((code >> 27) & 3u) - 1;
    const float2 oi = s_pos[k], pj = s_pos[j], vi = s_vel[k], vj = s_vel[j];
    const float dx = shift_off(oi.x, dcx, d.cs) - pj.x, dy = shift_off(oi.y, dcy, d.cs) - pj.y;
    const float r2 = dx * dx + dy * dy;
    float ex, ey;
    const float F = dpd_pair_scalar(d, dx, dy, vi.x - vj.x, vi.y - vj.y, s_id[k], s_id[j], s_lo, s_hi, r2, ex, ey);
    const float gx = F * ex, gy = F * ey;
    atomicAdd(&s_fx[k], gx);
    atomicAdd(&s_fy[k], gy);
    if (COUNT) atomicAdd(&s_cnt[k], 1u);
    if (newton) {
        atomicAdd(&s_fx[j], -gx);
        atomicAdd(&s_fy[j], -gy);
        if (COUNT) atomicAdd(&s_cnt[j], 1u);
    }
}

template <int B, bool COUNT>
__device__ __forceinline__ void pairs_queue(const Sys &d, int n_own, int tw, int th_, const int *s_cbeg,
                                            const int *s_ccnt, const float2 *s_pos, const float2 *s_vel,
                                            const uint32_t *s_id, float *s_fx, float *s_fy, uint32_t *s_cnt,
                                            const unsigned char *s_lc, volatile uint32_t *q, int *s_next,
                                            uint32_t s_lo, uint32_t s_hi)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int k = -1, j = 0, je = 0, lc0 = 0;
    uint32_t visit = 0, own = 0, pid = 0, tag = 0;
    float2 oi = make_float2(0.f, 0.f);
    float pix = 0.f, piy = 0.f;
    bool more = true;
    int qn = 0;   // warp-uniform queue length (entries q[0, qn))
    while (true) {
        // At most one advance per lane per round (to the next neighbour
        // range of its bead, or to its next bead), so a lane switching cells
        // costs the warp one short divergent step instead of a loop.
        bool have = j < je;
        if (!have && more) {
            if (visit == 0u) {
                k = atomicAdd(s_next, 1);
                if (k >= n_own) {
                    more = false;
                } else {
                    oi = s_pos[k];
                    const int lx = s_lc[k] & 15, ly = s_lc[k] >> 4;
                    lc0 = (ly + 1) * (B + 2) + lx + 1;
                    pid = d.excl ? (s_id[k] ^ 1u) : 0xffffffffu;
                    // which neighbour cells are owned by this tile (Newton-3 side)
                    const uint32_t px = lx < tw - 1, nx = lx > 0, py = ly < th_ - 1, ny = ly > 0;
                    own = 1u | (px << 1) | ((px & py) << 2) | (py << 3) | ((nx & py) << 4) | (nx << 5) |
                          ((nx & ny) << 6) | (ny << 7) | ((px & ny) << 8);
                    visit = 0x1fu | (~own & 0x1e0u);   // cells behind only when they are halo
                }
            }
            if (more) {
                const int nb = __ffs(visit) - 1;
                visit &= visit - 1u;
                const int ox_ = (int)((NB_DX >> (2 * nb)) & 3u) - 1, oy_ = (int)((NB_DY >> (2 * nb)) & 3u) - 1;
                const int lc = lc0 + oy_ * (B + 2) + ox_;
                j = s_cbeg[lc];
                je = j + s_ccnt[lc];
                if (nb == 0) j = k + 1;
                pix = shift_off(oi.x, ox_, d.cs);
                piy = shift_off(oi.y, oy_, d.cs);
                tag = (uint32_t)k | (((own >> nb) & 1u) << 24) | ((uint32_t)(ox_ + 1) << 25) |
                      ((uint32_t)(oy_ + 1) << 27);
                have = j < je;
            }
        }
        if (!__any_sync(FULL, have || more)) break;
        // two candidates per lane per round (j and j + 1 while in range),
        // tested branch-free; one append point per round
        bool p0 = false, p1 = false;
        uint32_t c0 = 0, c1 = 0;
        if (have) {
            const float2 pj = s_pos[j];
            const float dx = pix - pj.x, dy = piy - pj.y;
            const float r2 = dx * dx + dy * dy;
            p0 = (r2 < d.rc2) & (r2 > 0.f) & (s_id[j] != pid);
            c0 = tag | ((uint32_t)j << 12);
            ++j;
            if (j < je) {
                const float2 pk = s_pos[j];
                const float ex = pix - pk.x, ey = piy - pk.y;
                const float s2 = ex * ex + ey * ey;
                p1 = (s2 < d.rc2) & (s2 > 0.f) & (s_id[j] != pid);
                c1 = tag | ((uint32_t)j << 12);
                ++j;
            }
        }
        const unsigned m0 = __ballot_sync(FULL, p0);
        const unsigned m1 = __ballot_sync(FULL, p1);
        const int n0 = __popc(m0);
        if (p0) q[qn + __popc(m0 & lt)] = c0;
        if (p1) q[qn + n0 + __popc(m1 & lt)] = c1;
        qn += n0 + __popc(m1);
        __syncwarp();
        while (qn >= 32) {
            // evaluate the oldest 32 entries, move the rest to the front
            const uint32_t mine = q[lane];
            const uint32_t carry0 = q[32 + lane], carry1 = q[64 + lane];
            __syncwarp();
            if (lane < qn - 32) q[lane] = carry0;
            if (lane + 32 < qn - 32) q[lane + 32] = carry1;
            qn -= 32;
            __syncwarp();
            queue_eval<COUNT>(d, mine, s_pos, s_vel, s_id, s_fx, s_fy, s_cnt, s_lo, s_hi);
        }
    }
    __syncwarp();
    if (lane < qn) queue_eval<COUNT>(d, q[lane], s_pos, s_vel, s_id, s_fx, s_fy, s_cnt, s_lo, s_hi);
}

// Global-memory path for a tile whose beads do not fit in shared memory: one
// thread per owned bead, pairs from both sides (no Newton-3), same arithmetic.
template <int B, bool COUNT>
__device__ void force_tile_global(const Sys &d, uint32_t g0, int n_own, uint32_t s_lo, uint32_t s_hi, int flags,
                                  Thermo3 &th)
{
    const uint32_t n = (uint32_t)d.n;
    const int NT = blockDim.x, tid = threadIdx.x;
    if (tid == 0) atomicAdd(d.ovf, 1ull);
    for (int k = tid; k < n_own; k += NT) {
        const int g = (int)g0 + k;
        const uint4 xv = d.S_xv[g];
        const float vix = vbits(xv.z), viy = vbits(xv.w);
        const uint32_t idi = d.S_id[g], pid = d.excl ? (idi ^ 1u) : 0xffffffffu;
        const int cx = cell_coord(d, xv.x), cy = cell_coord(d, xv.y);
        float fx = 0.f, fy = 0.f;
        uint32_t cnt = 0;
        for (int oy_ = -1; oy_ <= 1; ++oy_)
            for (int ox_ = -1; ox_ <= 1; ++ox_) {
                int ncx = cx + ox_, ncy = cy + oy_;
                ncx += (ncx < 0) ? d.nc : ((ncx >= d.nc) ? -d.nc : 0);
                ncy += (ncy < 0) ? d.nc : ((ncy >= d.nc) ? -d.nc : 0);
                const int gc = cell_of<B>(d, ncx, ncy);
                const uint32_t b = min(d.cstart[gc], n), e = min(max(d.cstart[gc + 1], b), n);
                for (uint32_t q = b; q < e; ++q) {
                    if (q == (uint32_t)g) continue;
                    const uint32_t idj = d.S_id[q];
                    if (idj == pid) continue;
                    const uint4 xj = d.S_xv[q];
                    const float dx = mdiff(d, xv.x, xj.x);
                    const float dy = mdiff(d, xv.y, xj.y);
                    const float r2 = dx * dx + dy * dy;
                    if (r2 < d.rc2 && r2 > 0.f) {
                        float ex, ey;
                        const float F = dpd_pair_scalar(d, dx, dy, vix - vbits(xj.z), viy - vbits(xj.w), idi,
                                                        idj, s_lo, s_hi, r2, ex, ey);
                        fx += F * ex;
                        fy += F * ey;
                        if (COUNT) ++cnt;
                    }
                }
            }
        if (COUNT && d.pcnt) d.pcnt[idi] = cnt;
        integrate_bead<B>(d, g, xv, idi, fx, fy, flags, th);
    }
}

// ------------------------------------------------- grid-order tile (VAR 3) --
// The tile's owned and halo cells are staged in shared memory in the row-major
// order of the local (B+2) x (B+2) cell grid, with raw fixed-point positions,
// so every row of the local grid is one contiguous bead range and a pair
// separation is the wrapped integer difference of two positions (exact) times
// the unit.  The forward half-stencil of an owned cell (own cell after the
// bead, E, and NW..NE) is then two ranges instead of five; a cell on the tile
// edge adds at most three ranges of halo cells behind it (W, and SW..SE or
// parts of that row).  Each lane walks the candidates of one owned bead at a
// time, CPR candidates per round; pairs inside r_c go through the warp's pair
// queue as in variant 2 (Newton-3 when the partner is owned).
template <int B>
struct TilePlanG {
    static constexpr int W = B + 2;
    static constexpr int NCL = W * W;
    static constexpr int NINT = 3 * NCL + 1 + 4;   // counts, begins (+1), global sources, misc
    static constexpr int CPR = 4;                   // candidates per lane per round
    static constexpr int QLEN = 32 * (CPR + 1);     // queue entries per warp
    static __host__ __device__ size_t red_off() { return ((size_t)NINT * 4 + 7) & ~size_t(7); }
    static __host__ __device__ size_t bead_off(int nthreads)
    {
        return (red_off() + sizeof(double) * 3 * (size_t)(nthreads / 32 + 1) + 15) & ~size_t(15);
    }
    // per staged bead: position 8, velocity 8, id 4, fx 4, fy 4, (count 4),
    // owned-bead slot 2, owned flag 1
    static __host__ __device__ size_t bead_bytes(bool count) { return count ? 35 : 31; }
    static __host__ __device__ size_t queue_off(int cap, int nthreads, bool count)
    {
        return (bead_off(nthreads) + (size_t)cap * bead_bytes(count) + 15) & ~size_t(15);
    }
    static __host__ __device__ size_t bytes(int cap, int nthreads, bool count)
    {
        return queue_off(cap, nthreads, count) + sizeof(uint32_t) * QLEN * (size_t)(nthreads / 32);
    }
};

template <bool COUNT>
__device__ __forceinline__ void queue_eval_g(const Sys &d, uint32_t code, const uint2 *s_X, const float2 *s_vel,
                                             const uint32_t *s_id, const unsigned char *s_own, float *s_fx,
                                             float *s_fy, uint32_t *s_cnt, uint32_t s_lo, uint32_t s_hi)
{
    const int k = code & 0xfffu, j = (code >> 12) & 0xfffu;
    const uint2 xi = s_X[k], xj = s_X[j];
    const float2 vi = s_vel[k], vj = s_vel[j];
    const float dx = mdiff(d, xi.x, xj.x), dy = mdiff(d, xi.y, xj.y);
    const float r2 = dx * dx + dy * dy;
    float ex, ey;
    const float F = dpd_pair_scalar(d, dx, dy, vi.x - vj.x, vi.y - vj.y, s_id[k], s_id[j], s_lo, s_hi, r2, ex, ey);
    const float gx = F * ex, gy = F * ey;
    atomicAdd(&s_fx[k], gx);
    atomicAdd(&s_fy[k], gy);
    if (COUNT) atomicAdd(&s_cnt[k], 1u);
    if (s_own[j]) {
        atomicAdd(&s_fx[j], -gx);
        atomicAdd(&s_fy[j], -gy);
        if (COUNT) atomicAdd(&s_cnt[j], 1u);
    }
}

template <int B, bool COUNT>
__device__ __forceinline__ void pairs_grid(const Sys &d, int n_own, int x0, int y0, int tw, const int *s_lbeg,
                                           const uint2 *s_X, const float2 *s_vel, const uint32_t *s_id,
                                           const unsigned char *s_own, const uint16_t *s_oslot, float *s_fx,
                                           float *s_fy, uint32_t *s_cnt, volatile uint32_t *q, int *s_next,
                                           uint32_t s_lo, uint32_t s_hi)
{
    using TP = TilePlanG<B>;
    constexpr int W = TP::W, CPR = TP::CPR;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int j = 0, je = 0, stage = 5, lc = 0, lx = 0, ly = 0, si = 0;
    uint32_t Xi = 0, Yi = 0, pid = 0;
    bool more = true;
    int qn = 0;   // warp-uniform queue length
    while (true) {
        bool have = j < je;
        if (!have && more) {
            if (stage >= 5) {
                const int k = atomicAdd(s_next, 1);
                if (k >= n_own) {
                    more = false;
                } else {
                    si = s_oslot[k];
                    const uint2 x = s_X[si];
                    Xi = x.x;
                    Yi = x.y;
                    pid = d.excl ? (s_id[si] ^ 1u) : 0xffffffffu;
                    lx = cell_coord(d, Xi) - x0;
                    ly = cell_coord(d, Yi) - y0;
                    lx += lx < -1 ? d.nc : 0;   // a tile never spans the box, so one wrap at most
                    ly += ly < -1 ? d.nc : 0;
                    lc = (ly + 1) * W + lx + 1;
                    stage = 0;
                }
            }
            // next non-empty range of this bead (stages 0..4)
            while (more && stage < 5 && !have) {
                int b = 0, e = 0;
                if (stage == 0) {          // W, when it is a halo cell
                    if (lx == 0) { b = s_lbeg[lc - 1]; e = s_lbeg[lc]; }
                } else if (stage == 1) {   // own cell after the bead, then E
                    b = si + 1;
                    e = s_lbeg[lc + 2];
                } else if (stage == 2) {   // NW, N, NE
                    b = s_lbeg[lc + W - 1];
                    e = s_lbeg[lc + W + 2];
                } else if (stage == 3) {   // the row below: all of it, or SW
                    if (ly == 0) { b = s_lbeg[lc - W - 1]; e = s_lbeg[lc - W + 2]; }
                    else if (lx == 0) { b = s_lbeg[lc - W - 1]; e = s_lbeg[lc - W]; }
                } else {                   // SE on the right edge
                    if (ly != 0 && lx == tw - 1) { b = s_lbeg[lc - W + 1]; e = s_lbeg[lc - W + 2]; }
                }
                ++stage;
                j = b;
                je = e;
                have = j < je;
            }
        }
        if (!__any_sync(FULL, have || more)) break;
        bool p[CPR];
        uint32_t c[CPR];
#pragma unroll
        for (int u = 0; u < CPR; ++u) {
            p[u] = false;
            c[u] = 0u;
            if (j < je) {
                const uint2 xj = s_X[j];
                const float dx = mdiff(d, Xi, xj.x), dy = mdiff(d, Yi, xj.y);
                const float r2 = dx * dx + dy * dy;
                p[u] = (r2 < d.rc2) & (r2 > 0.f) & (s_id[j] != pid);
                c[u] = (uint32_t)si | ((uint32_t)j << 12);
                ++j;
            }
        }
#pragma unroll
        for (int u = 0; u < CPR; ++u) {
            const unsigned m = __ballot_sync(FULL, p[u]);
            if (p[u]) q[qn + __popc(m & lt)] = c[u];
            qn += __popc(m);
        }
        __syncwarp();
        while (qn >= 32) {
            // evaluate the oldest 32 entries, move the rest (< 32 CPR) to the front
            const uint32_t mine = q[lane];
            uint32_t carry[CPR];
#pragma unroll
            for (int u = 0; u < CPR; ++u) carry[u] = q[32 * (u + 1) + lane];
            __syncwarp();
#pragma unroll
            for (int u = 0; u < CPR; ++u)
                if (lane + 32 * u < qn - 32) q[lane + 32 * u] = carry[u];
            qn -= 32;
            __syncwarp();
            queue_eval_g<COUNT>(d, mine, s_X, s_vel, s_id, s_own, s_fx, s_fy, s_cnt, s_lo, s_hi);
        }
    }
    __syncwarp();
    if (lane < qn) queue_eval_g<COUNT>(d, q[lane], s_X, s_vel, s_id, s_own, s_fx, s_fy, s_cnt, s_lo, s_hi);
}

template <int B, bool COUNT>
__device__ void force_tile_g(const Sys &d, int tile, int flags, unsigned char *smem, Thermo3 &th)
{
    using TP = TilePlanG<B>;
    constexpr int W = TP::W;
    const int NT = blockDim.x, tid = threadIdx.x;
    int *s_lcnt = (int *)smem;
    int *s_lbeg = s_lcnt + TP::NCL;
    int *s_lsrc = s_lbeg + TP::NCL + 1;
    int *s_sc = s_lsrc + TP::NCL;
    const int cap = d.cap;
    uint2 *s_X = (uint2 *)(smem + TP::bead_off(NT));
    float2 *s_vel = (float2 *)(s_X + cap);
    uint32_t *s_id = (uint32_t *)(s_vel + cap);
    float *s_fx = (float *)(s_id + cap);
    float *s_fy = s_fx + cap;
    uint32_t *s_cnt = (uint32_t *)(s_fy + cap);                       // COUNT only
    uint16_t *s_oslot = (uint16_t *)(COUNT ? (void *)(s_cnt + cap) : (void *)s_cnt);
    unsigned char *s_own = (unsigned char *)(s_oslot + cap);

    const int ty = tile / d.ntx, tx = tile - ty * d.ntx;
    const int x0 = tx * B, y0 = ty * B;
    const int tw = min(B, d.nc - x0), th_ = min(B, d.nc - y0);
    const int base = y0 * d.nc + x0 * th_;
    const uint32_t n = (uint32_t)d.n;
    const long long step = *d.step;
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xffffffffull);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
    const uint32_t g0 = min(d.cstart[base], n);
    const uint32_t g1 = max(g0, min(d.cstart[base + tw * th_], n));
    const int n_own = (int)(g1 - g0);

    // bead counts and global sources of the local grid (cells past the halo
    // of a ragged tile stay empty)
    for (int c = tid; c < TP::NCL; c += NT) {
        const int ly = c / W - 1, lx = c - (ly + 1) * W - 1;
        int cnt = 0, src = 0;
        if (lx <= tw && ly <= th_) {
            if (lx >= 0 && lx < tw && ly >= 0 && ly < th_) {
                const int oc = ly * tw + lx;
                const uint32_t b = min(max(d.cstart[base + oc], g0), g1), e = min(max(d.cstart[base + oc + 1], b), g1);
                src = (int)b;
                cnt = (int)(e - b);
            } else {
                int cx = x0 + lx, cy = y0 + ly;
                cx += cx < 0 ? d.nc : (cx >= d.nc ? -d.nc : 0);
                cy += cy < 0 ? d.nc : (cy >= d.nc ? -d.nc : 0);
                const int gc = cell_of<B>(d, cx, cy);
                const uint32_t b = min(d.cstart[gc], n), e = min(max(d.cstart[gc + 1], b), n);
                src = (int)b;
                cnt = (int)(e - b);
            }
        }
        s_lcnt[c] = cnt;
        s_lsrc[c] = src;
    }
    __syncthreads();
    if (tid < 32) {   // exclusive scan of the counts in grid order
        constexpr int PER = (TP::NCL + 31) / 32;
        int v[PER];
        int sum = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int c = tid * PER + i;
            v[i] = c < TP::NCL ? s_lcnt[c] : 0;
            sum += v[i];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += t;
        }
        int run = incl - sum;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int c = tid * PER + i;
            if (c < TP::NCL) s_lbeg[c] = run;
            run += v[i];
        }
        if (tid == 31) {
            s_lbeg[TP::NCL] = incl;
            s_sc[0] = incl;
            s_sc[1] = 0;   // next owned bead for the pair walk
        }
    }
    __syncthreads();
    const int total = s_sc[0];

    if (total <= cap) {
        // ---- stage every bead of the local grid: slot s lies in the last
        // cell whose begin is <= s
        for (int s = tid; s < total; s += NT) {
            int lo = 0, hi = TP::NCL - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_lbeg[mid] <= s) lo = mid; else hi = mid - 1;
            }
            const int c = lo;
            const int ly = c / W - 1, lx = c - (ly + 1) * W - 1;
            const bool owned = lx >= 0 && lx < tw && ly >= 0 && ly < th_;
            const uint32_t g = min((uint32_t)(s_lsrc[c] + (s - s_lbeg[c])), n - 1);
            const uint4 xv = d.S_xv[g];
            s_X[s] = make_uint2(xv.x, xv.y);
            s_vel[s] = make_float2(vbits(xv.z), vbits(xv.w));
            s_id[s] = d.S_id[g];
            s_fx[s] = 0.f;
            s_fy[s] = 0.f;
            if (COUNT) s_cnt[s] = 0u;
            s_own[s] = owned ? 1 : 0;
            if (owned) s_oslot[g - g0] = (uint16_t)s;
        }
        __syncthreads();

        pairs_grid<B, COUNT>(d, n_own, x0, y0, tw, s_lbeg, s_X, s_vel, s_id, s_own, s_oslot, s_fx, s_fy, s_cnt,
                             (uint32_t *)(smem + TP::queue_off(cap, NT, COUNT)) + TP::QLEN * (tid >> 5), s_sc + 1,
                             s_lo, s_hi);
        __syncthreads();

        // ---- integrate owned beads (state read back from shared memory)
        for (int k = tid; k < n_own; k += NT) {
            const int s = s_oslot[k];
            const uint2 x = s_X[s];
            const float2 v = s_vel[s];
            const uint32_t id = s_id[s];
            if (COUNT && d.pcnt) d.pcnt[id] = s_cnt[s];
            integrate_bead<B>(d, (int)g0 + k, make_uint4(x.x, x.y, fbits(v.x), fbits(v.y)), id, s_fx[s], s_fy[s],
                              flags, th);
        }
    } else {
        force_tile_global<B, COUNT>(d, g0, n_own, s_lo, s_hi, flags, th);
    }
}

// Fused force + integrate for one tile.  Thread-per-owned-bead pair search:
// pairs inside the tile are taken once (Newton-3 through shared-memory
// atomics on the partner's slot), pairs with halo beads are taken from the
// owned side only (the neighbouring tile takes the other side with the same
// random number), so every bead's force is complete when the tile finishes
// and the integration runs in the same kernel.  A tile whose beads do not
// fit in shared memory takes the same arithmetic from global memory.
template <int B, bool COUNT, int VAR>
__device__ void force_tile(const Sys &d, int tile, int flags, unsigned char *smem, Thermo3 &th)
{
    if constexpr (VAR == 3) {
        force_tile_g<B, COUNT>(d, tile, flags, smem, th);
        return;
    }
    using TP = TilePlan<B>;
    const int NT = blockDim.x, tid = threadIdx.x;
    int *s_cbeg = (int *)smem;
    int *s_ccnt = s_cbeg + TP::NCL;
    int *s_hg = s_ccnt + TP::NCL;
    int *s_hbeg = s_hg + (TP::NH + 1);
    int *s_hcnt = s_hbeg + (TP::NH + 1);
    int *s_hsx = s_hcnt + (TP::NH + 1);
    int *s_hsy = s_hsx + (TP::NH + 1);
    uint32_t *s_crx = (uint32_t *)(s_hsy + (TP::NH + 1));   // cell corners (fixed point)
    uint32_t *s_cry = s_crx + (B + 2);
    int *s_sc = (int *)(s_cry + (B + 2));
    const int cap = d.cap;
    float2 *s_pos = (float2 *)(smem + TP::bead_off(NT));
    float2 *s_vel = s_pos + cap;
    uint32_t *s_id = (uint32_t *)(s_vel + cap);
    float *s_fx = (float *)(s_id + cap);
    float *s_fy = s_fx + cap;
    unsigned char *s_lc = (unsigned char *)(s_fy + cap);
    uint32_t *s_cnt = (uint32_t *)(smem + ((TP::bead_off(NT) + (size_t)cap * 29 + 3) & ~size_t(3)));  // COUNT only

    const int ty = tile / d.ntx, tx = tile - ty * d.ntx;
    const int x0 = tx * B, y0 = ty * B;
    const int tw = min(B, d.nc - x0), th_ = min(B, d.nc - y0);
    const int base = y0 * d.nc + x0 * th_;
    const int nh = 2 * (tw + 2) + 2 * th_;
    // Each staged bead keeps its offset from its own cell's corner
    // C(c) = ceil(c 2^32 / nc) (exact integer difference, one rounding), so
    // the precision of a pair separation does not depend on the tile size or
    // on L; the separation to a bead in the cell (dcx, dcy) away is
    // off_i - off_j - (dcx, dcy) cs up to one fixed-point unit.
    const uint32_t n = (uint32_t)d.n;
    const long long step = *d.step;
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xffffffffull);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);

    const uint32_t g0 = min(d.cstart[base], n);
    const uint32_t g1 = max(g0, min(d.cstart[base + tw * th_], n));
    const int n_own = (int)(g1 - g0);

    for (int c = tid; c < 2 * (B + 2); c += NT) {
        const int q = c < B + 2 ? c : c - (B + 2);
        int cc = (c < B + 2 ? x0 : y0) + q - 1;
        cc += cc < 0 ? d.nc : (cc >= d.nc ? -d.nc : 0);
        const uint32_t corner = (uint32_t)((((unsigned long long)cc << 32) + (unsigned)d.nc - 1ull) / (unsigned)d.nc);
        if (c < B + 2) s_crx[q] = corner; else s_cry[q] = corner;
    }
    // owned cell table
    for (int c = tid; c < tw * th_; c += NT) {
        const int ly = c / tw, lx = c - ly * tw;
        const uint32_t b = min(max(d.cstart[base + c], g0), g1), e = min(max(d.cstart[base + c + 1], b), g1);
        const int lc = (ly + 1) * (B + 2) + lx + 1;
        s_cbeg[lc] = (int)(b - g0);
        s_ccnt[lc] = (int)(e - b);
    }
    // halo cell table
    for (int h = tid; h < nh; h += NT) {
        int lx, ly;
        if (h < tw + 2) { lx = h - 1; ly = -1; }
        else if (h < 2 * (tw + 2)) { lx = h - (tw + 2) - 1; ly = th_; }
        else if (h < 2 * (tw + 2) + th_) { lx = -1; ly = h - 2 * (tw + 2); }
        else { lx = tw; ly = h - 2 * (tw + 2) - th_; }
        int cx = x0 + lx, cy = y0 + ly, sx = 0, sy = 0;
        if (cx < 0) { cx += d.nc; sx = -1; } else if (cx >= d.nc) { cx -= d.nc; sx = 1; }
        if (cy < 0) { cy += d.nc; sy = -1; } else if (cy >= d.nc) { cy -= d.nc; sy = 1; }
        const int gc = cell_of<B>(d, cx, cy);
        const uint32_t b = min(d.cstart[gc], n), e = min(max(d.cstart[gc + 1], b), n);
        s_hg[h] = (int)b;
        s_hcnt[h] = (int)(e - b);
        s_hsx[h] = sx;
        s_hsy[h] = sy;
    }
    __syncthreads();
    if (tid == 0) {
        int run = n_own;
        for (int h = 0; h < nh; ++h) {
            int lx, ly;
            if (h < tw + 2) { lx = h - 1; ly = -1; }
            else if (h < 2 * (tw + 2)) { lx = h - (tw + 2) - 1; ly = th_; }
            else if (h < 2 * (tw + 2) + th_) { lx = -1; ly = h - 2 * (tw + 2); }
            else { lx = tw; ly = h - 2 * (tw + 2) - th_; }
            const int lc = (ly + 1) * (B + 2) + lx + 1;
            s_hbeg[h] = run;
            s_cbeg[lc] = run;
            s_ccnt[lc] = s_hcnt[h];
            run += s_hcnt[h];
        }
        s_hbeg[nh] = run;
        s_sc[0] = run;
        s_sc[1] = 0;   // next owned bead for the pair queue
    }
    __syncthreads();
    const int total = s_sc[0];

    if (total <= cap) {
        // ---- stage owned + halo beads in shared memory (tile-local frame)
        for (int k = tid; k < n_own; k += NT) {
            const uint4 xv = d.S_xv[g0 + k];
            const int lx = min(max(cell_coord(d, xv.x) - x0, 0), tw - 1);
            const int ly = min(max(cell_coord(d, xv.y) - y0, 0), th_ - 1);
            s_pos[k] = make_float2((float)(int)(xv.x - s_crx[lx + 1]) * d.ulen,
                                   (float)(int)(xv.y - s_cry[ly + 1]) * d.ulen);
            s_vel[k] = make_float2(vbits(xv.z), vbits(xv.w));
            s_id[k] = d.S_id[g0 + k];
            s_fx[k] = 0.f;
            s_fy[k] = 0.f;
            if (COUNT) s_cnt[k] = 0u;
            s_lc[k] = (unsigned char)(lx | (ly << 4));
        }
        for (int k = n_own + tid; k < total; k += NT) {
            int lo = 0, hi = nh - 1;   // last h with hbeg[h] <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_hbeg[mid] <= k) lo = mid; else hi = mid - 1;
            }
            const int h = lo;
            const uint32_t gsrc = (uint32_t)s_hg[h] + (uint32_t)(k - s_hbeg[h]);
            const uint4 xv = d.S_xv[min(gsrc, n - 1)];
            int hx, hy;   // local cell of halo cell h (perimeter order)
            if (h < tw + 2) { hx = h - 1; hy = -1; }
            else if (h < 2 * (tw + 2)) { hx = h - (tw + 2) - 1; hy = th_; }
            else if (h < 2 * (tw + 2) + th_) { hx = -1; hy = h - 2 * (tw + 2); }
            else { hx = tw; hy = h - 2 * (tw + 2) - th_; }
            // the offset from the cell corner is the same for a periodic image
            s_pos[k] = make_float2((float)(int)(xv.x - s_crx[hx + 1]) * d.ulen,
                                   (float)(int)(xv.y - s_cry[hy + 1]) * d.ulen);
            s_vel[k] = make_float2(vbits(xv.z), vbits(xv.w));
            s_id[k] = d.S_id[min(gsrc, n - 1)];
        }
        __syncthreads();

        // ---- pair forces
        if (VAR == 1)
            pairs_thread<B, COUNT>(d, n_own, tw, th_, s_cbeg, s_ccnt, s_pos, s_vel, s_id, s_fx, s_fy, s_cnt, s_lc,
                                   s_lo, s_hi);
        else
            pairs_queue<B, COUNT>(d, n_own, tw, th_, s_cbeg, s_ccnt, s_pos, s_vel, s_id, s_fx, s_fy, s_cnt, s_lc,
                                  (uint32_t *)(smem + TP::queue_off(cap, NT, COUNT)) + 128 * (tid >> 5), s_sc + 1, s_lo,
                                  s_hi);
        __syncthreads();

        // ---- integrate owned beads
        for (int k = tid; k < n_own; k += NT) {
            const int g = (int)g0 + k;
            const uint4 xv = d.S_xv[g];
            const uint32_t id = s_id[k];
            if (COUNT && d.pcnt) d.pcnt[id] = s_cnt[k];
            integrate_bead<B>(d, g, xv, id, s_fx[k], s_fy[k], flags, th);
        }
    } else {
        force_tile_global<B, COUNT>(d, g0, n_own, s_lo, s_hi, flags, th);
    }
}

// Block reduction of the thermo partials into the FP64 ring slot of `step`
// (FP32 inside a warp, FP64 across warps and blocks).
__device__ __forceinline__ void thermo_flush(const Sys &d, Thermo3 th, double *s_red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        th.ke += __shfl_xor_sync(0xffffffffu, th.ke, o);
        th.px += __shfl_xor_sync(0xffffffffu, th.px, o);
        th.py += __shfl_xor_sync(0xffffffffu, th.py, o);
    }
    if (lane == 0) {
        s_red[3 * wid + 0] = (double)th.ke;
        s_red[3 * wid + 1] = (double)th.px;
        s_red[3 * wid + 2] = (double)th.py;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < nw; ++w) { a += s_red[3 * w]; b += s_red[3 * w + 1]; c += s_red[3 * w + 2]; }
        double *t = d.thermo + 4 * (size_t)(*d.step % THERMO_CAP);
        atomicAdd(&t[0], a);
        atomicAdd(&t[1], b);
        atomicAdd(&t[2], c);
    }
}

}  // namespace dpd
