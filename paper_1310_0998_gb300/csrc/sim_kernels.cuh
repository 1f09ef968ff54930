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
// Thermo partials of one thread, FP64: sum |v|^2, sum v_x, sum v_y.
struct Thermo3 { double ke, px, py; };

// Pair forces are summed per bead in fixed point, 2^-24 force units per
// count.  Integer addition is associative, so a bead's force does not depend
// on the order in which its pairs are met (the in-cell order of the counting
// sort comes from atomic tickets and varies from run to run); every FP32 pair
// contribution of magnitude 1/2 or more converts exactly.  In shared memory a
// component is two 32-bit words updated with native integer atomics: hi, the
// count shifted right by 16 (signed), and lo, its low 16 bits (unsigned); the
// sum is hi 2^16 + lo exactly as long as a bead meets fewer than 2^16 pairs and
// its pair forces add up to less than 2^23 in magnitude.  A pair force of
// magnitude FQ_MAX or more (a blown-up state) is reported as non-finite.
constexpr float FQ_SCALE = 16777216.0f;              // 2^24
constexpr float FQ_INV = 5.9604644775390625e-08f;    // 2^-24
constexpr float FQ_MAX = 65536.0f;
__device__ __forceinline__ long long fq(float g) { return __float2ll_rn(__fmul_rn(g, FQ_SCALE)); }
__device__ __forceinline__ float fq_to_f(long long q) { return __fmul_rn(__ll2float_rn(q), FQ_INV); }
// a: the hi word of one force component in shared memory, its lo word `fs`
// words further on
__device__ __forceinline__ void fq_add(int *a, int fs, long long q)
{
    atomicAdd(a, (int)(q >> 16));
    atomicAdd((unsigned *)(a + fs), (unsigned)(q & 0xffffll));
}
__device__ __forceinline__ float fq_load(const int *a, int fs)
{
    return fq_to_f((long long)a[0] * 65536ll + (long long)(unsigned)a[fs]);
}

// Everything after the pair sum for one owned bead at sorted slot g:
// bond + propulsion (partner through slot[id ^ 1]), drag, the two half kicks
// and the drift, canonical output, binning of the new position.
// Every floating-point operation of the step is written with an explicit
// rounding (fused where a fused multiply-add is meant), so that the kernels
// that inline this code, whose flags the compiler may or may not know, all
// produce the same bits.
template <int B>
__device__ __forceinline__ void integrate_bead(const Sys &d, int g, uint4 xv, uint32_t id, float fx, float fy,
                                               int flags, Thermo3 &th)
{
    if (id >= (uint32_t)d.n) {
        set_err_at(d, ERR_INTERNAL, 7, g, id, d.n);
        return;
    }
    const uint32_t ps = d.slot[id ^ 1u];
    if (ps < (uint32_t)d.n) {
        const uint4 xp = d.S_xv[ps];
        const float dx = mdiff(d, xv.x, xp.x);
        const float dy = mdiff(d, xv.y, xp.y);
        const float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        if (r2 > 0.f) {
            const float r = __fsqrt_rn(r2);
            const float inv = __fdiv_rn(1.0f, r);
            const float ex = __fmul_rn(dx, inv), ey = __fmul_rn(dy, inv);   // from partner to self
            const float fb = __fmul_rn(-d.kbond, __fsub_rn(r, d.r0));
            const float sp = (id & 1u) ? -d.fp : d.fp;                        // n_k = head - tail
            fx = __fmaf_rn(__fadd_rn(fb, sp), ex, fx);
            fy = __fmaf_rn(__fadd_rn(fb, sp), ey, fy);
        }
    } else {
        set_err_at(d, ERR_INTERNAL, 2, g, id, ps);
    }
    float vx = vbits(xv.z), vy = vbits(xv.w);
    fx = __fmaf_rn(-d.zeta, vx, fx);
    fy = __fmaf_rn(-d.zeta, vy, fy);
    if (!(flags & F_FIRST)) { vx = __fmaf_rn(d.hdtm, fx, vx); vy = __fmaf_rn(d.hdtm, fy, vy); }
    {
        const double dvx = (double)vx, dvy = (double)vy;
        th.ke = fma(dvx, dvx, fma(dvy, dvy, th.ke));
        th.px += dvx;
        th.py += dvy;
    }
    if (flags & F_FINAL) {
        d.C_xv[id] = make_uint4(xv.x, xv.y, fbits(vx), fbits(vy));
        d.C_f[id] = make_float2(fx, fy);
    }
    if (flags & F_ADVANCE) {
        vx = __fmaf_rn(d.hdtm, fx, vx);
        vy = __fmaf_rn(d.hdtm, fy, vy);
        const float ddx = __fmul_rn(d.dt, vx), ddy = __fmul_rn(d.dt, vy);
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

// ------------------------------------------------------------- pair force ----
// Pair separation in fixed-point units: the exact integer difference of the
// two coordinates, one rounding to FP32.  Negating the pair negates it
// exactly, so a pair evaluated from either bead (or by either of two tiles)
// gives exactly opposite forces, and the range test is the same decision from
// both sides.
__device__ __forceinline__ float sep_u(uint32_t a, uint32_t b) { return (float)(int)(a - b); }
__device__ __forceinline__ float r2_u(float ux, float uy) { return __fmaf_rn(ux, ux, __fmul_rn(uy, uy)); }
// The pair test r < r_c on the FP32 square of the separation in units (every
// kernel and path takes this same decision from the same two positions, so
// the set of interacting pairs is a property of the positions alone).
__device__ __forceinline__ bool in_range(const Sys &d, uint32_t xa, uint32_t ya, uint32_t xb, uint32_t yb)
{
    const float r2u = r2_u(sep_u(xa, xb), sep_u(ya, yb));
    return (r2u < d.rc2u) & (r2u > 0.f);
}

// Scalar F of the pair force F e_ij (Eqs. DPDf, DPDcdr, weightFunc01):
// F = w [a - gamma w (v_ij . e_ij) + sigma alpha_ij / sqrt(dt)], w = 1 - r / r_c,
// e_ij = (x_i - x_j) / r; returns F and e_ij.  Written with explicit roundings
// (no contraction left to the compiler) so that every kernel that inlines it
// produces the same bits.
__device__ __forceinline__ float dpd_pair_scalar(const Sys &d, float ux, float uy, float r2u, float dvx, float dvy,
                                                 uint32_t idi, uint32_t idj, uint32_t s_lo, uint32_t s_hi,
                                                 float &ex, float &ey)
{
    const float rinv = rsqrtf(r2u);
    const float w = __fmaf_rn(-__fmul_rn(r2u, rinv), d.inv_rcu, 1.0f);
    ex = __fmul_rn(ux, rinv);
    ey = __fmul_rn(uy, rinv);
    const float dve = __fmaf_rn(dvx, ex, __fmul_rn(dvy, ey));
    const float nz = pair_noise(d, idi, idj, s_lo, s_hi);
    if (!d.gen_w)
        return __fmul_rn(w, __fmaf_rn(d.sig_r, nz, __fmaf_rn(-__fmul_rn(d.gamma, w), dve, d.a)));
    // changed exponent of w: w_R = w^(s/2), w_D = w_R^2 (uniform branch)
    const float wr = __powf(w, d.hwexp);
    return __fmaf_rn(d.a, w, __fmaf_rn(-__fmul_rn(d.gamma, __fmul_rn(wr, wr)), dve,
                                       __fmul_rn(__fmul_rn(d.sig_r, wr), nz)));
}

// Force of the pair (i, j) on i as fixed-point counts; flags a blown-up pair.
__device__ __forceinline__ void pair_force_q(const Sys &d, uint2 xi, uint2 xj, float2 vi, float2 vj, uint32_t idi,
                                             uint32_t idj, uint32_t s_lo, uint32_t s_hi, long long &qx, long long &qy)
{
    const float ux = sep_u(xi.x, xj.x), uy = sep_u(xi.y, xj.y);
    float ex, ey;
    const float F = dpd_pair_scalar(d, ux, uy, r2_u(ux, uy), __fsub_rn(vi.x, vj.x), __fsub_rn(vi.y, vj.y), idi, idj,
                                    s_lo, s_hi, ex, ey);
    if (!(fabsf(F) < FQ_MAX)) set_err(d, ERR_NONFINITE);
    qx = fq(__fmul_rn(F, ex));
    qy = fq(__fmul_rn(F, ey));
}

// ------------------------------------------------------------ force tile ----
// Shared-memory plan of one tile (B x B owned cells + one-cell halo) for the
// variants that stage owned beads first (1, 2, 4).  Variant 4 adds, per owned
// cell, its merged candidate ranges (FLAT_MAXI at most) and a per-warp table
// of the 32 ranges being enumerated.
constexpr int TILE_THREADS = 128;
constexpr int FLAT_MAXI = 6;
template <int B, int VAR = 2>
struct TilePlan {
    static constexpr int NCL = (B + 2) * (B + 2);   // local cell table
    static constexpr int NH = 4 * B + 4;            // halo cells
    static constexpr int NITEM = (VAR == 4 || VAR == 5) ? B * B * (FLAT_MAXI + 1) : 0;
    static constexpr int NINT = 2 * NCL + 3 * (NH + 1) + 8 + NITEM;
    // queue entries per warp: a drain starts at 32 and a round pushes at most
    // two per lane, so 31 + 64 entries are the most a queue holds
    static constexpr int QLEN = VAR == 4 ? 64 : 96;
    static constexpr int WARP_BYTES = 4 * QLEN + (VAR == 4 ? 16 * 32 : 0);
    static __host__ __device__ size_t red_off() { return ((size_t)NINT * 4 + 7) & ~size_t(7); }
    static __host__ __device__ size_t bead_off(int nthreads)
    {
        return (red_off() + sizeof(double) * 3 * (size_t)(nthreads / 32 + 1) + 15) & ~size_t(15);
    }
    // per staged bead: position 8, velocity 8, force counts 16, id 4,
    // local cell 1 (+ count 4)
    static __host__ __device__ size_t bead_bytes(bool count) { return count ? 41 : 37; }
    static __host__ __device__ size_t queue_off(int cap, int nthreads, bool count)
    {
        return (bead_off(nthreads) + (size_t)cap * bead_bytes(count) + 15) & ~size_t(15);
    }
    // variant 2: per owned cell, its walk descriptor (local cell index, the
    // neighbour cells owned by the tile and the ones it visits), so a lane
    // starting a bead reads it instead of deriving it
    static constexpr bool DESC = VAR == 2;
    static __host__ __device__ size_t desc_off(int cap, int nthreads, bool count)
    {
        return queue_off(cap, nthreads, count) + (size_t)WARP_BYTES * (size_t)(nthreads / 32);
    }
    // variant 2 on 8 x 8 blocks: the order in which the tile's lanes take
    // owned beads (u16 each; measured faster there, slower on 16 x 16)
    static constexpr bool ORDER = VAR == 2 && B == 8;
    static __host__ __device__ size_t order_off(int cap, int nthreads, bool count)
    {
        return desc_off(cap, nthreads, count) + (DESC ? 4 * (size_t)(B * B) : 0);
    }
    static __host__ __device__ size_t bytes(int cap, int nthreads, bool count)
    {
        return order_off(cap, nthreads, count) + (ORDER ? 2 * (size_t)cap : 0);
    }
};

// Shared arrays of a staged tile (variants 1 and 2): cap beads, cap a multiple
// of 32 so every array starts 16-byte aligned.
struct TileArrays {
    uint2 *X;          // fixed-point position
    float2 *v;         // velocity
    int *f;            // force counts, one array per word: x hi, x lo, y hi, y lo
    int fs;            // words per array (the capacity): bead k's words are
                       // f[k], f[fs + k], f[2 fs + k], f[3 fs + k], so the
                       // atomics of a warp's 32 pairs spread over all banks
    uint32_t *id;
    uint32_t *cnt;     // interacting neighbours (COUNT only)
    unsigned char *lc; // local cell (lx | ly << 4) of an owned bead
};

template <int B, int VAR>
__device__ __forceinline__ TileArrays tile_arrays(unsigned char *smem, int cap, int nthreads, bool count)
{
    TileArrays a;
    unsigned char *p = smem + TilePlan<B, VAR>::bead_off(nthreads);
    a.X = (uint2 *)p;
    a.v = (float2 *)(p + 8 * (size_t)cap);
    a.f = (int *)(p + 16 * (size_t)cap);
    a.fs = cap;
    a.id = (uint32_t *)(p + 32 * (size_t)cap);
    a.cnt = (uint32_t *)(p + 36 * (size_t)cap);
    a.lc = p + (count ? 40 : 36) * (size_t)cap;
    return a;
}

// Neighbour offsets packed 2 bits per entry (value + 1), entries in the
// order 0 = own cell, 1-4 ahead (E, NE, N, NW), 5-8 behind (W, SW, S, SE).
constexpr uint32_t NB_DX = 0x1u | (2u << 2) | (2u << 4) | (1u << 6) | (0u << 8) | (0u << 10) | (0u << 12) |
                           (1u << 14) | (2u << 16);
constexpr uint32_t NB_DY = 0x1u | (1u << 2) | (2u << 4) | (2u << 6) | (2u << 8) | (1u << 10) | (0u << 12) |
                           (0u << 14) | (0u << 16);

// Variant 1: one thread per owned bead walks its candidates and evaluates
// each interacting pair in place (divergent; kept as the simple reference
// kernel and as an alternative for the autotuner).
template <int B, bool COUNT>
__device__ __forceinline__ void pairs_thread(const Sys &d, int n_own, int tw, int th_, const int *s_cbeg,
                                             const int *s_ccnt, const TileArrays &t, uint32_t s_lo, uint32_t s_hi)
{
    for (int k = threadIdx.x; k < n_own; k += blockDim.x) {
        const uint2 xi = t.X[k];
        const float2 vi = t.v[k];
        const uint32_t idi = t.id[k], pid = d.excl ? (idi ^ 1u) : 0xffffffffu;
        const int lx = t.lc[k] & 15, ly = t.lc[k] >> 4;
        long long fx = 0, fy = 0;
        uint32_t cnt = 0;
#pragma unroll 1
        for (int nb = 0; nb < 9; ++nb) {
            const int ox_ = (int)((NB_DX >> (2 * nb)) & 3u) - 1, oy_ = (int)((NB_DY >> (2 * nb)) & 3u) - 1;
            const int nlx = lx + ox_, nly = ly + oy_;
            const bool owned = (nlx >= 0 && nlx < tw && nly >= 0 && nly < th_);
            if (nb >= 5 && owned) continue;    // the other bead's forward sweep takes it
            const int lc = (nly + 1) * (B + 2) + nlx + 1;
            int j = s_cbeg[lc];
            const int je = j + s_ccnt[lc];
            if (nb == 0) j = k + 1;
            for (; j < je; ++j) {
                const uint2 xj = t.X[j];
                if (!in_range(d, xi.x, xi.y, xj.x, xj.y)) continue;
                const uint32_t idj = t.id[j];
                if (idj == pid) continue;
                long long qx, qy;
                pair_force_q(d, xi, xj, vi, t.v[j], idi, idj, s_lo, s_hi, qx, qy);
                fx += qx;
                fy += qy;
                if (COUNT) ++cnt;
                if (owned) {
                    fq_add(&t.f[j], t.fs, -qx);
                    fq_add(&t.f[2 * t.fs + j], t.fs, -qy);
                    if (COUNT) atomicAdd(&t.cnt[j], 1u);
                }
            }
        }
        fq_add(&t.f[k], t.fs, fx);
        fq_add(&t.f[2 * t.fs + k], t.fs, fy);
        if (COUNT) atomicAdd(&t.cnt[k], cnt);
    }
}

// Variant 2: pair queue.  Each lane walks the candidates of one owned bead at
// a time (taking the next bead from a block-wide counter when it runs out, so
// warps stay balanced; on 8 x 8 blocks the counter runs through `order`,
// which lists the beads of the cells that also visit halo cells behind them
// first, so that the shortest walks come last and the lanes finish closer
// together); every candidate
// inside r_c is pushed, packed as
// (i, j, Newton-3 flag), into the warp's 128-entry buffer.  Whenever 32 pairs
// are queued the whole warp evaluates them together, so the Philox and force
// arithmetic runs with every lane active.  Forces land in shared memory
// through fixed-point atomics on both sides of a Newton-3 pair.
template <bool COUNT>
__device__ __forceinline__ void queue_eval(const Sys &d, uint32_t code, const TileArrays &t, uint32_t s_lo,
                                           uint32_t s_hi)
{
    const int k = code & 0xfffu, j = (code >> 12) & 0xfffu;
    long long qx, qy;
    pair_force_q(d, t.X[k], t.X[j], t.v[k], t.v[j], t.id[k], t.id[j], s_lo, s_hi, qx, qy);
    fq_add(&t.f[k], t.fs, qx);
    fq_add(&t.f[2 * t.fs + k], t.fs, qy);
    if (COUNT) atomicAdd(&t.cnt[k], 1u);
    if ((code >> 24) & 1u) {
        fq_add(&t.f[j], t.fs, -qx);
        fq_add(&t.f[2 * t.fs + j], t.fs, -qy);
        if (COUNT) atomicAdd(&t.cnt[j], 1u);
    }
}

// Evaluate the oldest 32 entries of a warp queue of qn >= 32 entries (NQ
// entries of capacity beyond the first 32) and move the rest to the front.
template <int NQ, typename EVAL>
__device__ __forceinline__ void queue_drain(volatile uint32_t *q, int &qn, EVAL eval)
{
    const int lane = threadIdx.x & 31;
    while (qn >= 32) {
        const uint32_t mine = q[lane];
        uint32_t carry[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) carry[u] = q[32 * (u + 1) + lane];
        __syncwarp();
#pragma unroll
        for (int u = 0; u < NQ; ++u)
            if (lane + 32 * u < qn - 32) q[lane + 32 * u] = carry[u];
        qn -= 32;
        __syncwarp();
        eval(mine);
    }
}

template <int B, bool COUNT>
__device__ __forceinline__ void pairs_queue(const Sys &d, int n_own, const int *s_cbeg, const int *s_ccnt,
                                            const TileArrays &t, volatile uint32_t *q, int *s_next, uint32_t s_lo,
                                            uint32_t s_hi, const uint32_t *desc, const uint16_t *order)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int k = -1, j = 0, je = 0, lc0 = 0;
    uint32_t visit = 0, own = 0, pid = 0, tag = 0;
    uint2 xi = make_uint2(0u, 0u);
    bool more = true;
    int qn = 0;   // warp-uniform queue length (entries q[0, qn))
    auto eval = [&](uint32_t code) { queue_eval<COUNT>(d, code, t, s_lo, s_hi); };
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
                    if constexpr (TilePlan<B, 2>::ORDER) k = order[k];
                    xi = t.X[k];
                    const uint32_t lcb = t.lc[k];
                    const uint32_t dsc = desc[(lcb >> 4) * B + (lcb & 15u)];
                    lc0 = (int)(dsc & 0x1ffu);
                    own = (dsc >> 9) & 0x1ffu;
                    visit = dsc >> 18;
                    pid = d.excl ? (t.id[k] ^ 1u) : 0xffffffffu;
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
                tag = (uint32_t)k | (((own >> nb) & 1u) << 24);
                have = j < je;
            }
        }
        if (!__any_sync(FULL, have || more)) break;
        // two candidates per lane per round (j and j + 1 while in range),
        // tested branch-free; one append point per round
        bool p0 = false, p1 = false;
        uint32_t c0 = 0, c1 = 0;
        if (have) {
            const uint2 xj = t.X[j];
            p0 = in_range(d, xi.x, xi.y, xj.x, xj.y) & (t.id[j] != pid);
            c0 = tag | ((uint32_t)j << 12);
            ++j;
            if (j < je) {
                const uint2 xk = t.X[j];
                p1 = in_range(d, xi.x, xi.y, xk.x, xk.y) & (t.id[j] != pid);
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
        queue_drain<2>(q, qn, eval);
    }
    __syncwarp();
    if (lane < qn) eval(q[lane]);
}

// Variant 4: flat enumeration.  Every owned cell has a short list of candidate
// ranges of the staged beads, built once per tile: its own cell (a bead starts
// after itself) merged with whatever owned cells follow contiguously (E), the
// row ahead (NW, N, NE, contiguous when owned or all in the top halo row) and
// the halo cells behind, adjacent ranges merged.  Each lane holds one range of
// one bead at a time; the warp concatenates its 32 current ranges (exclusive
// scan of their lengths) and tests the concatenation 32 candidates at a time,
// lane l taking candidate t0 + l, so every lane tests a candidate in every
// round whatever the range lengths.  A lane finds the range that holds its
// candidate from the bit mask of range starts inside the round (an OR across
// the warp) and a popcount.  Pairs inside r_c go through the warp's pair
// queue as in variant 2.  Every shared-memory index the walk derives is
// checked against the tile (a failed check is reported and the candidate
// dropped).
template <int B>
__device__ __forceinline__ void flat_cell_items(const Sys &d, int tw, int th_, int n_own, const int *s_cbeg,
                                                const int *s_ccnt, int *s_nit, uint32_t *s_items)
{
    for (int oc = threadIdx.x; oc < tw * th_; oc += blockDim.x) {
        const int ly = oc / tw, lx = oc - ly * tw;
        // keys (begin << 14) | (end << 1) | newton of the visited neighbour
        // cells; the own cell stays first (it has the lowest begin of the
        // owned cells, and halo beads are staged after all owned ones)
        uint32_t own = 0, key[8];
#pragma unroll
        for (int nb = 0; nb < 9; ++nb) {
            const int ox_ = (int)((NB_DX >> (2 * nb)) & 3u) - 1, oy_ = (int)((NB_DY >> (2 * nb)) & 3u) - 1;
            const int nlx = lx + ox_, nly = ly + oy_;
            const bool owned = (nlx >= 0 && nlx < tw && nly >= 0 && nly < th_);
            const int lc = (nly + 1) * (B + 2) + nlx + 1;
            const uint32_t b = (uint32_t)s_cbeg[lc], e = b + (uint32_t)s_ccnt[lc];
            const uint32_t k = (b << 14) | (e << 1) | (owned ? 1u : 0u);
            if (nb == 0) own = k;
            else key[nb - 1] = (nb >= 5 && owned) ? 0xffffffffu : k;   // behind: only halo cells
        }
        // sort the eight neighbour keys by begin (Batcher's network)
#define DPD_CE(a, b)                                                   \
        { const uint32_t lo_ = min(key[a], key[b]), hi_ = max(key[a], key[b]); key[a] = lo_; key[b] = hi_; }
        DPD_CE(0, 1) DPD_CE(2, 3) DPD_CE(4, 5) DPD_CE(6, 7)
        DPD_CE(0, 2) DPD_CE(1, 3) DPD_CE(4, 6) DPD_CE(5, 7)
        DPD_CE(1, 2) DPD_CE(5, 6)
        DPD_CE(0, 4) DPD_CE(1, 5) DPD_CE(2, 6) DPD_CE(3, 7)
        DPD_CE(2, 4) DPD_CE(3, 5)
        DPD_CE(1, 2) DPD_CE(3, 4) DPD_CE(5, 6)
#undef DPD_CE
        // merge ranges that continue each other with the same Newton-3 side
        uint32_t cb = own >> 14, ce = (own >> 1) & 0x1fffu, cn = own & 1u;
        int m = 0;
        bool first = true;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t k = key[i];
            if (k == 0xffffffffu) continue;
            const uint32_t b = k >> 14, e = (k >> 1) & 0x1fffu, nw = k & 1u;
            if (b == ce && nw == cn) { ce = e; continue; }
            if (e == b) continue;
            if (first || ce > cb) {
                if (m < FLAT_MAXI) s_items[oc * FLAT_MAXI + m] = cb | (ce << 13) | (cn << 26);
                ++m;
            }
            first = false;
            cb = b; ce = e; cn = nw;
        }
        if (first || ce > cb) {
            if (m < FLAT_MAXI) s_items[oc * FLAT_MAXI + m] = cb | (ce << 13) | (cn << 26);
            ++m;
        }
        if (m > FLAT_MAXI) set_err_at(d, ERR_INTERNAL, 5, oc, m, n_own);
        s_nit[oc] = min(m, FLAT_MAXI);
    }
}

template <bool COUNT>
__device__ __forceinline__ void pairs_flat(const Sys &d, int n_own, int total, int tw, const TileArrays &t,
                                           const int *s_nit, const uint32_t *s_items, uint4 *rec,
                                           volatile uint32_t *q, int *s_next, uint32_t s_lo, uint32_t s_hi)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u, le = (2u << lane) - 1u;
    int k = 0, ii = 0, ni = 0, oc = 0;
    uint32_t b = 0, e = 0, nw = 0, pid = 0;
    uint2 xi = make_uint2(0u, 0u);
    bool more = true;
    int qn = 0;   // warp-uniform queue length
    auto eval = [&](uint32_t code) { queue_eval<COUNT>(d, code, t, s_lo, s_hi); };
    while (true) {
        // this lane's next non-empty range (at most FLAT_MAXI + 1 per bead)
        while (more && b >= e) {
            if (ii >= ni) {
                k = atomicAdd(s_next, 1);
                if (k >= n_own) { more = false; break; }
                const uint32_t lc = t.lc[k];
                oc = (int)(lc >> 4) * tw + (int)(lc & 15u);
                ni = s_nit[oc];
                ii = 0;
                xi = t.X[k];
                pid = d.excl ? (t.id[k] ^ 1u) : 0xffffffffu;
            }
            const uint32_t it = s_items[oc * FLAT_MAXI + min(ii, FLAT_MAXI - 1)];
            b = ii == 0 ? (uint32_t)k + 1u : (it & 0x1fffu);
            e = (it >> 13) & 0x1fffu;
            nw = (it >> 26) & 1u;
            ++ii;
        }
        const uint32_t len = b < e ? e - b : 0u;
        const unsigned ne = __ballot_sync(FULL, len > 0u);
        if (ne == 0u) break;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t start = incl - len, T = __shfl_sync(FULL, incl, 31);
        // ranges in rank order: bead position, exclusion id, and
        // (bead slot | Newton-3 flag << 12 | (range begin - start) << 13)
        if (len > 0u)
            rec[__popc(ne & lt)] = make_uint4(xi.x, xi.y, pid, (uint32_t)k | (nw << 12) | ((b - start) << 13));
        __syncwarp();
        int c0 = 0;   // ranges that start before this round
        for (uint32_t t0 = 0; t0 < T; t0 += 32u) {
            const bool inb = (len > 0u) & (start >= t0) & (start < t0 + 32u);
            // OR of the start bits across the warp (a shuffle butterfly: the
            // warp OR-reduction instruction gave wrong masks in this loop)
            unsigned M = inb ? (1u << (start - t0)) : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) M |= __shfl_xor_sync(FULL, M, o);
            const int r = c0 + __popc(M & le) - 1;
            c0 += __popc(M);
            const uint32_t f = t0 + (uint32_t)lane;
            bool p = false;
            uint32_t code = 0;
            if (f < T) {
                const uint4 rc = rec[r & 31];
                const uint32_t j = f + (uint32_t)((int)rc.w >> 13);
                if (r >= 0 && r < 32 && j < (uint32_t)total && (rc.w & 0xfffu) < (uint32_t)n_own) {
                    const uint2 xj = t.X[j];
                    p = in_range(d, rc.x, rc.y, xj.x, xj.y) & (t.id[j] != rc.z);
                    code = (rc.w & 0xfffu) | (j << 12) | (((rc.w >> 12) & 1u) << 24);
                } else {
                    set_err_at(d, ERR_INTERNAL, 6, r, (long long)j, total);
                }
            }
            const unsigned m = __ballot_sync(FULL, p);
            if (p) q[qn + __popc(m & lt)] = code;
            qn += __popc(m);
            __syncwarp();
            queue_drain<1>(q, qn, eval);
        }
        b = e;
        __syncwarp();
    }
    __syncwarp();
    if (lane < qn) eval(q[lane]);
}

// Variant 5: the lane walk of variant 2 over the merged candidate ranges of
// variant 4's cell tables.  A lane holds one range of one bead; when it runs
// out it takes the next range of its bead (or the next bead), one step per
// round, so a bead costs about 2.3 range switches instead of one per
// neighbour cell; every round each lane tests CPR candidates and the pairs
// inside r_c go through the warp queue.
template <bool COUNT, int CPR>
__device__ __forceinline__ void pairs_items(const Sys &d, int n_own, int total, int tw, const TileArrays &t,
                                            const int *s_nit, const uint32_t *s_items, volatile uint32_t *q,
                                            int *s_next, uint32_t s_lo, uint32_t s_hi)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int k = 0, ii = 0, ni = 0, oc = 0;
    uint32_t j = 0, je = 0, tag = 0, pid = 0;
    uint2 xi = make_uint2(0u, 0u);
    bool more = true;
    int qn = 0;   // warp-uniform queue length
    auto eval = [&](uint32_t code) { queue_eval<COUNT>(d, code, t, s_lo, s_hi); };
    while (true) {
        bool have = j < je;
        if (!have && more) {
            if (ii >= ni) {
                k = atomicAdd(s_next, 1);
                if (k >= n_own) {
                    more = false;
                } else {
                    const uint32_t lc = t.lc[k];
                    oc = (int)(lc >> 4) * tw + (int)(lc & 15u);
                    ni = s_nit[oc];
                    ii = 0;
                    xi = t.X[k];
                    pid = d.excl ? (t.id[k] ^ 1u) : 0xffffffffu;
                }
            }
            if (more) {
                const uint32_t it = s_items[oc * FLAT_MAXI + min(ii, FLAT_MAXI - 1)];
                j = ii == 0 ? (uint32_t)k + 1u : (it & 0x1fffu);
                je = min((it >> 13) & 0x1fffu, (uint32_t)total);
                tag = (uint32_t)k | (((it >> 26) & 1u) << 24);
                ++ii;
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
                const uint2 xj = t.X[j];
                p[u] = in_range(d, xi.x, xi.y, xj.x, xj.y) & (t.id[j] != pid);
                c[u] = tag | (j << 12);
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
        queue_drain<CPR>(q, qn, eval);
    }
    __syncwarp();
    if (lane < qn) eval(q[lane]);
}

// Global-memory path for a tile whose beads do not fit in shared memory: one
// thread per owned bead, pairs from both sides (no Newton-3), the same pair
// arithmetic and fixed-point sums, hence the same bits as the shared path.
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
        const uint2 xi = make_uint2(xv.x, xv.y);
        const float2 vi = make_float2(vbits(xv.z), vbits(xv.w));
        const uint32_t idi = d.S_id[g], pid = d.excl ? (idi ^ 1u) : 0xffffffffu;
        const int cx = cell_coord(d, xv.x), cy = cell_coord(d, xv.y);
        long long fx = 0, fy = 0;
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
                    if (!in_range(d, xv.x, xv.y, xj.x, xj.y)) continue;
                    long long qx, qy;
                    pair_force_q(d, xi, make_uint2(xj.x, xj.y), vi, make_float2(vbits(xj.z), vbits(xj.w)), idi, idj,
                                 s_lo, s_hi, qx, qy);
                    fx += qx;
                    fy += qy;
                    if (COUNT) ++cnt;
                }
            }
        if (COUNT && d.pcnt) d.pcnt[idi] = cnt;
        integrate_bead<B>(d, g, xv, idi, fq_to_f(fx), fq_to_f(fy), flags, th);
    }
}

// ------------------------------------------------- grid-order tile (VAR 3) --
// The tile's owned and halo cells are staged in shared memory in the row-major
// order of the local (B+2) x (B+2) cell grid, so every row of the local grid is
// one contiguous bead range.  The forward half-stencil of an owned cell (own
// cell after the bead, E, and NW..NE) is then two ranges instead of five; a
// cell on the tile edge adds at most three ranges of halo cells behind it (W,
// and SW..SE or parts of that row).  Each lane walks the candidates of one
// owned bead at a time, CPR candidates per round; pairs inside r_c go through
// the warp's pair queue as in variant 2 (Newton-3 when the partner is owned).
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
    // per staged bead: position 8, velocity 8, force counts 16, id 4,
    // (count 4), owned-bead slot 2, owned flag 1
    static __host__ __device__ size_t bead_bytes(bool count) { return count ? 43 : 39; }
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
__device__ __forceinline__ void queue_eval_g(const Sys &d, uint32_t code, const TileArrays &t,
                                             const unsigned char *s_own, uint32_t s_lo, uint32_t s_hi)
{
    const int k = code & 0xfffu, j = (code >> 12) & 0xfffu;
    long long qx, qy;
    pair_force_q(d, t.X[k], t.X[j], t.v[k], t.v[j], t.id[k], t.id[j], s_lo, s_hi, qx, qy);
    fq_add(&t.f[k], t.fs, qx);
    fq_add(&t.f[2 * t.fs + k], t.fs, qy);
    if (COUNT) atomicAdd(&t.cnt[k], 1u);
    if (s_own[j]) {
        fq_add(&t.f[j], t.fs, -qx);
        fq_add(&t.f[2 * t.fs + j], t.fs, -qy);
        if (COUNT) atomicAdd(&t.cnt[j], 1u);
    }
}

template <int B, bool COUNT>
__device__ __forceinline__ void pairs_grid(const Sys &d, int n_own, int x0, int y0, int tw, const int *s_lbeg,
                                           const TileArrays &t, const unsigned char *s_own, const uint16_t *s_oslot,
                                           volatile uint32_t *q, int *s_next, uint32_t s_lo, uint32_t s_hi)
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
    auto eval = [&](uint32_t code) { queue_eval_g<COUNT>(d, code, t, s_own, s_lo, s_hi); };
    while (true) {
        bool have = j < je;
        if (!have && more) {
            if (stage >= 5) {
                const int k = atomicAdd(s_next, 1);
                if (k >= n_own) {
                    more = false;
                } else {
                    si = s_oslot[k];
                    const uint2 x = t.X[si];
                    Xi = x.x;
                    Yi = x.y;
                    pid = d.excl ? (t.id[si] ^ 1u) : 0xffffffffu;
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
                const uint2 xj = t.X[j];
                p[u] = in_range(d, Xi, Yi, xj.x, xj.y) & (t.id[j] != pid);
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
        queue_drain<CPR>(q, qn, eval);
    }
    __syncwarp();
    if (lane < qn) eval(q[lane]);
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
    TileArrays t;
    {
        unsigned char *p = smem + TP::bead_off(NT);
        t.X = (uint2 *)p;
        t.v = (float2 *)(p + 8 * (size_t)cap);
        t.f = (int *)(p + 16 * (size_t)cap);
        t.fs = cap;
        t.id = (uint32_t *)(p + 32 * (size_t)cap);
        t.cnt = (uint32_t *)(p + 36 * (size_t)cap);   // COUNT only
        t.lc = nullptr;
    }
    uint16_t *s_oslot = (uint16_t *)(smem + TP::bead_off(NT) + (COUNT ? 40 : 36) * (size_t)cap);
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
            const int tt = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += tt;
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
            t.X[s] = make_uint2(xv.x, xv.y);
            t.v[s] = make_float2(vbits(xv.z), vbits(xv.w));
            t.id[s] = d.S_id[g];
            t.f[s] = 0;
            t.f[t.fs + s] = 0;
            t.f[2 * t.fs + s] = 0;
            t.f[3 * t.fs + s] = 0;
            if (COUNT) t.cnt[s] = 0u;
            s_own[s] = owned ? 1 : 0;
            if (owned) s_oslot[g - g0] = (uint16_t)s;
        }
        __syncthreads();

        pairs_grid<B, COUNT>(d, n_own, x0, y0, tw, s_lbeg, t, s_own, s_oslot,
                             (uint32_t *)(smem + TP::queue_off(cap, NT, COUNT)) + TP::QLEN * (tid >> 5), s_sc + 1,
                             s_lo, s_hi);
        __syncthreads();

        // ---- integrate owned beads (state read back from shared memory)
        for (int k = tid; k < n_own; k += NT) {
            const int s = s_oslot[k];
            const uint2 x = t.X[s];
            const float2 v = t.v[s];
            const uint32_t id = t.id[s];
            if (COUNT && d.pcnt) d.pcnt[id] = t.cnt[s];
            integrate_bead<B>(d, (int)g0 + k, make_uint4(x.x, x.y, fbits(v.x), fbits(v.y)), id,
                              fq_load(&t.f[s], t.fs), fq_load(&t.f[2 * t.fs + s], t.fs), flags, th);
        }
    } else {
        force_tile_global<B, COUNT>(d, g0, n_own, s_lo, s_hi, flags, th);
    }
}

// Fused force + integrate for one tile.  Pairs inside the tile are taken once
// (Newton-3 through shared-memory atomics on the partner's slot), pairs with
// halo beads are taken from the owned side only (the neighbouring tile takes
// the other side and gets exactly the opposite force), so every bead's force
// is complete when the tile finishes and the integration runs in the same
// kernel.  A tile whose beads do not fit in shared memory takes the same
// arithmetic from global memory.
template <int B, bool COUNT, int VAR>
__device__ void force_tile(const Sys &d, int tile, int flags, unsigned char *smem, Thermo3 &th)
{
    if constexpr (VAR == 3) {
        force_tile_g<B, COUNT>(d, tile, flags, smem, th);
        return;
    }
    using TP = TilePlan<B, VAR>;
    const int NT = blockDim.x, tid = threadIdx.x;
    int *s_cbeg = (int *)smem;
    int *s_ccnt = s_cbeg + TP::NCL;
    int *s_hg = s_ccnt + TP::NCL;
    int *s_hbeg = s_hg + (TP::NH + 1);
    int *s_hcnt = s_hbeg + (TP::NH + 1);
    int *s_sc = s_hcnt + (TP::NH + 1);
    int *s_nit = s_sc + 8;                            // variant 4: ranges per owned cell
    uint32_t *s_items = (uint32_t *)(s_nit + B * B);  // variant 4: the ranges
    const int cap = d.cap;
    const TileArrays t = tile_arrays<B, VAR>(smem, cap, NT, COUNT);
    uint16_t *s_order = (uint16_t *)(smem + TP::order_off(cap, NT, COUNT));   // variant 2
    uint32_t *s_desc = (uint32_t *)(smem + TP::desc_off(cap, NT, COUNT));     // variant 2

    const int ty = tile / d.ntx, tx = tile - ty * d.ntx;
    const int x0 = tx * B, y0 = ty * B;
    const int tw = min(B, d.nc - x0), th_ = min(B, d.nc - y0);
    const int base = y0 * d.nc + x0 * th_;
    const int nh = 2 * (tw + 2) + 2 * th_;
    const uint32_t n = (uint32_t)d.n;
    const long long step = *d.step;
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xffffffffull);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);

    const uint32_t g0 = min(d.cstart[base], n);
    const uint32_t g1 = max(g0, min(d.cstart[base + tw * th_], n));
    const int n_own = (int)(g1 - g0);

    // owned cell table (and, for variant 2, each owned cell's walk
    // descriptor: local cell index, the neighbour cells the tile owns (the
    // Newton-3 side) and the ones to visit (ahead always, behind only when
    // halo))
    for (int c = tid; c < tw * th_; c += NT) {
        const int ly = c / tw, lx = c - ly * tw;
        const uint32_t b = min(max(d.cstart[base + c], g0), g1), e = min(max(d.cstart[base + c + 1], b), g1);
        const int lc = (ly + 1) * (B + 2) + lx + 1;
        s_cbeg[lc] = (int)(b - g0);
        s_ccnt[lc] = (int)(e - b);
        if constexpr (TP::DESC) {
            const uint32_t px = lx < tw - 1, nx = lx > 0, py = ly < th_ - 1, ny = ly > 0;
            const uint32_t own = 1u | (px << 1) | ((px & py) << 2) | (py << 3) | ((nx & py) << 4) | (nx << 5) |
                                 ((nx & ny) << 6) | (ny << 7) | ((px & ny) << 8);
            s_desc[ly * B + lx] = (uint32_t)lc | (own << 9) | ((0x1fu | (~own & 0x1e0u)) << 18);
        }
    }
    // halo cell table
    for (int h = tid; h < nh; h += NT) {
        int lx, ly;
        if (h < tw + 2) { lx = h - 1; ly = -1; }
        else if (h < 2 * (tw + 2)) { lx = h - (tw + 2) - 1; ly = th_; }
        else if (h < 2 * (tw + 2) + th_) { lx = -1; ly = h - 2 * (tw + 2); }
        else { lx = tw; ly = h - 2 * (tw + 2) - th_; }
        int cx = x0 + lx, cy = y0 + ly;
        cx += cx < 0 ? d.nc : (cx >= d.nc ? -d.nc : 0);
        cy += cy < 0 ? d.nc : (cy >= d.nc ? -d.nc : 0);
        const int gc = cell_of<B>(d, cx, cy);
        const uint32_t b = min(d.cstart[gc], n), e = min(max(d.cstart[gc + 1], b), n);
        s_hg[h] = (int)b;
        s_hcnt[h] = (int)(e - b);
    }
    __syncthreads();
    // halo cells staged after the owned beads: exclusive scan of their
    // populations by warp 0 (at most 4 B + 4 = 68 cells, three per lane)
    if (tid < 32) {
        const int per = (nh + 31) / 32;
        int local = 0;
        for (int u = 0; u < per; ++u) {
            const int h = tid * per + u;
            if (h < nh) local += s_hcnt[h];
        }
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int w = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += w;
        }
        int run = n_own + incl - local;
        for (int u = 0; u < per; ++u) {
            const int h = tid * per + u;
            if (h < nh) {
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
        }
        if (tid == 31) {
            s_hbeg[nh] = n_own + incl;
            s_sc[0] = n_own + incl;
            s_sc[1] = 0;   // next owned bead for the pair queue
            s_sc[2] = 0;   // variant 2 order: beads placed from the front
            s_sc[3] = 0;   // and from the back
        }
    }
    __syncthreads();
    const int total = s_sc[0];

    if (total <= cap) {
        // ---- stage owned + halo beads in shared memory (raw fixed point:
        // a periodic image has the same coordinates modulo 2^32)
        for (int k = tid; k < n_own; k += NT) {
            const uint4 xv = d.S_xv[g0 + k];
            const int lx = min(max(cell_coord(d, xv.x) - x0, 0), tw - 1);
            const int ly = min(max(cell_coord(d, xv.y) - y0, 0), th_ - 1);
            t.X[k] = make_uint2(xv.x, xv.y);
            t.v[k] = make_float2(vbits(xv.z), vbits(xv.w));
            t.id[k] = d.S_id[g0 + k];
            t.f[k] = 0;
            t.f[t.fs + k] = 0;
            t.f[2 * t.fs + k] = 0;
            t.f[3 * t.fs + k] = 0;
            if (COUNT) t.cnt[k] = 0u;
            t.lc[k] = (unsigned char)(lx | (ly << 4));
            if constexpr (TP::ORDER) {
                // cells whose walk also visits halo cells behind them (left
                // column, bottom row, right column) have the longest walks
                if (lx == 0 || ly == 0 || lx == tw - 1) s_order[atomicAdd(&s_sc[2], 1)] = (uint16_t)k;
                else s_order[n_own - 1 - atomicAdd(&s_sc[3], 1)] = (uint16_t)k;
            }
        }
        for (int k = n_own + tid; k < total; k += NT) {
            int lo = 0, hi = nh - 1;   // last h with hbeg[h] <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_hbeg[mid] <= k) lo = mid; else hi = mid - 1;
            }
            const int h = lo;
            const uint32_t gsrc = min((uint32_t)s_hg[h] + (uint32_t)(k - s_hbeg[h]), n - 1);
            const uint4 xv = d.S_xv[gsrc];
            t.X[k] = make_uint2(xv.x, xv.y);
            t.v[k] = make_float2(vbits(xv.z), vbits(xv.w));
            t.id[k] = d.S_id[gsrc];
        }
        __syncthreads();

        // ---- pair forces
        unsigned char *wbuf = smem + TP::queue_off(cap, NT, COUNT) + (size_t)TP::WARP_BYTES * (tid >> 5);
        if constexpr (VAR == 1) {
            pairs_thread<B, COUNT>(d, n_own, tw, th_, s_cbeg, s_ccnt, t, s_lo, s_hi);
        } else if constexpr (VAR == 4) {
            flat_cell_items<B>(d, tw, th_, n_own, s_cbeg, s_ccnt, s_nit, s_items);
            __syncthreads();
            pairs_flat<COUNT>(d, n_own, total, tw, t, s_nit, s_items, (uint4 *)wbuf, (uint32_t *)(wbuf + 16 * 32),
                              s_sc + 1, s_lo, s_hi);
        } else if constexpr (VAR == 5) {
            flat_cell_items<B>(d, tw, th_, n_own, s_cbeg, s_ccnt, s_nit, s_items);
            __syncthreads();
            pairs_items<COUNT, 2>(d, n_own, total, tw, t, s_nit, s_items, (uint32_t *)wbuf, s_sc + 1, s_lo, s_hi);
        } else {
            pairs_queue<B, COUNT>(d, n_own, s_cbeg, s_ccnt, t, (uint32_t *)wbuf, s_sc + 1, s_lo, s_hi, s_desc,
                                  s_order);
        }
        __syncthreads();

        // ---- integrate owned beads
        for (int k = tid; k < n_own; k += NT) {
            const int g = (int)g0 + k;
            const uint4 xv = d.S_xv[g];
            const uint32_t id = t.id[k];
            if (COUNT && d.pcnt && id < (uint32_t)d.n) d.pcnt[id] = t.cnt[k];
            integrate_bead<B>(d, g, xv, id, fq_load(&t.f[k], t.fs), fq_load(&t.f[2 * t.fs + k], t.fs), flags, th);
        }
    } else {
        force_tile_global<B, COUNT>(d, g0, n_own, s_lo, s_hi, flags, th);
    }
}

// Shared-memory offset of a buffer of 3 x TILE_THREADS doubles that is free
// once a tile's integration has finished (the staged bead arrays).
template <int B, int VAR>
__host__ __device__ inline size_t tile_flush_off()
{
    if constexpr (VAR == 3) return TilePlanG<B>::bead_off(TILE_THREADS);
    else return TilePlan<B, VAR>::bead_off(TILE_THREADS);
}

// Block reduction of a tile's thermo partials into the FP64 ring slot of
// `step` (FP64 throughout): every thread's partials to shared memory (buf,
// 3 blockDim doubles), then warp q adds quantity q (blockDim / 32 values per
// lane, then across its lanes) and adds it to the slot.  A third of the FP64
// additions of a shuffle tree in every warp (the FP64 pipe is narrow on this
// part).  buf is read by warps 0-2 after the call: the caller synchronises
// before reusing it.
__device__ __forceinline__ void thermo_flush_tile(const Sys &d, Thermo3 th, double *buf)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
    buf[tid] = th.ke;
    buf[nt + tid] = th.px;
    buf[2 * nt + tid] = th.py;
    __syncthreads();
    if (wid < 3) {
        double a = 0.0;
        for (int i = lane; i < nt; i += 32) a += buf[wid * nt + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) atomicAdd(&d.thermo[4 * (size_t)(*d.step % THERMO_CAP) + wid], a);
    }
}

// Block reduction of the thermo partials into the FP64 ring slot of `step`
// (FP64 throughout: per thread, across the warp, across warps and blocks).
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
        s_red[3 * wid + 0] = th.ke;
        s_red[3 * wid + 1] = th.px;
        s_red[3 * wid + 2] = th.py;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < nw; ++w) { a += s_red[3 * w]; b += s_red[3 * w + 1]; c += s_red[3 * w + 2]; }
        double *tt = d.thermo + 4 * (size_t)(*d.step % THERMO_CAP);
        atomicAdd(&tt[0], a);
        atomicAdd(&tt[1], b);
        atomicAdd(&tt[2], c);
    }
}

}  // namespace dpd
