// Three-dimensional variant of the simulator (include/dpd.h, dpd3_*).
//
// Sec. 2 states every force as a vector law, so the pair force (Eqs. DPDf,
// DPDcdr, weightFunc01), the bond (Eq. stiffSpring), propulsion and drag
// (Eq. DPDnp) and the velocity-Verlet step of Sec. 5 carry over to a periodic
// cube unchanged; only the geometry is new.  Positions are 32-bit fixed point
// per axis as in two dimensions (uniform resolution, wrap by overflow, exact
// minimum image and cell index).
//
// Layout (N beads, n_c^3 cells numbered (z n_c + y) n_c + x):
//   S_p  uint4[N]   (X, Y, Z, id) of the pre-force state, sorted by cell
//   S_v  float4[N]  the half-step velocity v_{s-1/2} (v_s at set-up)
//   U_p, U_v, U_rank  the next pre-force state in the order of S, with each
//                     bead's rank inside its new cell (atomic ticket)
//   slot u32[N]     id -> sorted slot (the bonded partner of bead id is id^1)
//   counts, cstart  cell populations and their exclusive scan (the same
//                   decoupled look-back scan as the 2D path)
//   C_p, C_v, C_f   canonical (X_s, v_s, f_s) in id order after each call
//   F    s64[N][4]  pair-force sums of the current step by sorted slot, in
//                   fixed point (2^-24 force units per count, as the 2D
//                   path), kept zero between steps
// One step: scan, scatter, pair forces, integration.  The pair kernel gives
// one thread per bead the half stencil (the rest of its cell and the 13
// cells ahead of it), so every pair inside r_c is evaluated once; the pairs
// go through a warp queue so that their arithmetic runs on full warps, the
// force lands on the owner through shared memory and its reaction on the
// partner through 64-bit integer atomics into F (sorted order).  Every sum is
// in fixed point, so it does not depend on the order in which pairs are met
// and a run is reproducible bit for bit.  The integration kernel reads and
// clears F, adds bond, propulsion and drag, does the second half-kick, the
// FP64 thermo partials, the next half-kick and drift, and bins the new
// position.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dpd.h"
#include "sim_host.h"
#include "sim3d_host.h"
#include "sim_kernels.cuh"

namespace dpd {


__device__ __forceinline__ int cell3(const Sys &d, uint32_t X, uint32_t Y, uint32_t Z)
{
    return (cell_coord(d, Z) * d.nc + cell_coord(d, Y)) * d.nc + cell_coord(d, X);
}

__global__ void __launch_bounds__(SCAN_NT) k3_scan(Sys d, int nblocks)
{
    __shared__ uint32_t s_buf[SCAN_BUF];
    scan_decoupled_t<SCAN_NT>(d, nblocks, s_buf);
}

__global__ void k3_bin(Sys3 s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.b.n) return;
    const uint4 p = s.U_p[k];
    s.U_rank[k] = atomicAdd(&s.b.counts[cell3(s.b, p.x, p.y, p.z)], 1u);
}

__global__ void k3_scatter(Sys3 s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.b.n) return;
    const uint4 p = s.U_p[k];
    const uint32_t dst = s.b.cstart[cell3(s.b, p.x, p.y, p.z)] + s.U_rank[k];
    if (dst >= (uint32_t)s.b.n || p.w >= (uint32_t)s.b.n) {
        set_err_at(s.b, ERR_INTERNAL, 11, k, dst, p.w);
        return;
    }
    s.S_p[dst] = p;
    s.S_v[dst] = s.U_v[k];
    s.slot[p.w] = dst;
    const Sys &d = s.b;
    s.S_off[dst] = make_float4((float)(int)(p.x - s.corner[cell_coord(d, p.x)]) * d.ulen,
                               (float)(int)(p.y - s.corner[cell_coord(d, p.y)]) * d.ulen,
                               (float)(int)(p.z - s.corner[cell_coord(d, p.z)]) * d.ulen, __uint_as_float(p.w));
}

// Double positions [N][3] and float velocities [N][3] (id order) -> U.
__global__ void k3_load(Sys3 s, const double *__restrict__ x, const float *__restrict__ v)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.b.n) return;
    uint32_t X[3];
    bool ok = true;
    for (int c = 0; c < 3; ++c) {
        const double u = x[3 * k + c] * s.b.inv_ulen_d;
        if (!(fabs(u) < 4503599627370496.0)) { ok = false; X[c] = 0u; }
        else X[c] = (uint32_t)(unsigned long long)llrint(u);
    }
    float4 vv = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], 0.f);
    if (!isfinite(vv.x) || !isfinite(vv.y) || !isfinite(vv.z)) ok = false;
    if (!ok) {
        set_err(s.b, ERR_NONFINITE);
        vv = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    s.U_p[k] = make_uint4(X[0], X[1], X[2], (uint32_t)k);
    s.U_v[k] = vv;
}

__global__ void k3_store(Sys3 s, double *__restrict__ x, float *__restrict__ v, float *__restrict__ f)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.b.n) return;
    const uint4 p = s.C_p[k];
    const float4 vv = s.C_v[k], ff = s.C_f[k];
    x[3 * k] = (double)p.x * s.b.ulen_d;
    x[3 * k + 1] = (double)p.y * s.b.ulen_d;
    x[3 * k + 2] = (double)p.z * s.b.ulen_d;
    v[3 * k] = vv.x; v[3 * k + 1] = vv.y; v[3 * k + 2] = vv.z;
    f[3 * k] = ff.x; f[3 * k + 1] = ff.y; f[3 * k + 2] = ff.z;
}

__global__ void k3_set_step(Sys d, long long s) { *d.step = s; }

// Pair force magnitude along e (as the 2D pair term, with dv.e in 3D).
__device__ __forceinline__ float pair_scalar3(const Sys &d, float r2, float rinv, float dve, uint32_t ia,
                                              uint32_t ib, uint32_t s_lo, uint32_t s_hi)
{
    const float r = r2 * rinv;
    const float w = 1.0f - r * d.inv_rc;
    const float nz = pair_noise(d, ia, ib, s_lo, s_hi);
    if (!d.gen_w) return w * (d.a - d.gamma * w * dve + d.sig_r * nz);
    const float wr = __powf(w, d.hwexp);
    return d.a * w - d.gamma * (wr * wr) * dve + d.sig_r * wr * nz;
}

// One queued pair (sorted slot q, owner lane o of this warp): the pair force
// on the owner, accumulated in shared memory ((hi, lo) words per component,
// as the 2D tile), and its reaction on q, added to q's 64-bit sums in global
// memory (Newton-3: every pair is evaluated once).
__device__ __forceinline__ void eval3(const Sys3 &s, uint32_t q, int o, const uint4 *pis, const float4 *vis,
                                      int (*fs)[6], uint32_t s_lo, uint32_t s_hi)
{
    const Sys &d = s.b;
    if (q >= (uint32_t)d.n) {   // cannot happen: every queued slot was read below n
        set_err_at(d, ERR_INTERNAL, 13, q, o, 0);
        return;
    }
    const uint4 pi = pis[o], pj = s.S_p[q];
    const float4 vi = vis[o], vj = s.S_v[q];
    const float dx = mdiff(d, pi.x, pj.x), dy = mdiff(d, pi.y, pj.y), dz = mdiff(d, pi.z, pj.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < d.rc2) || !(r2 > 0.f)) return;   // the walk's filter is a little wider than r_c
    const float rinv = rsqrtf(r2);
    const float ex = dx * rinv, ey = dy * rinv, ez = dz * rinv;   // e = (x_i - x_j)/r
    const float dve = (vi.x - vj.x) * ex + (vi.y - vj.y) * ey + (vi.z - vj.z) * ez;
    const float F = pair_scalar3(d, r2, rinv, dve, pi.w, pj.w, s_lo, s_hi);
    if (!(fabsf(F) < FQ_MAX)) set_err(d, ERR_NONFINITE);
    const long long qx = fq(F * ex), qy = fq(F * ey), qz = fq(F * ez);
    fq_add(&fs[o][0], 1, qx);
    fq_add(&fs[o][2], 1, qy);
    fq_add(&fs[o][4], 1, qz);
    unsigned long long *fq_q = (unsigned long long *)(s.F + 4 * (size_t)q);
    atomicAdd(fq_q, (unsigned long long)-qx);
    atomicAdd(fq_q + 1, (unsigned long long)-qy);
    atomicAdd(fq_q + 2, (unsigned long long)-qz);
}

// Pair forces, one thread per bead over the half stencil: the rest of its own
// cell and the 13 cells ahead of it in (z, y, x) order, so that every pair
// inside r_c is met once (n_c >= 3).  The lanes of a warp test their
// candidates in step and push the pairs inside r_c, as (slot, owner lane),
// into the warp's queue; every 32 queued pairs the whole warp evaluates
// Philox and the force together.  Sums go to F (sorted order).
__global__ void __launch_bounds__(256, 5) k3_pairs(Sys3 s)
{
    const Sys &d = s.b;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
    __shared__ uint32_t s_q[8][64];
    __shared__ unsigned char s_ql[8][64];
    __shared__ uint4 s_pi[8][32];
    __shared__ float4 s_vi[8][32];
    __shared__ int s_f[8][32][6];
    const bool active = g < d.n;
    const long long step = *d.step;
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xffffffffull);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
    const uint32_t n = (uint32_t)d.n;
    const uint4 pi = active ? s.S_p[g] : make_uint4(0u, 0u, 0u, 0xffffffffu);
    const float4 vi = active ? s.S_v[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t id = pi.w, pid = d.excl ? (id ^ 1u) : 0xffffffffu;
    s_pi[warp][lane] = pi;
    s_vi[warp][lane] = vi;
#pragma unroll
    for (int c = 0; c < 6; ++c) s_f[warp][lane][c] = 0;
    __syncwarp();
    const int cx = cell_coord(d, pi.x), cy = cell_coord(d, pi.y), cz = cell_coord(d, pi.z);
    // the walk tests separations from cell-corner offsets (no conversion per
    // candidate); a pair it passes is tested again exactly before evaluation
    const float4 oi = active ? s.S_off[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    int qn = 0;
    // entry 0: own cell after g; entries 1..13: (dz, dy, dx) > 0 lexicographically
#pragma unroll 1
    for (int e = 0; e < 14; ++e) {
        int oz = 0, oy = 0, ox = 0;
        if (e >= 5) { oz = 1; oy = (e - 5) / 3 - 1; ox = (e - 5) % 3 - 1; }
        else if (e >= 2) { oy = 1; ox = e - 3; }
        else if (e == 1) { ox = 1; }
        int x = cx + ox, y = cy + oy, z = cz + oz;
        x += x < 0 ? d.nc : (x >= d.nc ? -d.nc : 0);
        y += y < 0 ? d.nc : (y >= d.nc ? -d.nc : 0);
        z += z < 0 ? d.nc : (z >= d.nc ? -d.nc : 0);
        uint32_t b = 0, en = 0;
        if (active) {
            const int c = (z * d.nc + y) * d.nc + x;
            b = min(d.cstart[c], n);
            en = min(max(d.cstart[c + 1], b), n);
            if (e == 0) b = min((uint32_t)g + 1u, en);
        }
        const int len = (int)(en - b);
        const int maxlen = __reduce_max_sync(FULL, (unsigned)len);
        // bead i seen from the corner of the cell (ox, oy, oz) cells away
        const float pix = oi.x - (float)ox * d.cs, piy = oi.y - (float)oy * d.cs, piz = oi.z - (float)oz * d.cs;
        for (int t = 0; t < maxlen; ++t) {
            const uint32_t q = b + (uint32_t)t;
            bool hit = false;
            if (t < len) {
                const float4 oj = s.S_off[q];
                const float dx = pix - oj.x, dy = piy - oj.y, dz = piz - oj.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                hit = (r2 < s.rc2f) & (__float_as_uint(oj.w) != pid) & (q != (uint32_t)g);
            }
            const unsigned m = __ballot_sync(FULL, hit);
            if (hit) {
                const int pos = qn + __popc(m & lt);
                s_q[warp][pos] = q;
                s_ql[warp][pos] = (unsigned char)lane;
            }
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                const uint32_t mq = s_q[warp][lane];
                const int mo = s_ql[warp][lane];
                const uint32_t cq = s_q[warp][32 + lane];
                const unsigned char co = s_ql[warp][32 + lane];
                __syncwarp();
                if (lane < qn - 32) {
                    s_q[warp][lane] = cq;
                    s_ql[warp][lane] = co;
                }
                qn -= 32;
                eval3(s, mq, mo, s_pi[warp], s_vi[warp], s_f[warp], s_lo, s_hi);
                __syncwarp();
            }
        }
    }
    if (lane < qn) eval3(s, s_q[warp][lane], s_ql[warp][lane], s_pi[warp], s_vi[warp], s_f[warp], s_lo, s_hi);
    __syncwarp();
    if (active) {
        unsigned long long *fq_g = (unsigned long long *)(s.F + 4 * (size_t)g);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long qc = (long long)s_f[warp][lane][2 * c] * 65536ll + (long long)(unsigned)s_f[warp][lane][2 * c + 1];
            if (qc) atomicAdd(fq_g + c, (unsigned long long)qc);
        }
    }
}

// Everything after the pair sums, one thread per sorted slot: the pair force
// (reset to zero for the next step), bond and propulsion (partner id ^ 1),
// drag on the half-step velocity, the second half-kick, FP64 thermo
// partials, the next half-kick and drift, and the binning of the new position.
__global__ void __launch_bounds__(256) k3_integrate(Sys3 s, int flags)
{
    const Sys &d = s.b;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    const uint32_t n = (uint32_t)d.n;
    if (g < d.n) {
        const uint4 pi = s.S_p[g];
        const float4 vi = s.S_v[g];
        const uint32_t id = pi.w;
        longlong2 *fqg = (longlong2 *)(s.F + 4 * (size_t)g);
        const longlong2 f01 = fqg[0], f23 = fqg[1];
        fqg[0] = make_longlong2(0ll, 0ll);
        fqg[1] = make_longlong2(0ll, 0ll);
        float fx = fq_to_f(f01.x), fy = fq_to_f(f01.y), fz = fq_to_f(f23.x);
        // bond and propulsion (partner id ^ 1), drag on the half-step velocity
        const uint32_t ps = s.slot[id ^ 1u];
        if (ps < n) {
            const uint4 pp = s.S_p[ps];
            const float dx = mdiff(d, pi.x, pp.x), dy = mdiff(d, pi.y, pp.y), dz = mdiff(d, pi.z, pp.z);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > 0.f) {
                const float r = sqrtf(r2), inv = 1.0f / r;
                const float fb = -d.kbond * (r - d.r0);
                const float sp = (id & 1u) ? -d.fp : d.fp;   // n_k = head - tail
                fx += (fb + sp) * dx * inv;
                fy += (fb + sp) * dy * inv;
                fz += (fb + sp) * dz * inv;
            }
        } else {
            set_err_at(d, ERR_INTERNAL, 12, g, id, ps);
        }
        float vx = vi.x, vy = vi.y, vz = vi.z;
        fx -= d.zeta * vx;
        fy -= d.zeta * vy;
        fz -= d.zeta * vz;
        if (!(flags & F_FIRST)) { vx += d.hdtm * fx; vy += d.hdtm * fy; vz += d.hdtm * fz; }
        {
            const double dvx = (double)vx, dvy = (double)vy, dvz = (double)vz;
            ke = fma(dvx, dvx, fma(dvy, dvy, dvz * dvz));
            px = dvx; py = dvy; pz = dvz;
        }
        if (flags & F_FINAL) {
            s.C_p[id] = make_uint4(pi.x, pi.y, pi.z, 0u);
            s.C_v[id] = make_float4(vx, vy, vz, 0.f);
            s.C_f[id] = make_float4(fx, fy, fz, 0.f);
        }
        if (flags & F_ADVANCE) {
            vx += d.hdtm * fx;
            vy += d.hdtm * fy;
            vz += d.hdtm * fz;
            const float ddx = d.dt * vx, ddy = d.dt * vy, ddz = d.dt * vz;
            uint32_t nx = pi.x, ny = pi.y, nz = pi.z;
            const float lim = 0.25f * d.L;
            if (fabsf(ddx) < lim && fabsf(ddy) < lim && fabsf(ddz) < lim) {   // false for NaN too
                nx = fx_add(d, pi.x, ddx);
                ny = fx_add(d, pi.y, ddy);
                nz = fx_add(d, pi.z, ddz);
            } else {
                set_err(d, ERR_NONFINITE);
                vx = vy = vz = 0.f;
            }
            s.U_rank[g] = atomicAdd(&d.counts[cell3(d, nx, ny, nz)], 1u);
            s.U_p[g] = make_uint4(nx, ny, nz, id);
            s.U_v[g] = make_float4(vx, vy, vz, 0.f);
        }
    }
    // thermo partials in FP64 throughout (per bead, across the block, across
    // blocks).  One bead per thread, so the block sum goes through shared
    // memory: warp c adds quantity c (eight values per lane, then across its
    // lanes), a quarter of the FP64 additions of a shuffle tree in every warp
    // (the FP64 pipe is narrow on this part).
    if (flags & (F_ADVANCE | F_FINAL)) {
        __shared__ double red[4][256];
        const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
        red[0][tid] = ke;
        red[1][tid] = px;
        red[2][tid] = py;
        red[3][tid] = pz;
        __syncthreads();
        if (wid < 4) {
            double a = 0.0;
            for (int i = lane; i < (int)blockDim.x; i += 32) a += red[wid][i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) atomicAdd(&d.thermo[4 * (size_t)(*d.step % THERMO_CAP) + wid], a);
        }
    }
}

}  // namespace dpd

using namespace dpd;

#define CU3(x)                                                                      \
    do {                                                                            \
        const cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

static int latched3(dpd3_ctx *c)
{
    int *e = (int *)(c->h_pin + 500);
    CU3(cudaMemcpyAsync(e, c->s.b.err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU3(cudaStreamSynchronize(c->st));
    if (*e & ERR_NONFINITE) return DPD_ERR_NONFINITE;
    if (*e & ERR_TIMEOUT) return DPD_ERR_TIMEOUT;
    if (*e & ERR_INTERNAL) return DPD_ERR_INTERNAL;
    return DPD_OK;
}

int dpd3_internal_latched(dpd3_ctx *c) { return latched3(c); }

static void iteration3(dpd3_ctx *c, int flags)
{
    const int g = (c->s.b.n + 255) / 256;
    k3_scan<<<c->nscan, SCAN_NT, 0, c->st>>>(c->s.b, c->nscan);
    k3_scatter<<<g, 256, 0, c->st>>>(c->s);
    k3_pairs<<<g, 256, 0, c->st>>>(c->s);
    k3_integrate<<<g, 256, 0, c->st>>>(c->s, flags);
}

extern "C" {

int dpd3_create(const dpd_params *p, void *stream, dpd3_ctx **out)
{
    if (!out) return DPD_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    const int nc = n_cells_side(p->L, p->rc);
    if ((double)nc * nc * nc >= 2.0e9) return DPD_ERR_INVALID_ARG;
    dpd3_ctx *c = new (std::nothrow) dpd3_ctx();
    if (!c) return DPD_ERR_OOM;
    c->p = *p;
    if (stream) c->st = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) { delete c; return DPD_ERR_CUDA; }
        c->own_stream = true;
    }
    Sys &d = c->s.b;
    fill_physics(d, p);
    fill_geometry(d, p, 8);
    d.ncells = nc * nc * nc;
    d.ntx = 0;
    d.cap = 0;
    c->nscan = (d.ncells + SCAN_TILE - 1) / SCAN_TILE;
    const size_t n = (size_t)d.n, nce = (size_t)d.ncells;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_Sp = take(16 * n), o_Sv = take(16 * n), o_Up = take(16 * n), o_Uv = take(16 * n),
                 o_Cp = take(16 * n), o_Cv = take(16 * n), o_Cf = take(16 * n), o_rank = take(4 * n),
                 o_slot = take(4 * n), o_cnt = take(4 * nce), o_cst = take(4 * (nce + 1)),
                 o_th = take(32 * (size_t)THERMO_CAP), o_step = take(8), o_err = take(4), o_einfo = take(32),
                 o_ss = take(8 * (size_t)c->nscan), o_tk = take(8), o_stage = take(48 * n),
                 o_F = take(32 * n), o_off = take(16 * n), o_corner = take(4 * (size_t)nc);
    if (cudaMalloc(&c->pool, off) != cudaSuccess || cudaMallocHost((void **)&c->h_pin, 4096) != cudaSuccess) {
        dpd3_destroy(c);
        return DPD_ERR_OOM;
    }
    char *b = (char *)c->pool;
    c->s.S_p = (uint4 *)(b + o_Sp); c->s.S_v = (float4 *)(b + o_Sv);
    c->s.U_p = (uint4 *)(b + o_Up); c->s.U_v = (float4 *)(b + o_Uv);
    c->s.C_p = (uint4 *)(b + o_Cp); c->s.C_v = (float4 *)(b + o_Cv); c->s.C_f = (float4 *)(b + o_Cf);
    c->s.U_rank = (uint32_t *)(b + o_rank); c->s.slot = (uint32_t *)(b + o_slot);
    c->s.F = (long long *)(b + o_F);   // zeroed with the pool; k3_integrate keeps it zero between steps
    c->s.S_off = (float4 *)(b + o_off);
    c->s.corner = (const uint32_t *)(b + o_corner);
    c->s.rc2f = (float)(p->rc * p->rc * (1.0 + 1e-5));
    d.slot = c->s.slot;
    d.counts = (uint32_t *)(b + o_cnt); d.cstart = (uint32_t *)(b + o_cst);
    d.thermo = (double *)(b + o_th); d.step = (long long *)(b + o_step);
    d.err = (int *)(b + o_err); d.errinfo = (long long *)(b + o_einfo);
    d.scan_status = (unsigned long long *)(b + o_ss); d.scan_ticket = (unsigned long long *)(b + o_tk);
    d.S_xv = nullptr; d.S_id = nullptr; d.U_xv = nullptr; d.U_id = nullptr; d.U_rank = c->s.U_rank;
    d.C_xv = nullptr; d.C_f = nullptr; d.pcnt = nullptr; d.ovf = nullptr;
    c->stage = b + o_stage;
    std::vector<uint32_t> corner((size_t)nc);
    for (int q = 0; q < nc; ++q)
        corner[q] = (uint32_t)((((unsigned long long)q << 32) + (unsigned long long)(nc - 1)) / (unsigned long long)nc);
    if (cudaMemsetAsync(c->pool, 0, off, c->st) != cudaSuccess ||
        cudaMemcpyAsync(b + o_corner, corner.data(), 4 * (size_t)nc, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
        dpd3_destroy(c);
        return DPD_ERR_CUDA;
    }
    *out = c;
    return DPD_OK;
}

void dpd3_destroy(dpd3_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->pool) cudaFree(c->pool);
    if (c->obs) cudaFree(c->obs);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

int dpd3_set_state(dpd3_ctx *c, const double *x, const float *v, int64_t step)
{
    if (!c || !x || !v) return DPD_ERR_INVALID_ARG;
    const size_t n = (size_t)c->s.b.n;
    char *st = c->stage;
    CU3(cudaMemcpyAsync(st, x, 24 * n, cudaMemcpyHostToDevice, c->st));
    CU3(cudaMemcpyAsync(st + 24 * n, v, 12 * n, cudaMemcpyHostToDevice, c->st));
    CU3(cudaMemsetAsync(c->s.b.err, 0, sizeof(int), c->st));
    CU3(cudaMemsetAsync(c->s.b.errinfo, 0, 32, c->st));
    CU3(cudaMemsetAsync(c->s.b.counts, 0, 4 * (size_t)c->s.b.ncells, c->st));
    const int g = (int)((n + 255) / 256);
    k3_load<<<g, 256, 0, c->st>>>(c->s, (const double *)st, (const float *)(st + 24 * n));
    k3_bin<<<g, 256, 0, c->st>>>(c->s);
    k3_set_step<<<1, 1, 0, c->st>>>(c->s.b, step - 1);
    iteration3(c, F_FIRST | F_FINAL | F_ADVANCE);
    CU3(cudaGetLastError());
    c->step = step;
    c->have_state = true;
    return latched3(c);
}

int dpd3_step(dpd3_ctx *c, int64_t n)
{
    if (!c || n < 0) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    for (int64_t i = 0; i < n; ++i) iteration3(c, i == n - 1 ? (F_ADVANCE | F_FINAL) : F_ADVANCE);
    CU3(cudaGetLastError());
    c->step += n;
    return DPD_OK;
}

int dpd3_sync(dpd3_ctx *c)
{
    if (!c) return DPD_ERR_INVALID_ARG;
    return latched3(c);
}

int dpd3_get_state(dpd3_ctx *c, double *x, float *v, float *f, int64_t *step)
{
    if (!c || !x || !v || !f) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const size_t n = (size_t)c->s.b.n;
    double *dx = (double *)c->stage;
    float *dv = (float *)(dx + 3 * n), *df = dv + 3 * n;
    k3_store<<<(int)((n + 255) / 256), 256, 0, c->st>>>(c->s, dx, dv, df);
    CU3(cudaMemcpyAsync(x, dx, 24 * n, cudaMemcpyDeviceToHost, c->st));
    CU3(cudaMemcpyAsync(v, dv, 12 * n, cudaMemcpyDeviceToHost, c->st));
    CU3(cudaMemcpyAsync(f, df, 12 * n, cudaMemcpyDeviceToHost, c->st));
    if (step) *step = c->step;
    return latched3(c);
}

int dpd3_thermo(dpd3_ctx *c, double out[5])
{
    if (!c || !out) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    CU3(cudaMemcpyAsync(c->h_pin, c->s.b.thermo + 4 * (size_t)(c->step % THERMO_CAP), 32, cudaMemcpyDeviceToHost,
                        c->st));
    const int rc = latched3(c);
    const double m = c->p.mass, n = (double)c->s.b.n;
    out[0] = 0.5 * m * c->h_pin[0];
    out[1] = m * c->h_pin[1];
    out[2] = m * c->h_pin[2];
    out[3] = m * c->h_pin[3];
    out[4] = m * c->h_pin[0] / (3.0 * n - 3.0);
    return rc;
}

}  // extern "C"
