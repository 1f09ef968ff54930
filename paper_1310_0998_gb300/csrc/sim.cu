// Single-system C ABI of the DPD dimer simulator (include/dpd.h).
//
// Per step three kernels run on the context's stream, captured once into CUDA
// graphs (1-step, 8-step and a final step that also writes the canonical
// state): scan -> scatter -> fused force/integrate (see sim_kernels.cuh).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "dpd.h"
#include "sim_kernels.cuh"
#include "sim_host.h"

namespace dpd {

// ----------------------------------------------------------------- kernels ----
__global__ void __launch_bounds__(SCAN_NT) k_scan(Sys d, int nblocks)
{
    __shared__ uint32_t s_buf[SCAN_BUF];
    scan_decoupled_t<SCAN_NT>(d, nblocks, s_buf);
}

template <int B>
__global__ void k_scatter(Sys d)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < d.n) scatter_one<B>(d, k);
}

template <int B>
__global__ void k_bin(Sys d)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < d.n) bin_one<B>(d, k);
}

__global__ void k_set_step(Sys d, long long s) { *d.step = s; }

// Double position -> fixed point: round x 2^32 / L to the nearest integer and
// keep it modulo 2^32, which is the wrap into [0, L) because L is exactly 2^32
// units.  One multiply instead of divides (FP64 is a slow pipe on this part);
// for a position already on the grid the product is within 2^-20 of an
// integer, so the result is exact.  |x| beyond 2^20 L is refused.
__device__ __forceinline__ uint32_t to_fixed(const Sys &d, double x, bool &ok)
{
    const double u = x * d.inv_ulen_d;
    if (!(fabs(u) < 4503599627370496.0)) { ok = false; return 0u; }   // 2^52 units; false for NaN
    return (uint32_t)(unsigned long long)llrint(u);
}

// Upload: positions (double [N][2]) and velocities (float [N][2]) in id order.
// into U (set-up path, f == NULL) or into the canonical buffers (with f).
__global__ void k_load_state(Sys d, const double *__restrict__ x, const float *__restrict__ v,
                             const float *__restrict__ f)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    bool ok = true;
    const uint32_t X = to_fixed(d, x[2 * k], ok), Y = to_fixed(d, x[2 * k + 1], ok);
    float vx = v[2 * k], vy = v[2 * k + 1];
    if (!isfinite(vx) || !isfinite(vy)) ok = false;
    float fx = 0.f, fy = 0.f;
    if (f) {
        fx = f[2 * k];
        fy = f[2 * k + 1];
        if (!isfinite(fx) || !isfinite(fy)) ok = false;
    }
    if (!ok) {
        set_err(d, ERR_NONFINITE);
        vx = vy = fx = fy = 0.f;
    }
    const uint4 r = make_uint4(X, Y, fbits(vx), fbits(vy));
    if (f) {
        d.C_xv[k] = r;
        d.C_f[k] = make_float2(fx, fy);
    } else {
        d.U_xv[k] = r;
        d.U_id[k] = (uint32_t)k;
    }
}

// Download of the canonical state: exact double positions (X L / 2^32).
__global__ void k_store_state(Sys d, double *__restrict__ x, float *__restrict__ v, float *__restrict__ f)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const uint4 r = d.C_xv[k];
    if (x) {
        x[2 * k] = (double)r.x * d.ulen_d;
        x[2 * k + 1] = (double)r.y * d.ulen_d;
    }
    if (v) {
        v[2 * k] = vbits(r.z);
        v[2 * k + 1] = vbits(r.w);
    }
    if (f) {
        const float2 ff = d.C_f[k];
        f[2 * k] = ff.x;
        f[2 * k + 1] = ff.y;
    }
}

// Canonical (X_s, v_s, f_s) in id order -> next pre-force state in U, plus
// the thermo entry of step s.
template <int B>
__global__ void k_kick_bin(Sys d)
{
    __shared__ double s_red[3 * 33];
    Thermo3 th{0.0, 0.0, 0.0};
    // grid-stride over the beads with a capped grid: the per-block FP64 thermo
    // flush targets one address, and one flush per 256 beads serialised there
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += gridDim.x * blockDim.x) {
        const uint4 xv = d.C_xv[k];
        const float2 f = d.C_f[k];
        float vx = vbits(xv.z), vy = vbits(xv.w);
        th.ke = fma((double)vx, (double)vx, fma((double)vy, (double)vy, th.ke));
        th.px += (double)vx;
        th.py += (double)vy;
        vx = __fmaf_rn(d.hdtm, f.x, vx);
        vy = __fmaf_rn(d.hdtm, f.y, vy);
        const float ddx = __fmul_rn(d.dt, vx), ddy = __fmul_rn(d.dt, vy);
        uint32_t nx = xv.x, ny = xv.y;
        if (fabsf(ddx) < 0.25f * d.L && fabsf(ddy) < 0.25f * d.L) {
            nx = fx_add(d, xv.x, ddx);
            ny = fx_add(d, xv.y, ddy);
        } else {
            set_err(d, ERR_NONFINITE);
            vx = 0.f; vy = 0.f;
        }
        const int c = cell_of<B>(d, cell_coord(d, nx), cell_coord(d, ny));
        d.U_rank[k] = atomicAdd(&d.counts[c], 1u);
        d.U_xv[k] = make_uint4(nx, ny, fbits(vx), fbits(vy));
        d.U_id[k] = (uint32_t)k;
    }
    thermo_flush(d, th, s_red);
}

template <int B, bool COUNT, int VAR>
__global__ void __launch_bounds__(TILE_THREADS, 10) k_force(Sys d, int flags)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Thermo3 th{0.0, 0.0, 0.0};
    force_tile<B, COUNT, VAR>(d, blockIdx.x, flags, smem, th);
    if (flags & (F_ADVANCE | F_FINAL)) {
        __syncthreads();
        thermo_flush_tile(d, th, (double *)(smem + tile_flush_off<B, VAR>()));
    }
}

// Paper's initial condition (Sec. 5): per agent k, Philox4x32-10 of counter
// (k, 0, 0, 0) under key (seed lo, seed hi ^ 0x1D17); words 0 and 1 are the
// centre's fixed-point coordinates (uniform on the box), word 2 the
// orientation 2 pi w2 / 2^32; beads at centre +/- (r0/2) n; v = 0.
__global__ void k_init_random(Sys d, unsigned long long seed)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * k + 1 >= d.n) return;
    uint32_t c0 = (uint32_t)k, c1 = 0, c2 = 0, c3 = 0;
    philox10(c0, c1, c2, c3, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32) ^ 0x1D17u);
    const float u2 = (float)(c2 >> 8) * 5.9604644775390625e-08f;
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    const float h = 0.5f * d.r0;
    const int hx = __float2int_rn(h * cs * d.inv_ulen), hy = __float2int_rn(h * sn * d.inv_ulen);
    d.U_xv[2 * k] = make_uint4(c0 + (uint32_t)hx, c1 + (uint32_t)hy, 0u, 0u);
    d.U_xv[2 * k + 1] = make_uint4(c0 - (uint32_t)hx, c1 - (uint32_t)hy, 0u, 0u);
    d.U_id[2 * k] = 2u * k;
    d.U_id[2 * k + 1] = 2u * k + 1u;
}

// ------------------------------------------------------------------- host ----
static int cuerr(cudaError_t e)
{
    if (e == cudaSuccess) return DPD_OK;
    if (e == cudaErrorMemoryAllocation) return DPD_ERR_OOM;
    return DPD_ERR_CUDA;
}
#define CU(x)                                  \
    do {                                       \
        const cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) return cuerr(e_); \
    } while (0)

int n_cells_side(double L, double rc) { return (int)std::floor(L / rc); }

int validate(const dpd_params *p)
{
    if (!p) return DPD_ERR_INVALID_ARG;
    if (!(p->rc > 0) || !(p->L >= 3 * p->rc) || !(p->dt > 0) || !(p->mass > 0)) return DPD_ERR_INVALID_ARG;
    if (!(p->gamma >= 0) || !(p->zeta >= 0) || !(p->k_bond >= 0) || !(p->kBT >= 0) || !(p->r0 >= 0) ||
        !(p->f_p >= 0) || !std::isfinite(p->a))
        return DPD_ERR_INVALID_ARG;
    if (p->n_beads < 2 || (p->n_beads & 1) || p->n_beads >= (1ll << 31)) return DPD_ERR_INVALID_ARG;
    if (!(p->tile == 0 || p->tile == 4 || p->tile == 8 || p->tile == 16)) return DPD_ERR_INVALID_ARG;
    if (p->variant < 0 || p->variant > 5) return DPD_ERR_INVALID_ARG;
    if (p->noise < 0 || p->noise > 1) return DPD_ERR_INVALID_ARG;
    if (!(p->wexp >= 0.0 && p->wexp <= 8.0)) return DPD_ERR_INVALID_ARG;
    const int nc = n_cells_side(p->L, p->rc);
    if (nc < 3 || (double)nc * nc >= 2.0e9) return DPD_ERR_INVALID_ARG;
    return DPD_OK;
}

void fill_physics(Sys &d, const dpd_params *p)
{
    d.rc2 = (float)(p->rc * p->rc);
    d.inv_rc = (float)(1.0 / p->rc);
    d.a = (float)p->a;
    d.gamma = (float)p->gamma;
    const double sig = std::sqrt(2.0 * p->gamma * p->kBT / p->dt);
    d.sig_r = p->noise == 0 ? (float)(sig * std::sqrt(3.0) * std::ldexp(1.0, -24)) : (float)sig;
    d.kbond = (float)p->k_bond;
    d.r0 = (float)p->r0;
    d.fp = (float)p->f_p;
    d.zeta = (float)p->zeta;
    d.dt = (float)p->dt;
    d.hdtm = (float)(0.5 * p->dt / p->mass);
    d.key0 = (uint32_t)(p->seed & 0xffffffffull);
    d.key1 = (uint32_t)(p->seed >> 32) ^ p->replica;
    for (int r = 0; r < 10; ++r) {
        d.rk0[r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
        d.rk1[r] = d.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    d.noise = p->noise;
    d.excl = p->exclude_bonded ? 1 : 0;
    const double s = p->wexp > 0.0 ? p->wexp : 2.0;
    d.gen_w = s != 2.0 ? 1 : 0;
    d.hwexp = (float)(0.5 * s);
    // pair geometry in fixed-point units (needs the geometry's unit length)
    const double rcu = p->rc / std::ldexp(p->L, -32);
    d.rc2u = (float)(rcu * rcu);
    d.inv_rcu = (float)(std::ldexp(p->L, -32) / p->rc);
}

void fill_geometry(Sys &d, const dpd_params *p, int B)
{
    const int nc = n_cells_side(p->L, p->rc);
    d.Ld = p->L;
    d.ulen_d = std::ldexp(p->L, -32);
    d.inv_ulen_d = std::ldexp(1.0, 32) / p->L;
    d.L = (float)p->L;
    d.ulen = (float)d.ulen_d;
    d.inv_ulen = (float)(std::ldexp(1.0, 32) / p->L);
    d.nc = nc;
    d.cs = (float)(p->L / nc);
    d.ntx = (nc + B - 1) / B;
    d.n = (int)p->n_beads;
    d.ncells = nc * nc;
}

int tile_capacity(const dpd_params *p, int B)
{
    const int nc = n_cells_side(p->L, p->rc);
    const double cs = p->L / nc;
    const double rho = (double)p->n_beads / (p->L * p->L);
    const double mean = rho * ((B + 2) * cs) * ((B + 2) * cs);
    // mean staged population plus a margin of eight Poisson standard
    // deviations, kept small so that ten tiles stay resident per SM at
    // density 3 (1.3 x mean measured 4% slower at 8 x 8 cells and 17% at
    // 16 x 16); a tile above it takes the (slower, exact) global-memory path,
    // and a context that sees such tiles grows its capacity at the next
    // synchronising call
    int cap = (int)std::ceil(mean + 8.0 * std::sqrt(mean) + 32.0);
    cap = (cap + 31) & ~31;
    return std::min(std::max(cap, 256), 4096);   // queue entries pack bead slots in 12 bits
}

size_t force_smem(int B, int var, int cap, bool count)
{
    if (var == 3) {
        switch (B) {
            case 4: return TilePlanG<4>::bytes(cap, TILE_THREADS, count);
            case 8: return TilePlanG<8>::bytes(cap, TILE_THREADS, count);
            default: return TilePlanG<16>::bytes(cap, TILE_THREADS, count);
        }
    }
    if (var == 4) {
        switch (B) {
            case 4: return TilePlan<4, 4>::bytes(cap, TILE_THREADS, count);
            case 8: return TilePlan<8, 4>::bytes(cap, TILE_THREADS, count);
            default: return TilePlan<16, 4>::bytes(cap, TILE_THREADS, count);
        }
    }
    if (var == 5) {
        switch (B) {
            case 4: return TilePlan<4, 5>::bytes(cap, TILE_THREADS, count);
            case 8: return TilePlan<8, 5>::bytes(cap, TILE_THREADS, count);
            default: return TilePlan<16, 5>::bytes(cap, TILE_THREADS, count);
        }
    }
    switch (B) {
        case 4: return TilePlan<4>::bytes(cap, TILE_THREADS, count);
        case 8: return TilePlan<8>::bytes(cap, TILE_THREADS, count);
        default: return TilePlan<16>::bytes(cap, TILE_THREADS, count);
    }
}

// The dynamic shared-memory limit is a per-kernel, process-wide attribute:
// raise it once to the device's opt-in maximum so contexts with different
// tile capacities never shrink each other's limit.
template <typename K>
static int set_dyn_limit(K kernel, int smax)
{
    cudaFuncAttributes fa;
    CU(cudaFuncGetAttributes(&fa, kernel));   // the limit covers static + dynamic
    CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smax - (int)fa.sharedSizeBytes));
    return DPD_OK;
}

template <int B>
static int set_force_attrs(int smax)
{
    int rc = set_dyn_limit(k_force<B, false, 1>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, true, 1>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, false, 2>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, true, 2>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, false, 3>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, true, 3>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, false, 4>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, true, 4>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, false, 5>, smax);
    if (!rc) rc = set_dyn_limit(k_force<B, true, 5>, smax);
    return rc;
}

int max_dynamic_smem()
{
    int dev = 0, smax = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 48 * 1024;
    return smax;
}

int set_force_smem(int B, int var, int cap)
{
    const int smax = max_dynamic_smem();
    if ((int)force_smem(B, var, cap, true) > smax) return DPD_ERR_INVALID_ARG;
    int rc = set_force_attrs<4>(smax);
    if (!rc) rc = set_force_attrs<8>(smax);
    if (!rc) rc = set_force_attrs<16>(smax);
    return rc;
}

template <int B, int VAR>
static void launch_force_t(const Sys &d, cudaStream_t st, size_t smem, int flags, bool count)
{
    const int ntiles = d.ntx * d.ntx;
    if (count) k_force<B, true, VAR><<<ntiles, TILE_THREADS, force_smem(B, VAR, d.cap, true), st>>>(d, flags);
    else k_force<B, false, VAR><<<ntiles, TILE_THREADS, smem, st>>>(d, flags);
}

void launch_force_only(const Sys &d, int B, int var, cudaStream_t st, size_t smem, int flags, bool count)
{
    if (var == 1) {
        switch (B) {
            case 4: launch_force_t<4, 1>(d, st, smem, flags, count); break;
            case 8: launch_force_t<8, 1>(d, st, smem, flags, count); break;
            default: launch_force_t<16, 1>(d, st, smem, flags, count); break;
        }
    } else if (var == 3) {
        switch (B) {
            case 4: launch_force_t<4, 3>(d, st, smem, flags, count); break;
            case 8: launch_force_t<8, 3>(d, st, smem, flags, count); break;
            default: launch_force_t<16, 3>(d, st, smem, flags, count); break;
        }
    } else if (var == 4) {
        switch (B) {
            case 4: launch_force_t<4, 4>(d, st, smem, flags, count); break;
            case 8: launch_force_t<8, 4>(d, st, smem, flags, count); break;
            default: launch_force_t<16, 4>(d, st, smem, flags, count); break;
        }
    } else if (var == 5) {
        switch (B) {
            case 4: launch_force_t<4, 5>(d, st, smem, flags, count); break;
            case 8: launch_force_t<8, 5>(d, st, smem, flags, count); break;
            default: launch_force_t<16, 5>(d, st, smem, flags, count); break;
        }
    } else {
        switch (B) {
            case 4: launch_force_t<4, 2>(d, st, smem, flags, count); break;
            case 8: launch_force_t<8, 2>(d, st, smem, flags, count); break;
            default: launch_force_t<16, 2>(d, st, smem, flags, count); break;
        }
    }
}

void launch_scatter(const Sys &d, int B, cudaStream_t st)
{
    const int g = (d.n + 255) / 256;
    switch (B) {
        case 4: k_scatter<4><<<g, 256, 0, st>>>(d); break;
        case 8: k_scatter<8><<<g, 256, 0, st>>>(d); break;
        default: k_scatter<16><<<g, 256, 0, st>>>(d); break;
    }
}

void launch_iteration(const Sys &d, int B, int var, cudaStream_t st, int nscan, size_t smem, int flags, bool count)
{
    k_scan<<<nscan, SCAN_NT, 0, st>>>(d, nscan);
    launch_scatter(d, B, st);
    launch_force_only(d, B, var, st, smem, flags, count);
}

void launch_bin(const Sys &d, int B, cudaStream_t st)
{
    const int g = (d.n + 255) / 256;
    switch (B) {
        case 4: k_bin<4><<<g, 256, 0, st>>>(d); break;
        case 8: k_bin<8><<<g, 256, 0, st>>>(d); break;
        default: k_bin<16><<<g, 256, 0, st>>>(d); break;
    }
}

void launch_kick_bin(const Sys &d, int B, cudaStream_t st)
{
    const int g = std::min((d.n + 255) / 256, 1024);
    switch (B) {
        case 4: k_kick_bin<4><<<g, 256, 0, st>>>(d); break;
        case 8: k_kick_bin<8><<<g, 256, 0, st>>>(d); break;
        default: k_kick_bin<16><<<g, 256, 0, st>>>(d); break;
    }
}

int host_cell_of(int B, int nc, int cx, int cy)
{
    const int tx = cx / B, lx = cx - tx * B, ty = cy / B, ly = cy - ty * B;
    const int th = std::min(B, nc - ty * B), tw = std::min(B, nc - tx * B);
    return ty * B * nc + tx * B * th + ly * tw + lx;
}

}  // namespace dpd

using namespace dpd;

static void free_graphs(dpd_ctx *c)
{
    if (c->g1) cudaGraphExecDestroy(c->g1);
    if (c->g8) cudaGraphExecDestroy(c->g8);
    if (c->gfin) cudaGraphExecDestroy(c->gfin);
    c->g1 = c->g8 = c->gfin = nullptr;
}

static int capture(dpd_ctx *c, int iters, int last_flags, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < iters; ++i)
        launch_iteration(c->d, c->B, c->var, c->st, c->nscan, c->smem, i == iters - 1 ? last_flags : F_ADVANCE, false);
    const cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (e != cudaSuccess) return cuerr(e);
    const cudaError_t e2 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuerr(e2);
}

static int ensure_graphs(dpd_ctx *c)
{
    if (c->g1 && c->g8 && c->gfin) return DPD_OK;
    free_graphs(c);
    int rc;
    if ((rc = capture(c, 1, F_ADVANCE, &c->g1))) return rc;
    if ((rc = capture(c, 8, F_ADVANCE, &c->g8))) return rc;
    if ((rc = capture(c, 1, F_ADVANCE | F_FINAL, &c->gfin))) return rc;
    return DPD_OK;
}

constexpr int H_PIN_STATUS = 510;   // h_pin holds 512 doubles; [510], [511]: error flag, overflow count

// A tile that did not fit in shared memory ran the global-memory path: raise
// the capacity by a quarter (within the shared-memory limit) and re-capture
// the step graphs at the next dpd_step.
static void grow_capacity(dpd_ctx *c)
{
    int cap = std::min(4096, ((c->d.cap * 5 / 4) + 31) & ~31);
    while (cap > c->d.cap && force_smem(c->B, c->var, cap, true) > 200 * 1024) cap -= 32;
    if (cap <= c->d.cap) return;
    c->d.cap = cap;
    c->smem = force_smem(c->B, c->var, cap, false);
    free_graphs(c);
}

int dpd_internal_latched(dpd_ctx *c)
{
    // the status words use their own slots at the end of the pinned buffer so
    // that a caller's values staged at its start (thermo_entry) survive
    int e = 0;
    unsigned long long ovf = 0;
    double *st = c->h_pin + H_PIN_STATUS;
    CU(cudaMemcpyAsync(st, c->d.err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(st + 1, c->d.ovf, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    std::memcpy(&e, st, sizeof(int));
    std::memcpy(&ovf, st + 1, sizeof(ovf));
    if (ovf > c->ovf_seen) {
        c->ovf_seen = ovf;
        if (!c->batch_owned) grow_capacity(c);
    }
    if (e & ERR_NONFINITE) return DPD_ERR_NONFINITE;
    if (e & ERR_TIMEOUT) return DPD_ERR_TIMEOUT;
    if (e & ERR_INTERNAL) return DPD_ERR_INTERNAL;
    return DPD_OK;
}

extern "C" {

const char *dpd_status_string(int s)
{
    switch (s) {
        case DPD_OK: return "ok";
        case DPD_ERR_INVALID_ARG: return "invalid argument";
        case DPD_ERR_CUDA: return "CUDA runtime error";
        case DPD_ERR_OOM: return "out of device memory";
        case DPD_ERR_NONFINITE: return "non-finite or runaway state";
        case DPD_ERR_TIMEOUT: return "bounded device wait timed out";
        case DPD_ERR_STATE: return "call not valid in this state";
        case DPD_ERR_INTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int dpd_create(const dpd_params *p, void *stream, dpd_ctx **out)
{
    if (!out) return DPD_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    dpd_ctx *c = new (std::nothrow) dpd_ctx();
    if (!c) return DPD_ERR_OOM;
    if (cudaGetDevice(&c->dev) != cudaSuccess) { delete c; return DPD_ERR_CUDA; }
    c->p = *p;
    c->B = p->tile ? p->tile : DEFAULT_TILE;
    c->var = p->variant ? p->variant : DEFAULT_VARIANT;
    if (!p->tile && !p->variant) {
        int t = 0, v = 0;
        if (tuned_shape(p, 1, &t, &v)) { c->B = t; c->var = v; }
    }
    if (stream) {
        c->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) { delete c; return DPD_ERR_CUDA; }
        c->own_stream = true;
    }
    Sys &d = c->d;
    fill_geometry(d, p, c->B);
    fill_physics(d, p);
    d.cap = tile_capacity(p, c->B);
    c->smem = force_smem(c->B, c->var, d.cap, false);
    if (force_smem(c->B, c->var, d.cap, true) > 200 * 1024) {
        d.cap = (int)((200 * 1024 - force_smem(c->B, c->var, 0, true)) / (c->var == 3 ? 43 : 41)) & ~31;
        c->smem = force_smem(c->B, c->var, d.cap, false);
    }
    c->nscan = (d.ncells + SCAN_TILE - 1) / SCAN_TILE;
    const size_t n = (size_t)d.n, nce = (size_t)d.ncells;
    // one pool, 256-byte aligned slices
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_S = take(16 * n), o_Sid = take(4 * n), o_U = take(16 * n), o_Uid = take(4 * n),
                 o_Ur = take(4 * n), o_slot = take(4 * n), o_cnt = take(4 * nce), o_cst = take(4 * (nce + 1)),
                 o_C = take(16 * n), o_Cf = take(8 * n), o_th = take(sizeof(double) * 4 * THERMO_CAP),
                 o_step = take(8), o_pc = take(4 * n), o_ovf = take(8), o_err = take(8), o_einfo = take(32),
                 o_ss = take(8 * (size_t)c->nscan), o_tk = take(8), o_stage = take(32 * n);
    c->pool_bytes = off;
    if (cudaMalloc(&c->pool, off) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->st);
        delete c;
        return DPD_ERR_OOM;
    }
    if (cudaMallocHost((void **)&c->h_pin, 4096) != cudaSuccess) {
        cudaFree(c->pool);
        if (c->own_stream) cudaStreamDestroy(c->st);
        delete c;
        return DPD_ERR_OOM;
    }
    char *b = (char *)c->pool;
    d.S_xv = (uint4 *)(b + o_S);
    d.S_id = (uint32_t *)(b + o_Sid);
    d.U_xv = (uint4 *)(b + o_U);
    d.U_id = (uint32_t *)(b + o_Uid);
    d.U_rank = (uint32_t *)(b + o_Ur);
    d.slot = (uint32_t *)(b + o_slot);
    d.counts = (uint32_t *)(b + o_cnt);
    d.cstart = (uint32_t *)(b + o_cst);
    d.C_xv = (uint4 *)(b + o_C);
    c->stage = b + o_stage;
    d.C_f = (float2 *)(b + o_Cf);
    d.thermo = (double *)(b + o_th);
    d.step = (long long *)(b + o_step);
    d.pcnt = nullptr;
    c->pcnt_buf = (uint32_t *)(b + o_pc);
    d.ovf = (unsigned long long *)(b + o_ovf);
    d.err = (int *)(b + o_err);
    d.errinfo = (long long *)(b + o_einfo);
    d.scan_status = (unsigned long long *)(b + o_ss);
    d.scan_ticket = (unsigned long long *)(b + o_tk);
    if (cudaMemsetAsync(c->pool, 0, off, c->st) != cudaSuccess ||
        (rc = set_force_smem(c->B, c->var, d.cap)) != DPD_OK) {
        dpd_destroy(c);
        return rc ? rc : DPD_ERR_CUDA;
    }
    if (cudaStreamSynchronize(c->st) != cudaSuccess) { dpd_destroy(c); return DPD_ERR_CUDA; }
    *out = c;
    return DPD_OK;
}

void dpd_destroy(dpd_ctx *c)
{
    if (!c || c->batch_owned) return;   // replicas belong to their batch
    if (c->st) cudaStreamSynchronize(c->st);
    free_graphs(c);
    dpd_internal_free_obs(c);
    if (c->pool) cudaFree(c->pool);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

int dpd_set_params(dpd_ctx *c, const dpd_params *p)
{
    if (!c) return DPD_ERR_INVALID_ARG;
    int rc = validate(p);
    if (rc) return rc;
    if (p->n_beads != c->p.n_beads || p->L != c->p.L || p->rc != c->p.rc) return DPD_ERR_STATE;
    const int B = p->tile ? p->tile : c->B;
    if (B != c->B) return DPD_ERR_STATE;
    c->var = p->variant ? p->variant : c->var;
    c->p = *p;
    fill_physics(c->d, p);
    free_graphs(c);   // kernel arguments carry the parameters
    return DPD_OK;
}

static int start_from_U(dpd_ctx *c, long long step)
{
    // U holds an unbinned state in id order: bin it, then the set-up step.
    launch_bin(c->d, c->B, c->st);
    k_set_step<<<1, 1, 0, c->st>>>(c->d, step - 1);
    launch_iteration(c->d, c->B, c->var, c->st, c->nscan, c->smem, F_FIRST | F_FINAL | F_ADVANCE, false);
    CU(cudaGetLastError());
    c->step = step;
    c->have_state = true;
    c->sorted_canonical = true;
    return dpd_internal_latched(c);
}

int dpd_set_state(dpd_ctx *c, const double *x, const float *v, const float *f, int64_t step, int where)
{
    if (!c || !x || !v || (where != DPD_HOST && where != DPD_DEVICE)) return DPD_ERR_INVALID_ARG;
    const size_t n = (size_t)c->d.n;
    const double *dx = x;
    const float *dv = v, *df = f;
    if (where == DPD_HOST) {
        char *st = (char *)c->stage;
        CU(cudaMemcpyAsync(st, x, 16 * n, cudaMemcpyHostToDevice, c->st));
        CU(cudaMemcpyAsync(st + 16 * n, v, 8 * n, cudaMemcpyHostToDevice, c->st));
        if (f) CU(cudaMemcpyAsync(st + 24 * n, f, 8 * n, cudaMemcpyHostToDevice, c->st));
        dx = (const double *)st;
        dv = (const float *)(st + 16 * n);
        df = f ? (const float *)(st + 24 * n) : nullptr;
    }
    CU(cudaMemsetAsync(c->d.err, 0, sizeof(int), c->st));
    CU(cudaMemsetAsync(c->d.errinfo, 0, 32, c->st));
    CU(cudaMemsetAsync(c->d.counts, 0, sizeof(uint32_t) * (size_t)c->d.ncells, c->st));
    k_load_state<<<(c->d.n + 255) / 256, 256, 0, c->st>>>(c->d, dx, dv, df);
    if (!f) return start_from_U(c, step);
    k_set_step<<<1, 1, 0, c->st>>>(c->d, step);
    CU(cudaMemsetAsync(c->d.thermo + 4 * (size_t)(step % THERMO_CAP), 0, 4 * sizeof(double), c->st));
    launch_kick_bin(c->d, c->B, c->st);
    CU(cudaGetLastError());
    c->step = step;
    c->have_state = true;
    c->sorted_canonical = false;
    return dpd_internal_latched(c);
}

int dpd_init_random(dpd_ctx *c, uint64_t seed)
{
    if (!c) return DPD_ERR_INVALID_ARG;
    CU(cudaMemsetAsync(c->d.err, 0, sizeof(int), c->st));
    CU(cudaMemsetAsync(c->d.errinfo, 0, 32, c->st));
    CU(cudaMemsetAsync(c->d.counts, 0, sizeof(uint32_t) * (size_t)c->d.ncells, c->st));
    k_init_random<<<(c->d.n / 2 + 255) / 256, 256, 0, c->st>>>(c->d, (unsigned long long)seed);
    return start_from_U(c, 0);
}

int dpd_step(dpd_ctx *c, int64_t n)
{
    if (!c || n < 0) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    if (n == 0) return DPD_OK;
    int rc = ensure_graphs(c);
    if (rc) return rc;
    const int64_t body = n - 1;
    for (int64_t i = 0; i < body / 8; ++i) CU(cudaGraphLaunch(c->g8, c->st));
    for (int64_t i = 0; i < body % 8; ++i) CU(cudaGraphLaunch(c->g1, c->st));
    CU(cudaGraphLaunch(c->gfin, c->st));
    c->step += n;
    c->sorted_canonical = true;
    return DPD_OK;
}

int dpd_sync(dpd_ctx *c)
{
    if (!c) return DPD_ERR_INVALID_ARG;
    return dpd_internal_latched(c);
}

int dpd_get_state(dpd_ctx *c, double *x, float *v, float *f, int64_t *step, int where)
{
    if (!c || (where != DPD_HOST && where != DPD_DEVICE)) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const size_t n = (size_t)c->d.n;
    if (where == DPD_DEVICE) {
        k_store_state<<<(c->d.n + 255) / 256, 256, 0, c->st>>>(c->d, x, v, f);
        CU(cudaGetLastError());
    } else {
        char *st = (char *)c->stage;
        k_store_state<<<(c->d.n + 255) / 256, 256, 0, c->st>>>(c->d, x ? (double *)st : nullptr,
                                                                v ? (float *)(st + 16 * n) : nullptr,
                                                                f ? (float *)(st + 24 * n) : nullptr);
        CU(cudaGetLastError());
        if (x) CU(cudaMemcpyAsync(x, st, 16 * n, cudaMemcpyDeviceToHost, c->st));
        if (v) CU(cudaMemcpyAsync(v, st + 16 * n, 8 * n, cudaMemcpyDeviceToHost, c->st));
        if (f) CU(cudaMemcpyAsync(f, st + 24 * n, 8 * n, cudaMemcpyDeviceToHost, c->st));
    }
    if (step) *step = c->step;
    return dpd_internal_latched(c);
}

static int thermo_entry(dpd_ctx *c, long long s, double out[4])
{
    CU(cudaMemcpyAsync(c->h_pin, c->d.thermo + 4 * (size_t)(s % THERMO_CAP), 4 * sizeof(double),
                       cudaMemcpyDeviceToHost, c->st));
    int rc = dpd_internal_latched(c);
    const double m = c->p.mass, n = (double)c->d.n;
    out[0] = 0.5 * m * c->h_pin[0];
    out[1] = m * c->h_pin[1];
    out[2] = m * c->h_pin[2];
    out[3] = m * c->h_pin[0] / (2.0 * n - 2.0);
    return rc;
}

int dpd_kinetic_energy(dpd_ctx *c, double *ke)
{
    if (!c || !ke) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    double t[4];
    const int rc = thermo_entry(c, c->step, t);
    *ke = t[0];
    return rc;
}

int dpd_momentum(dpd_ctx *c, double p[2])
{
    if (!c || !p) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    double t[4];
    const int rc = thermo_entry(c, c->step, t);
    p[0] = t[1];
    p[1] = t[2];
    return rc;
}

int dpd_temperature(dpd_ctx *c, double *T)
{
    if (!c || !T) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    double t[4];
    const int rc = thermo_entry(c, c->step, t);
    *T = t[3];
    return rc;
}

int dpd_thermo_log(dpd_ctx *c, int64_t first, int64_t count, double *out)
{
    if (!c || !out || count < 0) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    if (count == 0) return DPD_OK;
    if (first + count - 1 > c->step || first <= c->step - THERMO_CAP || count > THERMO_CAP)
        return DPD_ERR_INVALID_ARG;
    std::vector<double> raw(4 * (size_t)count);
    int64_t done = 0;
    while (done < count) {
        const int64_t s = first + done;
        const int64_t slot = s % THERMO_CAP;
        const int64_t run = std::min<int64_t>(count - done, THERMO_CAP - slot);
        CU(cudaMemcpyAsync(raw.data() + 4 * done, c->d.thermo + 4 * slot, 4 * sizeof(double) * run,
                           cudaMemcpyDeviceToHost, c->st));
        done += run;
    }
    const int rc = dpd_internal_latched(c);
    const double m = c->p.mass, n = (double)c->d.n;
    for (int64_t k = 0; k < count; ++k) {
        out[4 * k + 0] = 0.5 * m * raw[4 * k];
        out[4 * k + 1] = m * raw[4 * k + 1];
        out[4 * k + 2] = m * raw[4 * k + 2];
        out[4 * k + 3] = m * raw[4 * k] / (2.0 * n - 2.0);
    }
    return rc;
}

int dpd_cell_counts(dpd_ctx *c, uint32_t *counts)
{
    if (!c || !counts) return DPD_ERR_INVALID_ARG;
    if (!c->have_state || !c->sorted_canonical) return DPD_ERR_STATE;
    const int nc = c->d.nc;
    std::vector<uint32_t> cs((size_t)c->d.ncells + 1);
    CU(cudaMemcpyAsync(cs.data(), c->d.cstart, 4 * cs.size(), cudaMemcpyDeviceToHost, c->st));
    const int rc = dpd_internal_latched(c);
    for (int cy = 0; cy < nc; ++cy)
        for (int cx = 0; cx < nc; ++cx) {
            const int g = host_cell_of(c->B, nc, cx, cy);
            counts[(size_t)cy * nc + cx] = cs[g + 1] - cs[g];
        }
    return rc;
}

int dpd_pair_counts(dpd_ctx *c, uint32_t *cnt, uint64_t *total)
{
    if (!c) return DPD_ERR_INVALID_ARG;
    if (!c->have_state || !c->sorted_canonical) return DPD_ERR_STATE;
    const size_t n = (size_t)c->d.n;
    Sys d = c->d;
    d.pcnt = c->pcnt_buf;
    launch_force_only(d, c->B, c->var, c->st, c->smem, 0, true);
    CU(cudaGetLastError());
    std::vector<uint32_t> h(n);
    CU(cudaMemcpyAsync(h.data(), c->pcnt_buf, 4 * n, cudaMemcpyDeviceToHost, c->st));
    const int rc = dpd_internal_latched(c);
    uint64_t t = 0;
    for (size_t i = 0; i < n; ++i) t += h[i];
    if (cnt) std::memcpy(cnt, h.data(), 4 * n);
    if (total) *total = t / 2;
    return rc;
}

int dpd_profile_step(dpd_ctx *c, double ms[3])
{
    if (!c || !ms) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; ++i) CU(cudaEventCreate(&ev[i]));
    const Sys &d = c->d;
    CU(cudaEventRecord(ev[0], c->st));
    k_scan<<<c->nscan, SCAN_NT, 0, c->st>>>(d, c->nscan);
    CU(cudaEventRecord(ev[1], c->st));
    launch_scatter(d, c->B, c->st);
    CU(cudaEventRecord(ev[2], c->st));
    launch_force_only(d, c->B, c->var, c->st, c->smem, F_ADVANCE | F_FINAL, false);
    CU(cudaEventRecord(ev[3], c->st));
    CU(cudaGetLastError());
    c->step += 1;
    c->sorted_canonical = true;
    const int rc = dpd_internal_latched(c);
    for (int i = 0; i < 3; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
        ms[i] = t;
    }
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

int dpd_error_info(dpd_ctx *c, int64_t out[4])
{
    if (!c || !out) return DPD_ERR_INVALID_ARG;
    long long h[4];
    CU(cudaMemcpyAsync(h, c->d.errinfo, 32, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    for (int i = 0; i < 4; ++i) out[i] = h[i];
    return DPD_OK;
}

int dpd_get_info(dpd_ctx *c, dpd_info *info)
{
    if (!c || !info) return DPD_ERR_INVALID_ARG;
    unsigned long long ovf = 0;
    CU(cudaMemcpyAsync(c->h_pin, c->d.ovf, 8, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    std::memcpy(&ovf, c->h_pin, 8);
    info->n_beads = c->d.n;
    info->n_cells_side = c->d.nc;
    info->tile = c->B;
    info->n_tiles = c->d.ntx * c->d.ntx;
    info->variant = c->var;
    info->step = c->step;
    info->overflow_tiles = (int64_t)ovf;
    info->device_bytes = (int64_t)c->pool_bytes;
    return DPD_OK;
}

}  // extern "C"
