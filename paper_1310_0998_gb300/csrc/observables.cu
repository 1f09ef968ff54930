// Observables of Sec. 5.3-5.4 (arXiv:1310.0998) on the device, FP64.
//
//   agent COM     c_k = x_tail + 1/2 minimg(x_head - x_tail), wrapped;
//                 v_k = (v_head + v_tail)/2                       (Sec. 5.3)
//   u_M           square window of side eps around (i + 1/2) L/M, closed,
//                 minimum image; mean COM velocity inside, 0 if empty
//                 (Sec. 5.4, Eq. filterwidth)
//   E(k)          z = u_x + i u_y, Z = FFT2(z); |uhat_x|^2 + |uhat_y|^2 summed
//                 over a shell equals |Z|^2 / (2 M^4) summed over the same
//                 shell, because k -> -k maps each shell onto itself
//                 (Eqs. fourierTrans01, ESPf)
//   g_v, L_gv     pair histogram of COM separations, sums of v_a . v_b
//                 (Eqs. VCF, spatial01)
// Window and bin decisions use the same IEEE double operations, in the same
// order, as a plain evaluation of those definitions (explicit _rn intrinsics,
// no contraction), so they are reproducible bit for bit off the device.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dpd.h"
#include "obs_common.cuh"
#include "sim_host.h"

namespace dpd {

struct ObsScratch {
    void *buf = nullptr;
    size_t bytes = 0;
};

// Positions enter as the exact doubles X L / 2^32 of the fixed-point state.
__global__ void k_agent_com(const uint4 *__restrict__ xv, int na, double L, double ulen, double2 *c, double2 *v)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const uint4 h = xv[2 * k], t = xv[2 * k + 1];
    const double hx = __dmul_rn((double)h.x, ulen), hy = __dmul_rn((double)h.y, ulen);
    const double tx = __dmul_rn((double)t.x, ulen), ty = __dmul_rn((double)t.y, ulen);
    const double dx = minimg_d(__dsub_rn(hx, tx), L);
    const double dy = minimg_d(__dsub_rn(hy, ty), L);
    double cx = __dadd_rn(tx, __dmul_rn(0.5, dx));
    double cy = __dadd_rn(ty, __dmul_rn(0.5, dy));
    cx = __dsub_rn(cx, __dmul_rn(L, floor(__ddiv_rn(cx, L))));
    cy = __dsub_rn(cy, __dmul_rn(L, floor(__ddiv_rn(cy, L))));
    c[k] = make_double2(cx, cy);
    const double hvx = (double)__uint_as_float(h.z), hvy = (double)__uint_as_float(h.w);
    const double tvx = (double)__uint_as_float(t.z), tvy = (double)__uint_as_float(t.w);
    v[k] = make_double2(__dmul_rn(0.5, __dadd_rn(hvx, tvx)), __dmul_rn(0.5, __dadd_rn(hvy, tvy)));
}

__global__ void k_deposit(const double2 *c, const double2 *v, int na, double L, double dxg, double half, int M,
                          double *sx, double *sy, double *cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int ix[64], iy[64];
    const double2 ck = c[k], vk = v[k];
    const int nx = window_hits(ck.x, L, dxg, half, M, ix, 64);
    const int ny = window_hits(ck.y, L, dxg, half, M, iy, 64);
    for (int a = 0; a < ny; ++a)
        for (int b = 0; b < nx; ++b) {
            const size_t g = (size_t)iy[a] * M + ix[b];
            atomicAdd(&sx[g], vk.x);
            atomicAdd(&sy[g], vk.y);
            atomicAdd(&cnt[g], 1.0);
        }
}

__global__ void k_field_finish(const double *sx, const double *sy, const double *cnt, int MM, double2 *z)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= MM) return;
    const double n = cnt[g];
    z[g] = n > 0.0 ? make_double2(sx[g] / n, sy[g] / n) : make_double2(0.0, 0.0);
}

// Scalar vorticity of the field, omega = du_y/dx - du_x/dy (Sec. 5.3), by
// second-order central differences on the periodic grid of spacing h.
__global__ void k_vorticity(const double2 *__restrict__ z, int M, double inv2h, double *__restrict__ om)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M * M) return;
    const int iy = g / M, ix = g - iy * M;
    const int xp = ix + 1 == M ? 0 : ix + 1, xm = ix == 0 ? M - 1 : ix - 1;
    const int yp = iy + 1 == M ? 0 : iy + 1, ym = iy == 0 ? M - 1 : iy - 1;
    const double duy = __dsub_rn(z[(size_t)iy * M + xp].y, z[(size_t)iy * M + xm].y);
    const double dux = __dsub_rn(z[(size_t)yp * M + ix].x, z[(size_t)ym * M + ix].x);
    om[g] = __dsub_rn(__dmul_rn(duy, inv2h), __dmul_rn(dux, inv2h));
}

__global__ void k_shells(const double2 *Z, int M, double scale, double *E)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M * M) return;
    const int iy = g / M, ix = g - iy * M;
    const int ky = iy < M / 2 ? iy : iy - M, kx = ix < M / 2 ? ix : ix - M;
    const int sh = (int)rint(sqrt((double)(kx * kx + ky * ky)));
    if (sh >= 1 && sh <= M / 2) {
        const double2 a = Z[g];
        atomicAdd(&E[sh - 1], (a.x * a.x + a.y * a.y) * scale);
    }
}

__global__ void k_vmeans(const double2 *v, int na, double *acc)
{
    double sx = 0, sy = 0, s2 = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < na; k += gridDim.x * blockDim.x) {
        const double2 a = v[k];
        sx += a.x;
        sy += a.y;
        s2 += a.x * a.x + a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], sx);
        atomicAdd(&acc[1], sy);
        atomicAdd(&acc[2], s2);
    }
}

// All pairs a < b of agents: separation bin floor(r / dr) (IEEE double, as
// written), accumulate v_a . v_b and the pair count per bin in shared memory.
constexpr int VCF_TILE = 256;
__global__ void __launch_bounds__(VCF_TILE) k_vcf(const double2 *c, const double2 *v, int na, double L, double dr,
                                                  int nbins, double *gnum, unsigned long long *gcnt)
{
    extern __shared__ unsigned char smem[];
    double *snum = (double *)smem;
    unsigned long long *scnt = (unsigned long long *)(snum + nbins);
    double2 *sc = (double2 *)(scnt + nbins);
    double2 *sv = sc + VCF_TILE;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) { snum[b] = 0.0; scnt[b] = 0ull; }
    const int ntile = (na + VCF_TILE - 1) / VCF_TILE;
    // block -> (row tile ti, column tile tj >= ti) over the upper triangle
    // row ti starts at S(ti) = ti*ntile - ti*(ti-1)/2; invert with a square
    // root and correct by one step either way
    const long long bid = blockIdx.x, nt = ntile;
    const double disc = (2.0 * nt + 1.0) * (2.0 * nt + 1.0) - 8.0 * (double)bid;
    long long ti = (long long)floor(((2.0 * nt + 1.0) - sqrt(fmax(disc, 0.0))) * 0.5);
    ti = ti < 0 ? 0 : (ti > nt - 1 ? nt - 1 : ti);
    while (ti > 0 && ti * nt - ti * (ti - 1) / 2 > bid) --ti;
    while (ti < nt - 1 && (ti + 1) * nt - (ti + 1) * ti / 2 <= bid) ++ti;
    const int tj = (int)(ti + (bid - (ti * nt - ti * (ti - 1) / 2)));
    const int a = (int)ti * VCF_TILE + threadIdx.x;
    const int jb = tj * VCF_TILE;
    for (int q = threadIdx.x; q < VCF_TILE; q += blockDim.x) {
        const int j = jb + q;
        sc[q] = j < na ? c[j] : make_double2(0.0, 0.0);
        sv[q] = j < na ? v[j] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (a < na) {
        const double2 ca = c[a], va = v[a];
        const int jn = min(VCF_TILE, na - jb);
        const double hL = 0.5 * L;
        const double rmax2 = (double)nbins * dr * (double)nbins * dr * (1.0 + 1e-9);
        const float inv_drf = (float)(1.0 / dr), nbf = (float)nbins;
        for (int q = 0; q < jn; ++q) {
            const int j = jb + q;
            if (j <= a) continue;
            // minimum image: agent centres lie on the L / 2^33 grid, so d / L never
            // rounds onto +-1/2 and the comparison equals d - L rint(d / L)
            double dx = __dsub_rn(ca.x, sc[q].x), dy = __dsub_rn(ca.y, sc[q].y);
            dx = dx > hL ? __dsub_rn(dx, L) : (dx < -hL ? __dadd_rn(dx, L) : dx);
            dy = dy > hL ? __dsub_rn(dy, L) : (dy < -hL ? __dadd_rn(dy, L) : dy);
            const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            if (!(r2 < rmax2)) continue;   // beyond the last bin (a margin above it)
            // bin floor(sqrt(r2) / dr): FP32 where the value is at least 1e-3 from
            // a bin edge (its error here is ~1e-4), else the FP64 expression
            const float tf = sqrtf((float)r2) * inv_drf;
            const float fl = floorf(tf);
            int b;
            if (tf - fl > 1e-3f && fl + 1.0f - tf > 1e-3f && tf < nbf - 1e-3f) {
                b = (int)fl;
            } else {
                const double bf = floor(__ddiv_rn(sqrt(r2), dr));
                if (!(bf < (double)nbins)) continue;
                b = (int)bf;
            }
            atomicAdd(&snum[b], __dadd_rn(__dmul_rn(va.x, sv[q].x), __dmul_rn(va.y, sv[q].y)));
            atomicAdd(&scnt[b], 1ull);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (scnt[b]) {
            atomicAdd(&gnum[b], snum[b]);
            atomicAdd(&gcnt[b], scnt[b]);
        }
    }
}

// Sum over agents of |v_COM| with v_COM = (v_head + v_tail) / 2, FP64.
__global__ void k_agent_speed(const uint4 *__restrict__ xv, int na, double *acc)
{
    double s = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < na; k += gridDim.x * blockDim.x) {
        const uint4 h = xv[2 * k], t = xv[2 * k + 1];
        const double vx = __dmul_rn(0.5, __dadd_rn((double)__uint_as_float(h.z), (double)__uint_as_float(t.z)));
        const double vy = __dmul_rn(0.5, __dadd_rn((double)__uint_as_float(h.w), (double)__uint_as_float(t.w)));
        s += sqrt(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// ---- velocity correlation limited to r < r_max = nbins dr ------------------
// Agents are counting-sorted into a periodic grid of ncv x ncv cells of side
// L / ncv >= r_max, so every pair inside r_max lies in the same or an
// adjacent cell.  One block per cell takes its own agents against the agents
// of the cell itself (b after a) and of its four forward neighbours (E, NE,
// N, NW), each neighbour cell staged in shared memory in chunks.  Separations
// are taken in FP32 from offsets to the block's cell corner (error below
// 1e-5); a pair whose r / dr lies within 1e-3 of a shell edge or of r_max is
// decided by the FP64 expressions of k_vcf instead, so the shell of every
// pair, and hence the counts, equal the all-pairs kernel's; the products
// v_a . v_b are FP64 as there.
constexpr int VCFC_THREADS = 128, VCFC_CHUNK = 512, VCFC_WARPS = VCFC_THREADS / 32;

__device__ __forceinline__ int vcf_cell_of(double x, double cw, int ncv)
{
    const int c = (int)floor(__ddiv_rn(x, cw));
    return c < 0 ? 0 : (c >= ncv ? ncv - 1 : c);
}

__global__ void k_vcf_count(const double2 *c, int na, double cw, int ncv, unsigned *cnt, unsigned *rank)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const double2 p = c[k];
    const int cell = vcf_cell_of(p.y, cw, ncv) * ncv + vcf_cell_of(p.x, cw, ncv);
    rank[k] = atomicAdd(&cnt[cell], 1u);
}

__global__ void k_vcf_scatter(const double2 *c, const double2 *v, int na, double cw, int ncv, const unsigned *start,
                              const unsigned *rank, double2 *sc, double2 *sv)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const double2 p = c[k];
    const int cell = vcf_cell_of(p.y, cw, ncv) * ncv + vcf_cell_of(p.x, cw, ncv);
    const unsigned dst = start[cell] + rank[k];
    if (dst < (unsigned)na) {
        sc[dst] = p;
        sv[dst] = v[k];
    }
}

__global__ void __launch_bounds__(VCFC_THREADS) k_vcf_cells(const double2 *sc, const double2 *sv,
                                                            const unsigned *start, int ncv, double L, double cw,
                                                            double dr, int nbins, double *gnum,
                                                            unsigned long long *gcnt)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *snum = (double *)smem;                                          // [VCFC_WARPS][nbins]
    unsigned long long *scnt = (unsigned long long *)(snum + VCFC_WARPS * nbins);
    double2 *bc = (double2 *)(scnt + VCFC_WARPS * nbins);                   // [VCFC_CHUNK]
    double2 *bv = bc + VCFC_CHUNK;
    float2 *bo = (float2 *)(bv + VCFC_CHUNK);
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < VCFC_WARPS * nbins; i += blockDim.x) { snum[i] = 0.0; scnt[i] = 0ull; }
    const int cell = blockIdx.x, cy = cell / ncv, cx = cell - cy * ncv;
    const unsigned a0 = start[cell], a1 = start[cell + 1];
    const double ox = cx * cw, oy = cy * cw, hL = 0.5 * L;
    const double rmax2 = (double)nbins * dr * (double)nbins * dr * (1.0 + 1e-9);
    const float rscr = (float)(nbins * dr) * 1.0001f + 1e-4f * (float)cw, rscr2 = rscr * rscr;
    const float inv_drf = (float)(1.0 / dr), nbf = (float)nbins;
    double *wnum = snum + warp * nbins;
    unsigned long long *wcnt = scnt + warp * nbins;
    for (int nb = 0; nb < 5; ++nb) {
        // own cell, then E, NE, N, NW; periodic images carry their shift
        const int dxc = nb == 0 ? 0 : (nb <= 2 ? 1 : (nb == 3 ? 0 : -1));
        const int dyc = nb <= 1 ? 0 : 1;
        int nx = cx + dxc, ny = cy + dyc;
        double sx = 0.0, sy = 0.0;
        if (nx >= ncv) { nx -= ncv; sx = L; } else if (nx < 0) { nx += ncv; sx = -L; }
        if (ny >= ncv) { ny -= ncv; sy = L; }
        const int nc = ny * ncv + nx;
        const unsigned b0 = start[nc], b1 = start[nc + 1];
        for (unsigned c0 = b0; c0 < b1; c0 += VCFC_CHUNK) {
            const int m = (int)min((unsigned)VCFC_CHUNK, b1 - c0);
            __syncthreads();
            for (int q = threadIdx.x; q < m; q += blockDim.x) {
                const double2 p = sc[c0 + q];
                bc[q] = p;
                bv[q] = sv[c0 + q];
                bo[q] = make_float2((float)(p.x + sx - ox), (float)(p.y + sy - oy));
            }
            __syncthreads();
            for (unsigned a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const double2 ca = sc[a], va = sv[a];
                const float ax = (float)(ca.x - ox), ay = (float)(ca.y - oy);
                const int q0 = nb == 0 ? (int)max(0ll, (long long)a + 1 - (long long)c0) : 0;
                for (int q = q0; q < m; ++q) {
                    const float fx = ax - bo[q].x, fy = ay - bo[q].y;
                    const float r2f = fx * fx + fy * fy;
                    if (r2f >= rscr2) continue;
                    // the shell from the FP32 separation (error below 1e-5)
                    // wherever r / dr lies at least 1e-3 from a shell edge
                    // and from r_max; otherwise the FP64 expressions of k_vcf
                    const float tf = sqrtf(r2f) * inv_drf;
                    const float fl = floorf(tf);
                    int bin;
                    if (tf - fl > 1e-3f && fl + 1.0f - tf > 1e-3f && tf < nbf - 1e-3f) {
                        bin = (int)fl;
                    } else {
                        const double2 cb = bc[q];
                        double dx = __dsub_rn(ca.x, cb.x), dy = __dsub_rn(ca.y, cb.y);
                        dx = dx > hL ? __dsub_rn(dx, L) : (dx < -hL ? __dadd_rn(dx, L) : dx);
                        dy = dy > hL ? __dsub_rn(dy, L) : (dy < -hL ? __dadd_rn(dy, L) : dy);
                        const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                        if (!(r2 < rmax2)) continue;
                        const double bf = floor(__ddiv_rn(sqrt(r2), dr));
                        if (!(bf < (double)nbins)) continue;
                        bin = (int)bf;
                    }
                    const double2 vb = bv[q];
                    atomicAdd(&wnum[bin], __dadd_rn(__dmul_rn(va.x, vb.x), __dmul_rn(va.y, vb.y)));
                    atomicAdd(&wcnt[bin], 1ull);
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        double sn = 0.0;
        unsigned long long cn = 0ull;
        for (int w = 0; w < VCFC_WARPS; ++w) { sn += snum[w * nbins + b]; cn += scnt[w * nbins + b]; }
        if (cn) {
            atomicAdd(&gnum[b], sn);
            atomicAdd(&gcnt[b], cn);
        }
    }
}

}  // namespace dpd

using namespace dpd;

static ObsScratch *scratch_of(dpd_ctx *c, size_t bytes)
{
    static_assert(sizeof(void *) == 8, "64-bit only");
    auto *s = reinterpret_cast<ObsScratch *>(c->obs);
    if (!s) {
        s = new ObsScratch();
        c->obs = s;
    }
    if (s->bytes < bytes) {
        if (s->buf) cudaFree(s->buf);
        s->buf = nullptr;
        s->bytes = 0;
        if (cudaMalloc(&s->buf, bytes) != cudaSuccess) return nullptr;
        s->bytes = bytes;
    }
    return s;
}

void dpd_internal_free_obs(dpd_ctx *c)
{
    auto *s = reinterpret_cast<ObsScratch *>(c->obs);
    if (s) {
        if (s->buf) cudaFree(s->buf);
        delete s;
        c->obs = nullptr;
    }
}

#define CUO(x)                                                    \
    do {                                                          \
        const cudaError_t e_ = (x);                               \
        if (e_ != cudaSuccess)                                    \
            return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

// Field on the device: z [M*M] double2 (u_x, u_y), cnt [M*M], and a tail of
// at least tail_bytes for the caller.  Every sub-buffer starts on a 256-byte
// boundary (z is read as double2, which needs 16; an odd M*M must not shift it).
static int field_device(dpd_ctx *c, int M, double eps, size_t tail_bytes, double2 **z_out, double **cnt_out,
                        char **tail)
{
    const int na = c->d.n / 2;
    const size_t MM = (size_t)M * M;
    auto up = [](size_t o) { return (o + 255) & ~size_t(255); };
    const size_t o_cc = 0, o_vv = up(o_cc + 16 * (size_t)na), o_s = up(o_vv + 16 * (size_t)na);
    const size_t o_z = up(o_s + 24 * MM), o_tail = up(o_z + 16 * MM);
    ObsScratch *s = scratch_of(c, o_tail + tail_bytes + 256);
    if (!s) return DPD_ERR_OOM;
    char *b = (char *)s->buf;
    double2 *cc = (double2 *)(b + o_cc);
    double2 *vv = (double2 *)(b + o_vv);
    double *sx = (double *)(b + o_s), *sy = sx + MM, *cn = sy + MM;   // contiguous: one clear
    double2 *z = (double2 *)(b + o_z);
    const double L = c->p.L;
    if (eps <= 0.0) eps = L * std::sqrt(10.0 / (double)na);
    CUO(cudaMemsetAsync(sx, 0, 8 * MM * 3, c->st));
    k_agent_com<<<(na + 255) / 256, 256, 0, c->st>>>(c->d.C_xv, na, L, c->d.ulen_d, cc, vv);
    k_deposit<<<(na + 127) / 128, 128, 0, c->st>>>(cc, vv, na, L, L / M, 0.5 * eps, M, sx, sy, cn);
    k_field_finish<<<(int)((MM + 255) / 256), 256, 0, c->st>>>(sx, sy, cn, (int)MM, z);
    CUO(cudaGetLastError());
    *z_out = z;
    *cnt_out = cn;
    if (tail) *tail = b + o_tail;
    return DPD_OK;
}

extern "C" {

int dpd_velocity_field(dpd_ctx *c, int M, double eps, double *u, double *n_in)
{
    if (!c || !u || M < 2 || M > 1024) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    if (eps <= 0.0) eps = c->p.L * std::sqrt(10.0 / (double)(c->d.n / 2));
    if (eps / (c->p.L / M) > 56.0) return DPD_ERR_INVALID_ARG;   // window wider than 56 grid points
    double2 *z;
    double *cn;
    int rc = field_device(c, M, eps, 0, &z, &cn, nullptr);
    if (rc) return rc;
    const size_t MM = (size_t)M * M;
    CUO(cudaMemcpyAsync(u, z, 16 * MM, cudaMemcpyDeviceToHost, c->st));
    if (n_in) CUO(cudaMemcpyAsync(n_in, cn, 8 * MM, cudaMemcpyDeviceToHost, c->st));
    return dpd_internal_latched(c);
}

int dpd_energy_spectrum(dpd_ctx *c, int M, double eps, double *E)
{
    if (!c || !E || M < 4 || M > 1024 || (M & (M - 1))) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    if (eps <= 0.0) eps = c->p.L * std::sqrt(10.0 / (double)(c->d.n / 2));
    if (eps / (c->p.L / M) > 56.0) return DPD_ERR_INVALID_ARG;
    double2 *z;
    double *cn;
    char *tail;
    int rc = field_device(c, M, eps, 8 * (size_t)(M / 2), &z, &cn, &tail);
    if (rc) return rc;
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const size_t sm = 16 * (size_t)M;
    const int thr = M / 2 < 512 ? M / 2 : 512;
    k_fft<<<M, thr, sm, c->st>>>(z, M, logM, 1, M, M, 0);   // rows (along x)
    k_fft<<<M, thr, sm, c->st>>>(z, M, logM, M, M, 1, 0);   // columns (along y)
    double *dE = (double *)tail;
    CUO(cudaMemsetAsync(dE, 0, 8 * (size_t)(M / 2), c->st));
    const double M2 = (double)M * (double)M;
    k_shells<<<(M * M + 255) / 256, 256, 0, c->st>>>(z, M, 0.5 / (M2 * M2), dE);
    CUO(cudaGetLastError());
    CUO(cudaMemcpyAsync(E, dE, 8 * (size_t)(M / 2), cudaMemcpyDeviceToHost, c->st));
    return dpd_internal_latched(c);
}

int dpd_vorticity(dpd_ctx *c, int M, double eps, double *omega)
{
    if (!c || !omega || M < 3 || M > 1024) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const int na = c->d.n / 2;
    if (eps <= 0.0) eps = c->p.L * std::sqrt(10.0 / (double)na);
    if (eps / (c->p.L / M) > 56.0) return DPD_ERR_INVALID_ARG;
    const size_t MM = (size_t)M * M;
    double2 *z;
    double *cn;
    char *tail;
    int rc = field_device(c, M, eps, 8 * MM, &z, &cn, &tail);
    if (rc) return rc;
    double *om = (double *)tail;
    k_vorticity<<<(int)((MM + 255) / 256), 256, 0, c->st>>>(z, M, (double)M / (2.0 * c->p.L), om);
    CUO(cudaGetLastError());
    CUO(cudaMemcpyAsync(omega, om, 8 * MM, cudaMemcpyDeviceToHost, c->st));
    return dpd_internal_latched(c);
}

int dpd_agent_speed(dpd_ctx *c, double *mean_speed)
{
    if (!c || !mean_speed) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const int na = c->d.n / 2;
    ObsScratch *s = scratch_of(c, 256);
    if (!s) return DPD_ERR_OOM;
    double *acc = (double *)s->buf;
    CUO(cudaMemsetAsync(acc, 0, 8, c->st));
    k_agent_speed<<<std::min((na + 255) / 256, 1024), 256, 0, c->st>>>(c->d.C_xv, na, acc);
    CUO(cudaGetLastError());
    double h = 0.0;
    CUO(cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, c->st));
    const int rc = dpd_internal_latched(c);
    *mean_speed = h / na;
    return rc;
}

int dpd_velocity_correlation(dpd_ctx *c, double dr, int nbins, double *g, double *L_int, double *num,
                             int64_t *cnt)
{
    if (!c || !g || !(dr > 0) || nbins < 1 || nbins > 8192) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const int na = c->d.n / 2;
    const double L = c->p.L;
    // pairs within r_max = nbins dr only: a cell grid of side >= r_max when at
    // least three cells fit per side (and the grid stays below 4 M cells),
    // else all pairs; both evaluate a pair with the same arithmetic
    const double rmax = (double)nbins * dr * (1.0 + 1e-9);
    const double ncv_d = std::floor(L / rmax);
    const bool cells = ncv_d >= 3.0 && ncv_d <= 2048.0;
    const int ncv = cells ? (int)ncv_d : 0, ncell = ncv * ncv;
    const size_t a256 = 256;
    auto up = [&](size_t x) { return (x + a256 - 1) & ~(a256 - 1); };
    const size_t o_cc = 0, o_vv = up(o_cc + 16 * (size_t)na), o_num = up(o_vv + 16 * (size_t)na),
                 o_cnt = up(o_num + 8 * (size_t)nbins), o_acc = up(o_cnt + 8 * (size_t)nbins),
                 o_ccnt = up(o_acc + 64), o_cst = up(o_ccnt + 4 * (size_t)ncell),
                 o_rnk = up(o_cst + 4 * ((size_t)ncell + 1)), o_scs = up(o_rnk + (cells ? 4 * (size_t)na : 0)),
                 o_svs = up(o_scs + (cells ? 16 * (size_t)na : 0)), bytes = up(o_svs + (cells ? 16 * (size_t)na : 0));
    ObsScratch *s = scratch_of(c, bytes);
    if (!s) return DPD_ERR_OOM;
    char *b = (char *)s->buf;
    double2 *cc = (double2 *)(b + o_cc), *vv = (double2 *)(b + o_vv);
    double *gnum = (double *)(b + o_num);
    unsigned long long *gcnt = (unsigned long long *)(b + o_cnt);
    double *acc = (double *)(b + o_acc);
    CUO(cudaMemsetAsync(gnum, 0, 8 * (size_t)nbins, c->st));
    CUO(cudaMemsetAsync(gcnt, 0, 8 * (size_t)nbins, c->st));
    CUO(cudaMemsetAsync(acc, 0, 64, c->st));
    k_agent_com<<<(na + 255) / 256, 256, 0, c->st>>>(c->d.C_xv, na, L, c->d.ulen_d, cc, vv);
    k_vmeans<<<64, 256, 0, c->st>>>(vv, na, acc);
    if (cells) {
        const double cw = L / ncv;
        unsigned *ccnt = (unsigned *)(b + o_ccnt), *cst = (unsigned *)(b + o_cst), *rnk = (unsigned *)(b + o_rnk);
        double2 *scs = (double2 *)(b + o_scs), *svs = (double2 *)(b + o_svs);
        CUO(cudaMemsetAsync(ccnt, 0, 4 * (size_t)ncell, c->st));
        k_vcf_count<<<(na + 255) / 256, 256, 0, c->st>>>(cc, na, cw, ncv, ccnt, rnk);
        k_vcf_scan<<<1, 1024, 0, c->st>>>(ccnt, ncell, cst);
        k_vcf_scatter<<<(na + 255) / 256, 256, 0, c->st>>>(cc, vv, na, cw, ncv, cst, rnk, scs, svs);
        const size_t sm = (size_t)VCFC_WARPS * nbins * 16 + (size_t)VCFC_CHUNK * 40;
        if (sm > 200 * 1024) return DPD_ERR_INVALID_ARG;
        CUO(cudaFuncSetAttribute(k_vcf_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_vcf_cells<<<ncell, VCFC_THREADS, sm, c->st>>>(scs, svs, cst, ncv, L, cw, dr, nbins, gnum, gcnt);
    } else {
        const int ntile = (na + VCF_TILE - 1) / VCF_TILE;
        const long long nblk = (long long)ntile * (ntile + 1) / 2;
        const size_t sm = 16 * (size_t)nbins + 32 * VCF_TILE;
        if (sm > 200 * 1024 || nblk > 2147483647ll) return DPD_ERR_INVALID_ARG;
        CUO(cudaFuncSetAttribute(k_vcf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_vcf<<<(unsigned)nblk, VCF_TILE, sm, c->st>>>(cc, vv, na, L, dr, nbins, gnum, gcnt);
    }
    CUO(cudaGetLastError());
    std::vector<double> hn(nbins), ha(3);
    std::vector<unsigned long long> hc(nbins);
    CUO(cudaMemcpyAsync(hn.data(), gnum, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, c->st));
    CUO(cudaMemcpyAsync(hc.data(), gcnt, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, c->st));
    CUO(cudaMemcpyAsync(ha.data(), acc, 24, cudaMemcpyDeviceToHost, c->st));
    const int rc = dpd_internal_latched(c);
    const double mx = ha[0] / na, my = ha[1] / na, v2 = ha[2] / na, m2 = mx * mx + my * my;
    const double den = v2 - m2;
    double li = 0.0, rprev = 0.0, gprev = 1.0;
    for (int k = 0; k < nbins; ++k) {
        if (hc[k] > 0 && den > 0) {
            g[k] = (hn[k] / (double)hc[k] - m2) / den;
            const double r = (k + 0.5) * dr;
            li += 0.5 * (g[k] + gprev) * (r - rprev);
            rprev = r;
            gprev = g[k];
        } else {
            g[k] = NAN;
        }
        if (num) num[k] = hn[k];
        if (cnt) cnt[k] = (int64_t)hc[k];
    }
    if (L_int) *L_int = den > 0 ? li : NAN;
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// E(k) with no allocation: dpd_energy_spectrum_noalloc.
//
// Which callers cannot allocate, and why.  dpd_energy_spectrum grows a scratch
// buffer with cudaMalloc on first use (and again when a larger M or box comes
// along).  Two kinds of caller cannot accept that in the middle of a run: one
// whose simulation state was sized to fill the device's memory (the largest
// boxes), where the late cudaMalloc fails; and one that samples E(k) every few
// hundred steps from inside a pipelined run, where cudaMalloc / cudaFree
// synchronise the whole device and stall the other streams.  This variant
// keeps its scratch in one fixed static device array instead.
//
// How.  The agent centres of mass and velocities, which the allocating path
// stages in a per-agent buffer, are recomputed inside the deposit kernel
// (k_deposit_state, the same IEEE operations as k_agent_com), so the scratch
// no longer grows with the number of agents; what remains is the grid:
// per point the window sums of u_x and u_y, the window count and the complex
// field (5 doubles), plus M/2 shell sums: 2,622,464 bytes at the maximum
// M = 256.  Larger M is rejected.
//
// What must start at zero.  The three window sums and the shell sums are
// accumulated with atomics; every call clears them (cudaMemsetAsync on the
// caller's stream) before the deposit.  The field is overwritten in full.
//
// Sharing.  There is one array per device, shared by every context on it:
// two calls whose stream work overlaps (two host threads, or two contexts on
// different streams) race on it and return wrong values.  Serialise them.
//
// Set-up.  The first call on a device, made with that device current, looks up
// the array's device address with cudaGetSymbolAddress and keeps it for later
// calls on that device; make that first call before any stream capture.
// ---------------------------------------------------------------------------

namespace {
constexpr int NOALLOC_MAX_M = 256;
constexpr size_t NOALLOC_MAX_GRID = (size_t)NOALLOC_MAX_M * NOALLOC_MAX_M;
constexpr size_t NOALLOC_DOUBLES = 5 * NOALLOC_MAX_GRID + NOALLOC_MAX_M / 2;
constexpr int NOALLOC_MAX_DEVICES = 64;
}  // namespace

static __device__ __align__(256) double g_spectrum_scratch[NOALLOC_DOUBLES];

static double *g_spectrum_scratch_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_spectrum_scratch_mu;

// Device address of the static scratch on the context's device (set-up on the
// first call per device).  The symbol lookup answers for the current device,
// so that must be the device the context was created on.
static int spectrum_scratch(int ctx_dev, double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DPD_ERR_CUDA;
    if (dev != ctx_dev) return DPD_ERR_INVALID_ARG;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return DPD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_spectrum_scratch_mu);
    if (!g_spectrum_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
        if (e != cudaSuccess || !p) return DPD_ERR_CUDA;
        g_spectrum_scratch_ptr[dev] = (double *)p;
    }
    *out = g_spectrum_scratch_ptr[dev];
    return DPD_OK;
}

namespace dpd {

// k_agent_com followed by k_deposit for one agent, without staging the
// centres of mass and velocities in memory.
__global__ void k_deposit_state(const uint4 *__restrict__ xv, int na, double L, double ulen, double dxg,
                                double half, int M, double *sx, double *sy, double *cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const uint4 h = xv[2 * k], t = xv[2 * k + 1];
    const double hx = __dmul_rn((double)h.x, ulen), hy = __dmul_rn((double)h.y, ulen);
    const double tx = __dmul_rn((double)t.x, ulen), ty = __dmul_rn((double)t.y, ulen);
    const double dx = minimg_d(__dsub_rn(hx, tx), L);
    const double dy = minimg_d(__dsub_rn(hy, ty), L);
    double cx = __dadd_rn(tx, __dmul_rn(0.5, dx));
    double cy = __dadd_rn(ty, __dmul_rn(0.5, dy));
    cx = __dsub_rn(cx, __dmul_rn(L, floor(__ddiv_rn(cx, L))));
    cy = __dsub_rn(cy, __dmul_rn(L, floor(__ddiv_rn(cy, L))));
    const double hvx = (double)__uint_as_float(h.z), hvy = (double)__uint_as_float(h.w);
    const double tvx = (double)__uint_as_float(t.z), tvy = (double)__uint_as_float(t.w);
    const double vx = __dmul_rn(0.5, __dadd_rn(hvx, tvx)), vy = __dmul_rn(0.5, __dadd_rn(hvy, tvy));
    int ix[64], iy[64];
    const int nx = window_hits(cx, L, dxg, half, M, ix, 64);
    const int ny = window_hits(cy, L, dxg, half, M, iy, 64);
    for (int a = 0; a < ny; ++a)
        for (int b = 0; b < nx; ++b) {
            const size_t g = (size_t)iy[a] * M + ix[b];
            atomicAdd(&sx[g], vx);
            atomicAdd(&sy[g], vy);
            atomicAdd(&cnt[g], 1.0);
        }
}

}  // namespace dpd

extern "C" int dpd_energy_spectrum_noalloc(dpd_ctx *c, int M, double eps, double *E)
{
    if (!c || !E || M < 4 || M > NOALLOC_MAX_M || (M & (M - 1))) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const int na = c->d.n / 2;
    const double L = c->p.L;
    if (eps <= 0.0) eps = L * std::sqrt(10.0 / (double)na);
    if (eps / (L / M) > 56.0) return DPD_ERR_INVALID_ARG;
    double *scr = nullptr;
    const int rc = spectrum_scratch(c->dev, &scr);
    if (rc) return rc;
    const size_t MM = (size_t)M * M;
    double *sx = scr, *sy = sx + MM, *cn = sy + MM;
    double2 *z = (double2 *)(cn + MM);          // 16-byte aligned: 3 MM doubles, MM even
    double *dE = (double *)(z + MM);
    CUO(cudaMemsetAsync(sx, 0, 8 * MM * 3, c->st));
    CUO(cudaMemsetAsync(dE, 0, 8 * (size_t)(M / 2), c->st));
    k_deposit_state<<<(na + 127) / 128, 128, 0, c->st>>>(c->d.C_xv, na, L, c->d.ulen_d, L / M, 0.5 * eps, M, sx,
                                                         sy, cn);
    k_field_finish<<<(int)((MM + 255) / 256), 256, 0, c->st>>>(sx, sy, cn, (int)MM, z);
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const size_t sm = 16 * (size_t)M;
    const int thr = M / 2 < 512 ? M / 2 : 512;
    k_fft<<<M, thr, sm, c->st>>>(z, M, logM, 1, M, M, 0);
    k_fft<<<M, thr, sm, c->st>>>(z, M, logM, M, M, 1, 0);
    const double M2 = (double)M * (double)M;
    k_shells<<<(M * M + 255) / 256, 256, 0, c->st>>>(z, M, 0.5 / (M2 * M2), dE);
    CUO(cudaGetLastError());
    CUO(cudaMemcpyAsync(E, dE, 8 * (size_t)(M / 2), cudaMemcpyDeviceToHost, c->st));
    return dpd_internal_latched(c);
}
