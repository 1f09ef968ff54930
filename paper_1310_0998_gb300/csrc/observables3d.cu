// Observables of Secs. 5.3-5.4 (arXiv:1310.0998) for the three-dimensional
// variant (include/dpd.h, dpd3_velocity_field / energy_spectrum / vorticity /
// velocity_correlation), FP64 on the device.
//
// The paper defines them in two dimensions; each carries over axis by axis:
//   agent COM     c_k = x_tail + 1/2 minimg(x_head - x_tail), wrapped;
//                 v_k = (v_head + v_tail) / 2
//   u_M           cubic window of side eps around (i + 1/2) L/M per axis,
//                 closed, minimum image; mean COM velocity inside, 0 if empty;
//                 default eps = L (N_f / N)^(1/3), N_f = 10 (the window holds
//                 N_f agents on average, as the square window of Eq.
//                 filterwidth does in two dimensions)
//   E(k)          uhat = M^-3 sum u e^{-2 pi i k.x/L}; E(k) = sum over
//                 nint|k| = k of (|uhat_x|^2 + |uhat_y|^2 + |uhat_z|^2) / 2,
//                 k = 1..M/2.  z1 = u_x + i u_y and z2 = u_z are transformed;
//                 k -> -k maps a shell onto itself, so the shell sum of
//                 |Z1|^2 + |Z2|^2 equals M^6 times that of the three |uhat|^2
//   omega         curl u_M by second-order central differences
//   g_v, L_gv     agent pairs a < b within r_max: bin floor(r / dr) of the
//                 COM separation r = sqrt((dx^2 + dy^2) + dz^2), sums of
//                 v_a . v_b (a cell grid of side >= r_max, or all pairs);
//                 g_v(b) = (<v_a . v_b>_b - |<v>|^2) / (<|v|^2> - |<v>|^2),
//                 L_gv by the trapezoid rule over r = 0 (g = 1) and the
//                 centres of the non-empty bins
// Window and bin decisions use the same IEEE double operations, in the same
// order, as a plain evaluation of those definitions.
#include <cmath>
#include <vector>

#include "dpd.h"
#include "obs_common.cuh"
#include "sim3d_host.h"

namespace dpd {

// Agent position or velocity, FP64 (x, y, z, padding), 32-byte aligned.
struct __align__(32) D4 {
    double x, y, z, w;
};

__global__ void k3_agent_com(const uint4 *__restrict__ p, const float4 *__restrict__ v, int na, double L, double ulen,
                             D4 *c, D4 *vc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const uint4 h = p[2 * k], t = p[2 * k + 1];
    const double hx = __dmul_rn((double)h.x, ulen), hy = __dmul_rn((double)h.y, ulen), hz = __dmul_rn((double)h.z, ulen);
    const double tx = __dmul_rn((double)t.x, ulen), ty = __dmul_rn((double)t.y, ulen), tz = __dmul_rn((double)t.z, ulen);
    double cx = __dadd_rn(tx, __dmul_rn(0.5, minimg_d(__dsub_rn(hx, tx), L)));
    double cy = __dadd_rn(ty, __dmul_rn(0.5, minimg_d(__dsub_rn(hy, ty), L)));
    double cz = __dadd_rn(tz, __dmul_rn(0.5, minimg_d(__dsub_rn(hz, tz), L)));
    cx = __dsub_rn(cx, __dmul_rn(L, floor(__ddiv_rn(cx, L))));
    cy = __dsub_rn(cy, __dmul_rn(L, floor(__ddiv_rn(cy, L))));
    cz = __dsub_rn(cz, __dmul_rn(L, floor(__ddiv_rn(cz, L))));
    c[k] = D4{cx, cy, cz, 0.0};
    const float4 a = v[2 * k], b = v[2 * k + 1];
    vc[k] = D4{__dmul_rn(0.5, __dadd_rn((double)a.x, (double)b.x)), __dmul_rn(0.5, __dadd_rn((double)a.y, (double)b.y)),
               __dmul_rn(0.5, __dadd_rn((double)a.z, (double)b.z)), 0.0};
}

constexpr int WIN3 = 32;   // window hits per axis (the host keeps eps / (L / M) <= 28)

// Window sums: sum u_x, u_y, u_z and count per grid point (z-major [iz][iy][ix]).
__global__ void k3_deposit(const D4 *c, const D4 *vc, int na, double L, double dxg, double half, int M,
                           double *sx, double *sy, double *sz, double *cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    int ix[WIN3], iy[WIN3], iz[WIN3];
    const D4 ck = c[k], vk = vc[k];
    const int nx = window_hits(ck.x, L, dxg, half, M, ix, WIN3);
    const int ny = window_hits(ck.y, L, dxg, half, M, iy, WIN3);
    const int nz = window_hits(ck.z, L, dxg, half, M, iz, WIN3);
    for (int a = 0; a < nz; ++a)
        for (int b = 0; b < ny; ++b)
            for (int q = 0; q < nx; ++q) {
                const size_t g = ((size_t)iz[a] * M + iy[b]) * M + ix[q];
                atomicAdd(&sx[g], vk.x);
                atomicAdd(&sy[g], vk.y);
                atomicAdd(&sz[g], vk.z);
                atomicAdd(&cnt[g], 1.0);
            }
}

// u = window mean (0 if empty), stored as z1 = u_x + i u_y and z2 = u_z + 0 i.
__global__ void k3_field_finish(const double *sx, const double *sy, const double *sz, const double *cnt, long long MMM,
                                double2 *z1, double2 *z2)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= MMM) return;
    const double n = cnt[g];
    z1[g] = n > 0.0 ? make_double2(sx[g] / n, sy[g] / n) : make_double2(0.0, 0.0);
    z2[g] = make_double2(n > 0.0 ? sz[g] / n : 0.0, 0.0);
}

__global__ void k3_field_out(const double2 *z1, const double2 *z2, long long MMM, double *u)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= MMM) return;
    u[3 * g] = z1[g].x;
    u[3 * g + 1] = z1[g].y;
    u[3 * g + 2] = z2[g].x;
}

// omega = curl u by central differences on the periodic grid (spacing h):
// (d u_z/dy - d u_y/dz, d u_x/dz - d u_z/dx, d u_y/dx - d u_x/dy).
__global__ void k3_vorticity(const double2 *__restrict__ z1, const double2 *__restrict__ z2, int M, double inv2h,
                             double *__restrict__ om)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long MM = (long long)M * M;
    if (g >= MM * M) return;
    const int iz = (int)(g / MM), iy = (int)((g / M) % M), ix = (int)(g % M);
    const int xp = ix + 1 == M ? 0 : ix + 1, xm = ix == 0 ? M - 1 : ix - 1;
    const int yp = iy + 1 == M ? 0 : iy + 1, ym = iy == 0 ? M - 1 : iy - 1;
    const int zp = iz + 1 == M ? 0 : iz + 1, zm = iz == 0 ? M - 1 : iz - 1;
    auto at = [&](int z, int y, int x) { return ((long long)z * M + y) * M + x; };
    const double duz_dy = __dsub_rn(z2[at(iz, yp, ix)].x, z2[at(iz, ym, ix)].x);
    const double duy_dz = __dsub_rn(z1[at(zp, iy, ix)].y, z1[at(zm, iy, ix)].y);
    const double dux_dz = __dsub_rn(z1[at(zp, iy, ix)].x, z1[at(zm, iy, ix)].x);
    const double duz_dx = __dsub_rn(z2[at(iz, iy, xp)].x, z2[at(iz, iy, xm)].x);
    const double duy_dx = __dsub_rn(z1[at(iz, iy, xp)].y, z1[at(iz, iy, xm)].y);
    const double dux_dy = __dsub_rn(z1[at(iz, yp, ix)].x, z1[at(iz, ym, ix)].x);
    om[3 * g] = __dsub_rn(__dmul_rn(duz_dy, inv2h), __dmul_rn(duy_dz, inv2h));
    om[3 * g + 1] = __dsub_rn(__dmul_rn(dux_dz, inv2h), __dmul_rn(duz_dx, inv2h));
    om[3 * g + 2] = __dsub_rn(__dmul_rn(duy_dx, inv2h), __dmul_rn(dux_dy, inv2h));
}

// Shell sums of (|Z1|^2 + |Z2|^2) scale, per block in shared memory first.
__global__ void k3_shells(const double2 *Z1, const double2 *Z2, int M, double scale, double *E)
{
    extern __shared__ double es[];
    const int nsh = M / 2;
    for (int i = threadIdx.x; i < nsh; i += blockDim.x) es[i] = 0.0;
    __syncthreads();
    const long long MM = (long long)M * M;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < MM * M;
         g += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(g / MM), iy = (int)((g / M) % M), ix = (int)(g % M);
        const int kz = iz < M / 2 ? iz : iz - M, ky = iy < M / 2 ? iy : iy - M, kx = ix < M / 2 ? ix : ix - M;
        const int sh = (int)rint(sqrt((double)(kx * kx + ky * ky + kz * kz)));
        if (sh >= 1 && sh <= nsh) {
            const double2 a = Z1[g], b = Z2[g];
            atomicAdd(&es[sh - 1], (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y) * scale);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nsh; i += blockDim.x)
        if (es[i] != 0.0) atomicAdd(&E[i], es[i]);
}

__global__ void k3_vmeans(const D4 *v, int na, double *acc)
{
    double sx = 0, sy = 0, sz = 0, s2 = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < na; k += gridDim.x * blockDim.x) {
        const D4 a = v[k];
        sx += a.x;
        sy += a.y;
        sz += a.z;
        s2 += a.x * a.x + a.y * a.y + a.z * a.z;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], sx);
        atomicAdd(&acc[1], sy);
        atomicAdd(&acc[2], sz);
        atomicAdd(&acc[3], s2);
    }
}

// All pairs a < b: one block per (row tile, column tile >= row tile) of the
// upper triangle, the column tile staged in shared memory, per-bin sums in
// shared memory.  The bin is taken in FP32 where sqrt(r2)/dr lies at least
// 1e-3 from a bin edge (its error there is ~1e-4), else by the FP64 formula.
constexpr int VCF3_TILE = 256;
__global__ void __launch_bounds__(VCF3_TILE) k3_vcf(const D4 *c, const D4 *v, int na, double L, double dr,
                                                    int nbins, double *gnum, unsigned long long *gcnt)
{
    extern __shared__ unsigned char smem3[];
    double *snum = (double *)smem3;
    unsigned long long *scnt = (unsigned long long *)(snum + nbins);
    D4 *sc = (D4 *)(((uintptr_t)(scnt + nbins) + 31) & ~(uintptr_t)31);
    D4 *sv = sc + VCF3_TILE;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) { snum[b] = 0.0; scnt[b] = 0ull; }
    const long long nt = (na + VCF3_TILE - 1) / VCF3_TILE, bid = blockIdx.x;
    // row ti starts at S(ti) = ti nt - ti (ti - 1) / 2 blocks: invert by a
    // square root, then correct by single steps
    const double disc = (2.0 * nt + 1.0) * (2.0 * nt + 1.0) - 8.0 * (double)bid;
    long long ti = (long long)floor(((2.0 * nt + 1.0) - sqrt(fmax(disc, 0.0))) * 0.5);
    ti = ti < 0 ? 0 : (ti > nt - 1 ? nt - 1 : ti);
    while (ti > 0 && ti * nt - ti * (ti - 1) / 2 > bid) --ti;
    while (ti < nt - 1 && (ti + 1) * nt - (ti + 1) * ti / 2 <= bid) ++ti;
    const long long tj = ti + (bid - (ti * nt - ti * (ti - 1) / 2));
    const int a = (int)(ti * VCF3_TILE) + threadIdx.x;
    const int jb = (int)(tj * VCF3_TILE);
    for (int q = threadIdx.x; q < VCF3_TILE; q += blockDim.x) {
        const int j = jb + q;
        sc[q] = j < na ? c[j] : D4{0.0, 0.0, 0.0, 0.0};
        sv[q] = j < na ? v[j] : D4{0.0, 0.0, 0.0, 0.0};
    }
    __syncthreads();
    if (a < na) {
        const D4 ca = c[a], va = v[a];
        const int jn = min(VCF3_TILE, na - jb);
        const double hL = 0.5 * L;
        const double rmax2 = (double)nbins * dr * (double)nbins * dr * (1.0 + 1e-9);
        const float inv_drf = (float)(1.0 / dr), nbf = (float)nbins;
        for (int q = 0; q < jn; ++q) {
            const int j = jb + q;
            if (j <= a) continue;
            // agent centres lie on the L / 2^33 grid, so d / L never rounds onto
            // +-1/2 and this comparison equals d - L rint(d / L)
            double dx = __dsub_rn(ca.x, sc[q].x), dy = __dsub_rn(ca.y, sc[q].y), dz = __dsub_rn(ca.z, sc[q].z);
            dx = dx > hL ? __dsub_rn(dx, L) : (dx < -hL ? __dadd_rn(dx, L) : dx);
            dy = dy > hL ? __dsub_rn(dy, L) : (dy < -hL ? __dadd_rn(dy, L) : dy);
            dz = dz > hL ? __dsub_rn(dz, L) : (dz < -hL ? __dadd_rn(dz, L) : dz);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (!(r2 < rmax2)) continue;
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
            const double dot = __dadd_rn(__dadd_rn(__dmul_rn(va.x, sv[q].x), __dmul_rn(va.y, sv[q].y)),
                                         __dmul_rn(va.z, sv[q].z));
            atomicAdd(&snum[b], dot);
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

// Pairs within r_max only: agents counting-sorted into a periodic grid of
// n_v^3 cells of side cw >= r_max (z-major), one block per cell taking its
// agents against its own cell (b after a) and the 13 forward neighbours
// (dz > 0, or dz = 0 and dy > 0, or dz = dy = 0 and dx > 0), staged in
// shared memory in chunks.  The shell is taken from FP32 offsets to the
// block's cell corner where r / dr lies at least 1e-3 from a shell edge and
// from r_max, else by the FP64 expressions of k3_vcf, so every pair lands in
// the shell the all-pairs pass gives it; per-warp FP64 histograms.
constexpr int VCF3C_THREADS = 128, VCF3C_CHUNK = 256, VCF3C_WARPS = VCF3C_THREADS / 32;

__device__ __forceinline__ int vcf3_cell(const D4 &p, double cw, int nv)
{
    auto one = [&](double x) {
        const int c = (int)floor(__ddiv_rn(x, cw));
        return c < 0 ? 0 : (c >= nv ? nv - 1 : c);
    };
    return (one(p.z) * nv + one(p.y)) * nv + one(p.x);
}

__global__ void k3_vcf_count(const D4 *c, int na, double cw, int nv, unsigned *cnt, unsigned *rank)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    rank[k] = atomicAdd(&cnt[vcf3_cell(c[k], cw, nv)], 1u);
}

__global__ void k3_vcf_scatter(const D4 *c, const D4 *v, int na, double cw, int nv, const unsigned *start,
                               const unsigned *rank, D4 *sc, D4 *sv)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= na) return;
    const D4 p = c[k];
    const unsigned dst = start[vcf3_cell(p, cw, nv)] + rank[k];
    if (dst < (unsigned)na) {
        sc[dst] = p;
        sv[dst] = v[k];
    }
}

__global__ void __launch_bounds__(VCF3C_THREADS) k3_vcf_cells(const D4 *sc, const D4 *sv, const unsigned *start,
                                                              int nv, double L, double cw, double dr, int nbins,
                                                              double *gnum, unsigned long long *gcnt)
{
    extern __shared__ __align__(32) unsigned char smem3c[];
    D4 *bc = (D4 *)smem3c;                                                   // [VCF3C_CHUNK]
    D4 *bv = bc + VCF3C_CHUNK;
    float4 *bo = (float4 *)(bv + VCF3C_CHUNK);
    double *snum = (double *)(bo + VCF3C_CHUNK);                             // [VCF3C_WARPS][nbins]
    unsigned long long *scnt = (unsigned long long *)(snum + VCF3C_WARPS * nbins);
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < VCF3C_WARPS * nbins; i += blockDim.x) { snum[i] = 0.0; scnt[i] = 0ull; }
    const int cell = blockIdx.x, cz = cell / (nv * nv), cy = (cell / nv) % nv, cx = cell % nv;
    const unsigned a0 = start[cell], a1 = start[cell + 1];
    const double ox = cx * cw, oy = cy * cw, oz = cz * cw, hL = 0.5 * L;
    const double rmax2 = (double)nbins * dr * (double)nbins * dr * (1.0 + 1e-9);
    const float rscr = (float)(nbins * dr) * 1.0001f + 1e-4f * (float)cw, rscr2 = rscr * rscr;
    const float inv_drf = (float)(1.0 / dr), nbf = (float)nbins;
    double *wnum = snum + warp * nbins;
    unsigned long long *wcnt = scnt + warp * nbins;
    for (int nb = 0; nb < 14; ++nb) {
        // nb = 0: own cell; 1..13: the forward half of the 26 neighbours
        int dxc = 0, dyc = 0, dzc = 0;
        if (nb > 0) {
            const int o = nb + 13;   // offsets 14..26 of the 3 x 3 x 3 block in z-major order
            dzc = o / 9 - 1;
            dyc = (o / 3) % 3 - 1;
            dxc = o % 3 - 1;
        }
        int nx = cx + dxc, ny = cy + dyc, nz = cz + dzc;
        double sx = 0.0, sy = 0.0, sz = 0.0;
        if (nx >= nv) { nx -= nv; sx = L; } else if (nx < 0) { nx += nv; sx = -L; }
        if (ny >= nv) { ny -= nv; sy = L; } else if (ny < 0) { ny += nv; sy = -L; }
        if (nz >= nv) { nz -= nv; sz = L; }
        const int nc = (nz * nv + ny) * nv + nx;
        const unsigned b0 = start[nc], b1 = start[nc + 1];
        for (unsigned c0 = b0; c0 < b1; c0 += VCF3C_CHUNK) {
            const int m = (int)min((unsigned)VCF3C_CHUNK, b1 - c0);
            __syncthreads();
            for (int q = threadIdx.x; q < m; q += blockDim.x) {
                const D4 p = sc[c0 + q];
                bc[q] = p;
                bv[q] = sv[c0 + q];
                bo[q] = make_float4((float)(p.x + sx - ox), (float)(p.y + sy - oy), (float)(p.z + sz - oz), 0.f);
            }
            __syncthreads();
            for (unsigned a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
                const D4 ca = sc[a], va = sv[a];
                const float ax = (float)(ca.x - ox), ay = (float)(ca.y - oy), az = (float)(ca.z - oz);
                const int q0 = nb == 0 ? (int)max(0ll, (long long)a + 1 - (long long)c0) : 0;
                for (int q = q0; q < m; ++q) {
                    const float fx = ax - bo[q].x, fy = ay - bo[q].y, fz = az - bo[q].z;
                    const float r2f = fx * fx + fy * fy + fz * fz;
                    if (r2f >= rscr2) continue;
                    const float tf = sqrtf(r2f) * inv_drf;
                    const float fl = floorf(tf);
                    int bin;
                    if (tf - fl > 1e-3f && fl + 1.0f - tf > 1e-3f && tf < nbf - 1e-3f) {
                        bin = (int)fl;
                    } else {
                        const D4 cb = bc[q];
                        double dx = __dsub_rn(ca.x, cb.x), dy = __dsub_rn(ca.y, cb.y), dz = __dsub_rn(ca.z, cb.z);
                        dx = dx > hL ? __dsub_rn(dx, L) : (dx < -hL ? __dadd_rn(dx, L) : dx);
                        dy = dy > hL ? __dsub_rn(dy, L) : (dy < -hL ? __dadd_rn(dy, L) : dy);
                        dz = dz > hL ? __dsub_rn(dz, L) : (dz < -hL ? __dadd_rn(dz, L) : dz);
                        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                        if (!(r2 < rmax2)) continue;
                        const double bf = floor(__ddiv_rn(sqrt(r2), dr));
                        if (!(bf < (double)nbins)) continue;
                        bin = (int)bf;
                    }
                    const D4 vb = bv[q];
                    atomicAdd(&wnum[bin], __dadd_rn(__dadd_rn(__dmul_rn(va.x, vb.x), __dmul_rn(va.y, vb.y)),
                                                    __dmul_rn(va.z, vb.z)));
                    atomicAdd(&wcnt[bin], 1ull);
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        double sn = 0.0;
        unsigned long long cn = 0ull;
        for (int w = 0; w < VCF3C_WARPS; ++w) { sn += snum[w * nbins + b]; cn += scnt[w * nbins + b]; }
        if (cn) {
            atomicAdd(&gnum[b], sn);
            atomicAdd(&gcnt[b], cn);
        }
    }
}

}  // namespace dpd

using namespace dpd;

#define CUO3(x)                                                                     \
    do {                                                                            \
        const cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

static char *scratch3(dpd3_ctx *c, size_t bytes)
{
    if (c->obs_bytes < bytes) {
        if (c->obs) cudaFree(c->obs);
        c->obs = nullptr;
        c->obs_bytes = 0;
        if (cudaMalloc(&c->obs, bytes) != cudaSuccess) return nullptr;
        c->obs_bytes = bytes;
    }
    return (char *)c->obs;
}

static double default_eps3(const dpd3_ctx *c)
{
    return c->p.L * std::cbrt(10.0 / (double)(c->s.b.n / 2));
}

// Field on the device: z1 (u_x + i u_y) and z2 (u_z) [M^3] double2, back to
// back (one FFT launch per axis covers both), cnt [M^3], and a tail of at
// least tail_bytes.  Every sub-buffer starts on a 256-byte boundary.
static int field3_device(dpd3_ctx *c, int M, double eps, size_t tail_bytes, double2 **z_out, double **cnt_out,
                         char **tail)
{
    const int na = c->s.b.n / 2;
    const size_t MMM = (size_t)M * M * M;
    auto up = [](size_t o) { return (o + 255) & ~size_t(255); };
    const size_t o_cc = 0, o_vv = up(o_cc + 32 * (size_t)na), o_s = up(o_vv + 32 * (size_t)na);
    const size_t o_z = up(o_s + 32 * MMM), o_tail = up(o_z + 32 * MMM);
    char *b = scratch3(c, o_tail + tail_bytes + 256);
    if (!b) return DPD_ERR_OOM;
    D4 *cc = (D4 *)(b + o_cc), *vv = (D4 *)(b + o_vv);
    double *sx = (double *)(b + o_s), *sy = sx + MMM, *sz = sy + MMM, *cn = sz + MMM;   // one clear
    double2 *z = (double2 *)(b + o_z);
    const double L = c->p.L;
    CUO3(cudaMemsetAsync(sx, 0, 32 * MMM, c->st));
    k3_agent_com<<<(na + 255) / 256, 256, 0, c->st>>>(c->s.C_p, c->s.C_v, na, L, c->s.b.ulen_d, cc, vv);
    k3_deposit<<<(na + 127) / 128, 128, 0, c->st>>>(cc, vv, na, L, L / M, 0.5 * eps, M, sx, sy, sz, cn);
    k3_field_finish<<<(unsigned)((MMM + 255) / 256), 256, 0, c->st>>>(sx, sy, sz, cn, (long long)MMM, z, z + MMM);
    CUO3(cudaGetLastError());
    *z_out = z;
    *cnt_out = cn;
    if (tail) *tail = b + o_tail;
    return DPD_OK;
}

static int check_field_args(dpd3_ctx *c, int M, double *eps)
{
    if (!c->have_state) return DPD_ERR_STATE;
    if (*eps <= 0.0) *eps = default_eps3(c);
    if (!(*eps / (c->p.L / M) <= 28.0)) return DPD_ERR_INVALID_ARG;   // window wider than 28 grid points
    return DPD_OK;
}

extern "C" {

int dpd3_velocity_field(dpd3_ctx *c, int M, double eps, double *u, double *n_in)
{
    if (!c || !u || M < 2 || M > 256) return DPD_ERR_INVALID_ARG;
    int rc = check_field_args(c, M, &eps);
    if (rc) return rc;
    const size_t MMM = (size_t)M * M * M;
    double2 *z;
    double *cn;
    char *tail;
    rc = field3_device(c, M, eps, 24 * MMM, &z, &cn, &tail);
    if (rc) return rc;
    double *du = (double *)tail;
    k3_field_out<<<(unsigned)((MMM + 255) / 256), 256, 0, c->st>>>(z, z + MMM, (long long)MMM, du);
    CUO3(cudaGetLastError());
    CUO3(cudaMemcpyAsync(u, du, 24 * MMM, cudaMemcpyDeviceToHost, c->st));
    if (n_in) CUO3(cudaMemcpyAsync(n_in, cn, 8 * MMM, cudaMemcpyDeviceToHost, c->st));
    return dpd3_internal_latched(c);
}

int dpd3_energy_spectrum(dpd3_ctx *c, int M, double eps, double *E)
{
    if (!c || !E || M < 4 || M > 256 || (M & (M - 1))) return DPD_ERR_INVALID_ARG;
    int rc = check_field_args(c, M, &eps);
    if (rc) return rc;
    const long long MM = (long long)M * M, MMM = MM * M;
    double2 *z;
    double *cn;
    char *tail;
    rc = field3_device(c, M, eps, 8 * (size_t)(M / 2), &z, &cn, &tail);
    if (rc) return rc;
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const size_t sm = 16 * (size_t)M;
    const int thr = M / 2;
    const unsigned lines = (unsigned)(2 * MM);   // M^2 lines per axis in each of z1, z2
    k_fft<<<lines, thr, sm, c->st>>>(z, M, logM, 1, (int)(2 * MM), M, 0);    // along x
    k_fft<<<lines, thr, sm, c->st>>>(z, M, logM, M, M, 1, MM);               // along y
    k_fft<<<lines, thr, sm, c->st>>>(z, M, logM, MM, (int)MM, 1, MMM);       // along z
    double *dE = (double *)tail;
    CUO3(cudaMemsetAsync(dE, 0, 8 * (size_t)(M / 2), c->st));
    const double M3 = (double)MMM;
    const long long blocks = std::min<long long>((MMM + 255) / 256, 4096);
    k3_shells<<<(unsigned)blocks, 256, 8 * (size_t)(M / 2), c->st>>>(z, z + MMM, M, 0.5 / (M3 * M3), dE);
    CUO3(cudaGetLastError());
    CUO3(cudaMemcpyAsync(E, dE, 8 * (size_t)(M / 2), cudaMemcpyDeviceToHost, c->st));
    return dpd3_internal_latched(c);
}

int dpd3_vorticity(dpd3_ctx *c, int M, double eps, double *omega)
{
    if (!c || !omega || M < 3 || M > 256) return DPD_ERR_INVALID_ARG;
    int rc = check_field_args(c, M, &eps);
    if (rc) return rc;
    const size_t MMM = (size_t)M * M * M;
    double2 *z;
    double *cn;
    char *tail;
    rc = field3_device(c, M, eps, 24 * MMM, &z, &cn, &tail);
    if (rc) return rc;
    double *om = (double *)tail;
    k3_vorticity<<<(unsigned)((MMM + 255) / 256), 256, 0, c->st>>>(z, z + MMM, M, (double)M / (2.0 * c->p.L), om);
    CUO3(cudaGetLastError());
    CUO3(cudaMemcpyAsync(omega, om, 24 * MMM, cudaMemcpyDeviceToHost, c->st));
    return dpd3_internal_latched(c);
}

int dpd3_velocity_correlation(dpd3_ctx *c, double dr, int nbins, double *g, double *L_int, double *num,
                              int64_t *cnt)
{
    if (!c || !g || !(dr > 0) || nbins < 1 || nbins > 4096) return DPD_ERR_INVALID_ARG;
    if (!c->have_state) return DPD_ERR_STATE;
    const int na = c->s.b.n / 2;
    const double L = c->p.L;
    // a cell grid of side >= r_max when at least three cells fit per side (and
    // the grid stays below 16.8 M cells), else all agent pairs; both decide a
    // pair's shell with the same FP64 expressions
    const double rmax = (double)nbins * dr * (1.0 + 1e-9);
    const double nv_d = std::floor(L / rmax);
    const bool cells = nv_d >= 3.0 && nv_d <= 256.0;
    const int nv = cells ? (int)nv_d : 0;
    const size_t ncell = (size_t)nv * nv * nv;
    const long long ntile = (na + VCF3_TILE - 1) / VCF3_TILE, nblk = ntile * (ntile + 1) / 2;
    if (!cells && nblk > 2147483647ll) return DPD_ERR_INVALID_ARG;
    auto up = [](size_t o) { return (o + 255) & ~size_t(255); };
    const size_t o_cc = 0, o_vv = up(32 * (size_t)na), o_num = up(o_vv + 32 * (size_t)na),
                 o_cnt = up(o_num + 8 * (size_t)nbins), o_acc = up(o_cnt + 8 * (size_t)nbins),
                 o_ccnt = up(o_acc + 256), o_cst = up(o_ccnt + 4 * ncell), o_rnk = up(o_cst + 4 * (ncell + 1)),
                 o_scs = up(o_rnk + (cells ? 4 * (size_t)na : 0)), o_svs = up(o_scs + (cells ? 32 * (size_t)na : 0)),
                 bytes = up(o_svs + (cells ? 32 * (size_t)na : 0));
    char *b = scratch3(c, bytes);
    if (!b) return DPD_ERR_OOM;
    D4 *cc = (D4 *)(b + o_cc), *vv = (D4 *)(b + o_vv);
    double *gnum = (double *)(b + o_num), *acc = (double *)(b + o_acc);
    unsigned long long *gcnt = (unsigned long long *)(b + o_cnt);
    CUO3(cudaMemsetAsync(gnum, 0, 8 * (size_t)nbins, c->st));
    CUO3(cudaMemsetAsync(gcnt, 0, 8 * (size_t)nbins, c->st));
    CUO3(cudaMemsetAsync(acc, 0, 64, c->st));
    k3_agent_com<<<(na + 255) / 256, 256, 0, c->st>>>(c->s.C_p, c->s.C_v, na, L, c->s.b.ulen_d, cc, vv);
    k3_vmeans<<<64, 256, 0, c->st>>>(vv, na, acc);
    if (cells) {
        const double cw = L / nv;
        unsigned *ccnt = (unsigned *)(b + o_ccnt), *cst = (unsigned *)(b + o_cst), *rnk = (unsigned *)(b + o_rnk);
        D4 *scs = (D4 *)(b + o_scs), *svs = (D4 *)(b + o_svs);
        CUO3(cudaMemsetAsync(ccnt, 0, 4 * ncell, c->st));
        k3_vcf_count<<<(na + 255) / 256, 256, 0, c->st>>>(cc, na, cw, nv, ccnt, rnk);
        k_vcf_scan<<<1, 1024, 0, c->st>>>(ccnt, (int)ncell, cst);
        k3_vcf_scatter<<<(na + 255) / 256, 256, 0, c->st>>>(cc, vv, na, cw, nv, cst, rnk, scs, svs);
        const size_t sm = (size_t)VCF3C_CHUNK * 80 + (size_t)VCF3C_WARPS * nbins * 16;
        if (sm > 200 * 1024) return DPD_ERR_INVALID_ARG;
        CUO3(cudaFuncSetAttribute(k3_vcf_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k3_vcf_cells<<<(unsigned)ncell, VCF3C_THREADS, sm, c->st>>>(scs, svs, cst, nv, L, cw, dr, nbins, gnum, gcnt);
    } else {
        const size_t sm = 16 * (size_t)nbins + 32 + 64 * VCF3_TILE;
        if (sm > 200 * 1024) return DPD_ERR_INVALID_ARG;
        CUO3(cudaFuncSetAttribute(k3_vcf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k3_vcf<<<(unsigned)nblk, VCF3_TILE, sm, c->st>>>(cc, vv, na, L, dr, nbins, gnum, gcnt);
    }
    CUO3(cudaGetLastError());
    std::vector<double> hn(nbins), ha(4);
    std::vector<unsigned long long> hc(nbins);
    CUO3(cudaMemcpyAsync(hn.data(), gnum, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, c->st));
    CUO3(cudaMemcpyAsync(hc.data(), gcnt, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, c->st));
    CUO3(cudaMemcpyAsync(ha.data(), acc, 32, cudaMemcpyDeviceToHost, c->st));
    const int rc = dpd3_internal_latched(c);
    const double mx = ha[0] / na, my = ha[1] / na, mz = ha[2] / na, v2 = ha[3] / na;
    const double m2 = mx * mx + my * my + mz * mz, den = v2 - m2;
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
