// Device-side building blocks of the DPD dimer simulator (sm_103a).
//
// Model: Hinz, Panchenko, Kim & Fried, arXiv:1310.0998, Sec. 2 (forces),
// Sec. 5 (velocity-Verlet, periodic square).  Random numbers: Philox4x32-10
// (Salmon et al., SC'11).
//
// Positions are 32-bit fixed point: coordinate X in [0, 2^32) stands for
// x = X L / 2^32.  Resolution is uniform over the box (L 2^-32), the periodic
// wrap is the natural overflow of unsigned addition, the minimum-image
// displacement is the signed difference (int32)(X_i - X_j), and the cell of a
// bead is (X nc) >> 32 exactly.  Velocities and forces are FP32.
//
// Data layout in HBM (one system; the ensemble packs several side by side):
//   S_xv  uint4[N]   pre-force state (X, Y, bits of v*x, v*y) sorted by cell,
//                    where v* is the half-step velocity v_{s-1/2} (v_s at set-up)
//   S_id  u32[N]     bead id of each sorted slot
//   slot  u32[N]     id -> sorted slot (to find a bead's bonded partner)
//   U_*             next pre-force state written by the force kernel, in the
//                    order of S, plus each bead's rank inside its new cell
//   counts, cstart   cell populations and their exclusive prefix sum
//   C_xv, C_f        canonical (X_s, v_s), f_s in id order (last step of a call)
// Cells are numbered tile-major: the domain is cut into B x B cell blocks
// ("tiles", ragged at the high edge) and the cells of one tile are
// consecutive, so a tile's own beads form one contiguous run of S.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

enum : int { ERR_NONFINITE = 1, ERR_TIMEOUT = 2, ERR_INTERNAL = 4 };
enum : int { F_FIRST = 1, F_FINAL = 2, F_ADVANCE = 4 };

constexpr int THERMO_CAP = 65536;   // per-step (KE, Px, Py, -) ring
constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 16;        // cells per thread in the scan
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;
constexpr long long SPIN_LIMIT = 1ll << 22;  // bounded waits (x ~100 ns)

// Per-system view handed to every kernel by value.
struct Sys {
    double Ld, ulen_d, inv_ulen_d; // L, L / 2^32 and 2^32 / L in double (state conversion)
    float L, ulen, inv_ulen, cs;   // ulen = L / 2^32, inv_ulen = 2^32 / L
    int nc, ntx, n, ncells;
    float rc2, inv_rc, a, gamma, sig_r, kbond, r0, fp, zeta, dt, hdtm;
    float hwexp;                   // s/2 of w_R = w^(s/2) when gen_w
    float rc2u, inv_rcu;           // r_c^2 in fixed-point units^2, and ulen / r_c
    int gen_w;                     // 1: dissipative weight exponent s != 2
    uint32_t key0, key1;
    uint32_t rk0[10], rk1[10];   // Philox round keys key + r * (Weyl increments)
    int noise, excl, cap;
    uint4 *S_xv;
    uint32_t *S_id;
    uint4 *U_xv;
    uint32_t *U_id, *U_rank;
    uint32_t *slot, *counts, *cstart;
    uint4 *C_xv;
    float2 *C_f;
    double *thermo;
    long long *step;
    uint32_t *pcnt;
    unsigned long long *ovf;
    int *err;
    long long *errinfo;   // first failed check: site, then three values
    unsigned long long *scan_status, *scan_ticket;
};

// ---------------------------------------------------------------- Philox ----
// One Philox4x32-10 evaluation.  Round: multiply words 0 and 2 by the two
// round multipliers, mix the high halves with words 1, 3 and the key, keep
// the low halves; the key advances by the Weyl increments between rounds.
__device__ __forceinline__ void philox10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                         uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Same bijection with the ten round keys precomputed (k + r W per round).
__device__ __forceinline__ void philox10_rk(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                            const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ rk0[r];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk1[r];
        c3 = lo0;
    }
}

// Random factor of the pair (i, j) at step s: F_R = sig_r * w * noise.
// Uniform: the odd integer 2 (w0 >> 8) + 1 - 2^24 (|.| < 2^24, exact in FP32);
// sig_r carries sqrt(2 gamma kBT / dt) * sqrt(3) * 2^-24.
// Gaussian: Box-Muller on the top 24 bits of w0, w1; sig_r = sqrt(2 gamma kBT / dt).
__device__ __forceinline__ float pair_noise(const Sys &d, uint32_t ia, uint32_t ib, uint32_t s_lo,
                                            uint32_t s_hi)
{
    uint32_t c0 = min(ia, ib), c1 = max(ia, ib), c2 = s_lo, c3 = s_hi;
    philox10_rk(c0, c1, c2, c3, d.rk0, d.rk1);
    // 2 (w0 >> 8) + 1 - 2^24, formed exactly in FP32 (every term is an
    // integer below 2^25 in magnitude with at most 24 significant bits)
    if (d.noise == 0) return fmaf((float)(c0 >> 8), 2.0f, 1.0f - 16777216.0f);
    const float u1 = __fmul_rn(__fadd_rn((float)(c0 >> 8), 0.5f), 5.9604644775390625e-08f);
    const float u2 = __fmul_rn(__fadd_rn((float)(c1 >> 8), 0.5f), 5.9604644775390625e-08f);
    return __fmul_rn(__fsqrt_rn(__fmul_rn(-2.0f, logf(u1))), cospif(__fmul_rn(2.0f, u2)));
}

// ---------------------------------------------------------- cell geometry ----
// Cell coordinate of a fixed-point coordinate: floor(x nc / L) = (X nc) >> 32.
__device__ __forceinline__ int cell_coord(const Sys &d, uint32_t X) { return (int)__umulhi(X, (uint32_t)d.nc); }

template <int B>
__device__ __forceinline__ int cell_of(const Sys &d, int cx, int cy)
{
    const int tx = cx / B, lx = cx - tx * B, ty = cy / B, ly = cy - ty * B;
    const int th = min(B, d.nc - ty * B), tw = min(B, d.nc - tx * B);
    return ty * B * d.nc + tx * B * th + ly * tw + lx;
}

// Minimum-image displacement x_a - x_b in length units (exact integer
// difference, one rounding in the conversion).
__device__ __forceinline__ float mdiff(const Sys &d, uint32_t a, uint32_t b)
{
    return __fmul_rn((float)(int)(a - b), d.ulen);
}

// Fixed-point step of a coordinate by a displacement dx (|dx| < L/2):
// rounded to the nearest unit, wrapped by unsigned overflow.
__device__ __forceinline__ uint32_t fx_add(const Sys &d, uint32_t X, float dx)
{
    return X + (uint32_t)__float2int_rn(__fmul_rn(dx, d.inv_ulen));
}

__device__ __forceinline__ float vbits(uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ uint32_t fbits(float f) { return __float_as_uint(f); }

__device__ __forceinline__ void set_err(const Sys &d, int bits) { atomicOr(d.err, bits); }

// Record the first failed check (site code and three values) beside the bits.
__device__ __forceinline__ void set_err_at(const Sys &d, int bits, int site, long long a, long long b, long long c)
{
    atomicOr(d.err, bits);
    if (atomicCAS((unsigned long long *)d.errinfo, 0ull, (unsigned long long)site) == 0ull) {
        d.errinfo[1] = a;
        d.errinfo[2] = b;
        d.errinfo[3] = c;
    }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace dpd
