// Device pieces shared by the two- and three-dimensional observables
// (Secs. 5.3-5.4 of arXiv:1310.0998): the minimum image in FP64, the grid
// points whose filter window holds a coordinate, a radix-2 FFT along one
// axis of a complex grid, and the single-block scan of the velocity
// correlation's cell counts.
#pragma once
#include <cuda_runtime.h>

namespace dpd {

static __device__ __forceinline__ double minimg_d(double d, double L)
{
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// Grid indices i whose window [x_i - eps/2, x_i + eps/2] (minimum image,
// x_i = (i + 1/2) dxg) contains coordinate c; at most min(M, maxout) of them.
static __device__ __forceinline__ int window_hits(double c, double L, double dxg, double half, int M, int *out,
                                                  int maxout)
{
    const double lo = (c - half) / dxg - 0.5, hi = (c + half) / dxg - 0.5;
    int i0 = (int)floor(lo) - 1, i1 = (int)ceil(hi) + 1;
    if (i1 - i0 + 1 > M) { i0 = 0; i1 = M - 1; }
    int n = 0;
    for (int ii = i0; ii <= i1 && n < maxout; ++ii) {
        const int i = ((ii % M) + M) % M;
        const double xm = __dmul_rn(__dadd_rn((double)i, 0.5), dxg);
        const double d = minimg_d(__dsub_rn(xm, c), L);
        if (fabs(d) <= half) out[n++] = i;
    }
    return n;
}

// In-place radix-2 FFT (forward, e^{-2 pi i k n / M}) of M complex doubles
// with stride `stride` between elements.  Block b transforms the line that
// starts at (b / inner) outer_pitch + (b % inner) inner_pitch, so one launch
// covers every line of a 2D grid along either axis, or of a 3D grid along
// any axis.  M/2 threads per block at most, data staged in shared memory.
static __global__ void k_fft(double2 *z, int M, int logM, long long stride, int inner, long long inner_pitch,
                             long long outer_pitch)
{
    extern __shared__ double2 s[];
    const long long b = blockIdx.x;
    double2 *base = z + (b / inner) * outer_pitch + (b % inner) * inner_pitch;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const int r = __brev(i) >> (32 - logM);
        s[r] = base[(long long)i * stride];
    }
    __syncthreads();
    for (int len = 2; len <= M; len <<= 1) {
        const int half = len >> 1;
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            const int grp = t / half, pos = t - grp * half;
            const int i0 = grp * len + pos, i1 = i0 + half;
            double sn, cs;
            sincospi(-2.0 * (double)pos / (double)len, &sn, &cs);
            const double2 a = s[i0], c = s[i1];
            const double2 wc = make_double2(c.x * cs - c.y * sn, c.x * sn + c.y * cs);
            s[i0] = make_double2(a.x + wc.x, a.y + wc.y);
            s[i1] = make_double2(a.x - wc.x, a.y - wc.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) base[(long long)i * stride] = s[i];
}

// Exclusive scan of n counts in one block (n up to a few million): each
// thread sums a contiguous run, a block scan of the run sums, then the runs.
static __global__ void k_vcf_scan(const unsigned *cnt, int n, unsigned *start)
{
    __shared__ unsigned s_sum[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (n + T - 1) / T, b = t * per, e = min(n, b + per);
    unsigned sum = 0;
    for (int i = b; i < e; ++i) sum += cnt[i];
    s_sum[t] = sum;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const unsigned v = t >= o ? s_sum[t - o] : 0u;
        __syncthreads();
        s_sum[t] += v;
        __syncthreads();
    }
    unsigned run = s_sum[t] - sum;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += cnt[i];
    }
    if (t == T - 1) start[n] = s_sum[t];
}

}  // namespace dpd
