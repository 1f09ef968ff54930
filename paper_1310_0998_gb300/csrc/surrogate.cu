// Learned surrogate of the ensemble statistics (include/dpd.h, sur_*).
//
// A deep ensemble of K multilayer perceptrons 4 -> 256 -> 256 -> 40 (SiLU
// hidden activations, linear output) with BF16 weights and activations and
// FP32 accumulation on the tensor cores, trained with Adam on FP32 master
// weights by the kernels below.  Inputs are (area fraction, ln gamma,
// ln zeta, f_p); inputs and targets are standardised with statistics of the
// training set.
//
// All matrix products are one kernel, C[M x N] = A[M x K] B[N x K]^T with
// both operands K-contiguous BF16, computed by warps issuing
// mma.sync.m16n8k16 (BF16 x BF16 -> FP32), with an epilogue chosen per use:
//   forward      Z = X W^T + b; A = silu(Z) stored as BF16 row-major and
//                transposed (the transposed copy feeds the weight gradient)
//   dW           dW = dZ^T X  (A = dZ^T, B = X^T, both batch-contiguous)
//   dX           dA = dZ W    (B = W^T, kept beside W by the optimiser)
//   gate         dZ = dA * silu'(Z), stored as BF16 and transposed
// Padding: K and N are multiples of 16; padded input columns and output rows
// are zero and stay zero (zero gradients under Adam).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dpd.h"

namespace sur {

constexpr int NIN = 4, NIN_P = 16, NH = 256, NOUT = 40, NOUT_P = 48;

enum Epi : int { EPI_F32 = 0, EPI_BIAS_SILU = 1, EPI_BIAS = 2, EPI_GATE = 3 };

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

// C = A B^T.  Block: 4 warps in 2 x 2, each warp a 32 x 32 tile (2 x 4 mma
// tiles of 16 x 8).  Fragments are read straight from global memory (the
// operands are a few hundred KB and stay in L1/L2); rows and columns past
// M or N read as zero and are not stored.
__global__ void __launch_bounds__(128) k_gemm(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                                              int M, int N, int K, int epi, const float *__restrict__ bias,
                                              const float *__restrict__ gateZ, float *__restrict__ C32,
                                              __nv_bfloat16 *__restrict__ C16, __nv_bfloat16 *__restrict__ C16T)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * 64 + (warp >> 1) * 32, n0 = blockIdx.x * 64 + (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[2][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r0 = m0 + 16 * i + g, r1 = r0 + 8;
            const int c = k0 + 2 * t;
            a[i][0] = r0 < M ? ld_pair(A + (size_t)r0 * K + c) : 0u;
            a[i][1] = r1 < M ? ld_pair(A + (size_t)r1 * K + c) : 0u;
            a[i][2] = r0 < M ? ld_pair(A + (size_t)r0 * K + c + 8) : 0u;
            a[i][3] = r1 < M ? ld_pair(A + (size_t)r1 * K + c + 8) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 8 * j + g;
            const int c = k0 + 2 * t;
            b[j][0] = n < N ? ld_pair(B + (size_t)n * K + c) : 0u;
            b[j][1] = n < N ? ld_pair(B + (size_t)n * K + c + 8) : 0u;
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                    "{%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    // epilogue: element (r, c) of fragment q: r = base + g (+8 for q >= 2),
    // c = base + 2t (+1 for odd q)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = m0 + 16 * i + g + (q >= 2 ? 8 : 0);
                const int c = n0 + 8 * j + 2 * t + (q & 1);
                if (r >= M || c >= N) continue;
                float v = acc[i][j][q];
                const size_t o = (size_t)r * N + c;
                if (epi == EPI_F32) {
                    C32[o] = v;
                } else if (epi == EPI_BIAS) {
                    C32[o] = v + bias[c];
                } else if (epi == EPI_BIAS_SILU) {
                    v += bias[c];
                    C32[o] = v;
                    const __nv_bfloat16 h = __float2bfloat16_rn(silu(v));
                    C16[o] = h;
                    C16T[(size_t)c * M + r] = h;
                } else {   // EPI_GATE
                    const __nv_bfloat16 h = __float2bfloat16_rn(v * dsilu(gateZ[o]));
                    C16[o] = h;
                    C16T[(size_t)c * M + r] = h;
                }
            }
}

// Standardised inputs, BF16, row-major [M][16] and transposed [16][M];
// x = (phi, ln gamma, ln zeta, f_p), columns 4..15 and rows past n zero.
__global__ void k_inputs(const float *__restrict__ X, int n, int M, const float *__restrict__ mu,
                         const float *__restrict__ sd, __nv_bfloat16 *X0, __nv_bfloat16 *X0T)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    for (int c = 0; c < NIN_P; ++c) {
        float v = 0.f;
        if (r < n && c < NIN) {
            float x = X[(size_t)r * NIN + c];
            if (c == 1 || c == 2) x = logf(fmaxf(x, 1e-30f));
            v = (x - mu[c]) / sd[c];
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        X0[(size_t)r * NIN_P + c] = h;
        X0T[(size_t)c * M + r] = h;
    }
}

// Loss gradient of the mean squared error over the n x NOUT standardised
// targets: dY = 2 (Y - T) / (n NOUT), as BF16 row-major and transposed; the
// squared error is accumulated into *loss.
__global__ void k_loss(const float *__restrict__ Y, const float *__restrict__ T, int n, int M, float *loss,
                       __nv_bfloat16 *dY, __nv_bfloat16 *dYT, float *dY32)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * NOUT_P) return;
    const int r = idx / NOUT_P, c = idx - r * NOUT_P;
    float gsum = 0.f, d = 0.f;
    if (r < n && c < NOUT) {
        d = Y[(size_t)r * NOUT_P + c] - T[(size_t)r * NOUT + c];
        gsum = d * d;
        d = 2.0f * d / (float)(n * NOUT);
    }
    dY32[idx] = d;
    const __nv_bfloat16 h = __float2bfloat16_rn(d);
    dY[idx] = h;
    dYT[(size_t)c * M + r] = h;
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    if ((threadIdx.x & 31) == 0 && gsum != 0.f) atomicAdd(loss, gsum);
}

// Bias gradient: column sums of a [M][N] FP32 (dY) or BF16 (dZ) matrix.
__global__ void k_colsum(const float *__restrict__ D32, const __nv_bfloat16 *__restrict__ D16, int M, int N,
                         float *out)
{
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < M; r += blockDim.x)
        s += D32 ? D32[(size_t)r * N + c] : __bfloat162float(D16[(size_t)r * N + c]);
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[c] = t;
    }
}

// Adam on FP32 master parameters; writes the BF16 copies W [rows][cols] and
// W^T [cols][rows] (matrices) or nothing else (biases, wbf = nullptr).
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int n, int cols, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16 *wbf, __nv_bfloat16 *wbfT, int rows)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wbf) {
        const int r = i / cols, c = i - r * cols;
        const __nv_bfloat16 h = __float2bfloat16_rn(wi);
        wbf[i] = h;
        wbfT[(size_t)c * rows + r] = h;
    }
}

// Output: de-standardised mean and spread over the K members.
__global__ void k_predict_out(const float *__restrict__ Yall, int K, int n, int M, const float *__restrict__ mu,
                              const float *__restrict__ sd, float *Y, float *spread)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * NOUT) return;
    const int r = idx / NOUT, c = idx - r * NOUT;
    float s = 0.f, s2 = 0.f;
    for (int k = 0; k < K; ++k) {
        const float y = Yall[((size_t)k * M + r) * NOUT_P + c] * sd[c] + mu[c];
        s += y;
        s2 += y * y;
    }
    const float mean = s / K;
    Y[idx] = mean;
    if (spread) spread[idx] = K > 1 ? sqrtf(fmaxf(s2 / K - mean * mean, 0.f)) : 0.f;
}

// ---------------------------------------------------------------------------
// Forward pass on the 5th-generation tensor cores, for batches of 128 rows or
// more (prediction).  Conventions shared by the pieces below: operands sit in
// shared memory in the canonical no-swizzle K-major layout (core matrices of
// 8 rows x 16 bytes; core matrices adjacent in K 128 bytes apart = leading
// byte offset; 8-row groups (K/8) * 128 bytes apart = stride byte offset);
// one thread issues tcgen05.mma (kind::f16: BF16 x BF16 -> FP32 in tensor
// memory, 128 x N x 16 per instruction) and commits to an mbarrier; every
// thread waits on it a bounded number of times and the CTA takes one common
// decision on a timeout (flag the error word, wait once more for the MMAs in
// flight, free the tensor memory, return); tcgen05.ld reads the accumulator
// back, warp w holding rows 32w..32w+31 (one row per lane).
constexpr int TC_M = 128;
constexpr long long TC_SPIN = 1ll << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // bits 46-47: descriptor version 1
}

// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A BF16 (7-9 = 1),
// B BF16 (10-12 = 1), A and B K-major (bits 15, 16 = 0), N/8 at 17-22, M/16 at 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    for (long long i = 0; i < TC_SPIN; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Fused forward pass of one member for 128-row tiles, persistent (one CTA per
// SM).  The CTA stages W1, W2, W3 once as K-major core matrices (8, 128 and
// 24 KB) and keeps them in shared memory; per tile the inputs go into the
// activation buffer (64 KB) and each layer runs as tcgen05.mma into one of two
// 256-column tensor-memory accumulators, alternating from layer to layer.  The
// epilogue of a layer reads its accumulator back in four chunks of 64 columns
// (16 warps: warp w takes rows 32 (w % 4) .. +31 and 16 of the chunk's
// columns), adds the bias, applies SiLU and writes the BF16 activations into
// the activation buffer in the operand layout of the next layer; as soon as a
// chunk is written, one thread issues the next layer's products over those 64
// K columns into the other accumulator, so the tensor cores work while the
// warps run the rest of the epilogue.  A warp signals a written chunk on the
// chunk's mbarrier and goes on (its tensor-memory load of the next chunk is
// already in flight); only the issuing thread waits for all 16 warps.  The
// next tile's first layer is issued before the last layer's 48 output columns
// are read back and stored.  231,664 bytes of shared memory, 512
// tensor-memory columns.
constexpr int FW_W1 = NH * NIN_P * 2, FW_W2 = NH * NH * 2, FW_W3 = NOUT_P * NH * 2, FW_ACT = TC_M * NH * 2;
constexpr int FW_BIAS = (NH + NH + NOUT_P) * 4;
constexpr int FW_SMEM = FW_W1 + FW_W2 + FW_W3 + FW_ACT + FW_BIAS + 48;

// [rows x K] K-contiguous BF16 (leading dimension ld) -> K-major core
// matrices: 16-byte chunk (r, c) at ((r/8) (K/8) + c) 128 + (r%8) 16.
__device__ __forceinline__ void stage_kmajor(unsigned char *dst, const __nv_bfloat16 *src, int rows, int K, int ld)
{
    const int ncm = K >> 3;
    for (int q = threadIdx.x; q < rows * ncm; q += blockDim.x) {
        const int r = q / ncm, c = q - r * ncm;
        const uint4 v = *reinterpret_cast<const uint4 *>(src + (size_t)r * ld + 8 * c);
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * ncm + c) * 128 + (r & 7) * 16) = v;
    }
}

// tcgen05.ld of 16 columns of this warp's lane quadrant; the registers are
// valid only after tmem_wait, which takes them as operands so that no use can
// be scheduled before it.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t addr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
                 " [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(addr));
}

__device__ __forceinline__ void tmem_wait(uint32_t *r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :: "memory");
}

// SiLU for the tensor-core epilogue, which is bound by this arithmetic:
// silu(z) = z sigmoid(z) = z/2 (1 + tanh(z/2)), one tanh.approx.f32 (a single
// special-function operation, relative error about 2^-11, below the BF16
// rounding that follows) instead of an exponential and a reciprocal.
__device__ __forceinline__ float silu_fast(float z)
{
    const float h = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// K steps [ks0, ks1) of one layer's products, issued by a single thread:
// D[128 x N] (+)= A[128 x K] B[N x K]^T, the first K step overwriting D.
__device__ __forceinline__ void mma_range(uint32_t tmem, uint32_t a, uint32_t b, int K, int N, int ks0, int ks1)
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = tc_idesc(TC_M, N), sbo = (uint32_t)(K >> 3) * 128u;
    for (int ks = ks0; ks < ks1; ++ks) {
        const uint64_t ad = tc_desc(a + ks * 256, 128, sbo), bd = tc_desc(b + ks * 256, 128, sbo);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

// Epilogue of a 256-column accumulator in four chunks of 64 columns: warp w
// reads 16 columns (64 q + 16 (w / 4) ..) of lane quadrant w % 4 (the load of
// chunk q + 1 in flight while chunk q is processed), adds the bias, applies
// SiLU, stores BF16 into K chunks 8 q + 2 (w / 4) and the next of the K = 256
// operand tile, and arrives on chunk q's mbarrier (16 arrivals complete it).
// After each chunk `issue(q)` runs on every thread of the warp (it acts on
// thread 0 only), then the warp reconverges.
__device__ __forceinline__ void silu_store16(const uint32_t *u, const float *bias, unsigned char *row, int c0)
{
    const float4 *b4 = reinterpret_cast<const float4 *>(bias + c0);
    uint32_t h[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 b = b4[j];
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(silu_fast(__uint_as_float(u[4 * j]) + b.x),
                                                        silu_fast(__uint_as_float(u[4 * j + 1]) + b.y));
        const __nv_bfloat162 p1 = __floats2bfloat162_rn(silu_fast(__uint_as_float(u[4 * j + 2]) + b.z),
                                                        silu_fast(__uint_as_float(u[4 * j + 3]) + b.w));
        h[2 * j] = *reinterpret_cast<const uint32_t *>(&p0);
        h[2 * j + 1] = *reinterpret_cast<const uint32_t *>(&p1);
    }
    *reinterpret_cast<uint4 *>(row + (c0 >> 3) * 128) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(row + ((c0 >> 3) + 1) * 128) = make_uint4(h[4], h[5], h[6], h[7]);
}

template <typename ISSUE>
__device__ __forceinline__ void epi_silu_streamed(uint32_t tmem, const float *bias, unsigned char *act,
                                                  uint32_t cbar, ISSUE issue)
{
    const int warp = threadIdx.x >> 5, qd = warp & 3, part = warp >> 2, lane = threadIdx.x & 31;
    const int r = 32 * qd + lane;
    const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(16 * part);
    unsigned char *row = act + (r & 7) * 16 + (r >> 3) * (NH / 8) * 128;
    uint32_t ua[16], ub[16];
    tmem_ld16_issue(tb, ua);
    tmem_wait(ua);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t *cur = (q & 1) ? ub : ua;
        uint32_t *nxt = (q & 1) ? ua : ub;
        if (q < 3) tmem_ld16_issue(tb + (uint32_t)(64 * (q + 1)), nxt);
        silu_store16(cur, bias, row, 64 * q + 16 * part);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(cbar + 8u * (uint32_t)q)
                         : "memory");
        issue(q);
        __syncwarp();
        if (q < 3) tmem_wait(nxt);
    }
}

// Writers' shared-memory stores become visible to the tensor cores' reads,
// and tensor-memory accesses before the barrier are ordered before those after.
__device__ __forceinline__ void tc_block_sync()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

constexpr int FW_THREADS = 512;

__global__ void __launch_bounds__(FW_THREADS, 1) k_mlp_fwd_tc(const __nv_bfloat16 *__restrict__ X0,
                                                       const __nv_bfloat16 *__restrict__ W1,
                                                       const __nv_bfloat16 *__restrict__ W2,
                                                       const __nv_bfloat16 *__restrict__ W3,
                                                       const float *__restrict__ b1, const float *__restrict__ b2,
                                                       const float *__restrict__ b3, float *__restrict__ Y,
                                                       int ntiles, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sW1 = sm, *sW2 = sm + FW_W1, *sW3 = sW2 + FW_W2, *sAct = sW3 + FW_W3;
    float *sb = reinterpret_cast<float *>(sAct + FW_ACT);   // b1[256], b2[256], b3[48]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + NH + NH + NOUT_P);   // [0] products, [1..4] chunks
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 5);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mb = smem_u32(mbar), cbar = mb + 8u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        for (int q = 0; q < 4; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(cbar + 8u * (uint32_t)q), "r"(FW_THREADS / 32)
                         : "memory");
    }
    stage_kmajor(sW1, W1, NH, NIN_P, NIN_P);
    stage_kmajor(sW2, W2, NH, NH, NH);
    stage_kmajor(sW3, W3, NOUT_P, NH, NH);
    for (int i = tid; i < NH + NH + NOUT_P; i += blockDim.x)
        sb[i] = i < NH ? b1[i] : (i < 2 * NH ? b2[i - NH] : b3[i - 2 * NH]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t aA = smem_u32(sAct), a1 = smem_u32(sW1), a2 = smem_u32(sW2), a3 = smem_u32(sW3);
    uint32_t parity = 0, eph = 0;   // phases of the products' and of the chunks' mbarriers
    bool ok = true;
    // the two accumulators, used in turn by the layers of consecutive tiles
    auto acc = [&](int g) { return tmem + (uint32_t)((g & 1) * NH); };
    // the 128 x 16 input block of a tile is 256 chunks of 16 bytes, one per
    // thread: chunk (row tid / 2, column half tid % 2); the next tile's chunk is
    // loaded into registers while the current tile runs its three layers
    constexpr int XCH = TC_M * (NIN_P / 8);   // 16-byte input chunks per tile
    static_assert(FW_THREADS >= XCH && FW_THREADS % 128 == 0, "input chunks and lane quadrants");
    const bool xin = tid < XCH;
    const int xr = (tid & (XCH - 1)) >> 1, xc = tid & 1;
    const int xoff = ((xr >> 3) * 2 + xc) * 128 + (xr & 7) * 16;
    // one decision for the whole CTA (barriers follow); on a timeout the
    // error is flagged and the products still in flight are waited for once more
    auto wait_all = [&]() {
        if (__syncthreads_or(tc_wait(mb, parity) ? 0 : 1)) {
            if (tid == 0) atomicOr(err, 1);
            tc_wait(mb, parity);
            return false;
        }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return true;
    };
    int g = 0;
    int tile = blockIdx.x;
    if (tile < ntiles) {
        if (xin) *reinterpret_cast<uint4 *>(sAct + xoff) =
            *reinterpret_cast<const uint4 *>(X0 + (size_t)(tile * TC_M + xr) * NIN_P + 8 * xc);
        tc_block_sync();
        if (tid == 0) {
            mma_range(acc(g), aA, a1, NIN_P, NH, 0, 1);
            mma_commit(mb);
        }
    }
    for (; tile < ntiles && ok; tile += gridDim.x) {
        const int m0 = tile * TC_M;
        const bool more = tile + (int)gridDim.x < ntiles;
        uint4 xnext = make_uint4(0u, 0u, 0u, 0u);
        if (xin && more)
            xnext = *reinterpret_cast<const uint4 *>(X0 + (size_t)((tile + gridDim.x) * TC_M + xr) * NIN_P + 8 * xc);
        // layer 1's epilogue, streaming layer 2's products
        if (!(ok = wait_all())) break;
        epi_silu_streamed(acc(g), sb, sAct, cbar, [&](int q) {
            if (tid == 0) {
                if (!tc_wait(cbar + 8u * (uint32_t)q, eph)) atomicOr(err, 2);
                mma_range(acc(g + 1), aA, a2, NH, NH, 4 * q, 4 * q + 4);
            }
        });
        eph ^= 1u;
        if (tid == 0) mma_commit(mb);
        // layer 2's epilogue, streaming layer 3's products (its reads of the
        // activation buffer are over once layer 2's products have completed)
        if (!(ok = wait_all())) break;
        epi_silu_streamed(acc(g + 1), sb + NH, sAct, cbar, [&](int q) {
            if (tid == 0) {
                if (!tc_wait(cbar + 8u * (uint32_t)q, eph)) atomicOr(err, 2);
                mma_range(acc(g + 2), aA, a3, NH, NOUT_P, 4 * q, 4 * q + 4);
            }
        });
        eph ^= 1u;
        if (tid == 0) mma_commit(mb);
        if (!(ok = wait_all())) break;
        // the next tile's first layer, then this tile's 48 output columns
        if (more) {
            if (xin) *reinterpret_cast<uint4 *>(sAct + xoff) = xnext;
            tc_block_sync();
            if (tid == 0) {
                mma_range(acc(g + 3), aA, a1, NIN_P, NH, 0, 1);
                mma_commit(mb);
            }
        }
        {
            const int qd = warp & 3, part = warp >> 2;
            const int row = m0 + 32 * qd + lane;
            const uint32_t tb = acc(g + 2) + ((uint32_t)(32 * qd) << 16);
            if (part < NOUT_P / 16) {
                const int c0 = 16 * part;
                uint32_t u[16];
                tmem_ld16_issue(tb + (uint32_t)c0, u);
                tmem_wait(u);
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(u[j]);
                float4 *dst = reinterpret_cast<float4 *>(Y + (size_t)row * NOUT_P + c0);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dst[j] = make_float4(v[4 * j] + sb[2 * NH + c0 + 4 * j], v[4 * j + 1] + sb[2 * NH + c0 + 4 * j + 1],
                                         v[4 * j + 2] + sb[2 * NH + c0 + 4 * j + 2],
                                         v[4 * j + 3] + sb[2 * NH + c0 + 4 * j + 3]);
            }
        }
        g += 3;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
}

// The training products on the tensor cores: the same C = A B^T and
// epilogues as k_gemm, one CTA (4 warps) per 128-row tile of C with all N <= 256
// columns in tensor memory.  K is taken in chunks of GT_KC: every thread
// stages its share of the A and B chunks (rows past M or N as zeros) in the
// K-major no-swizzle layout, one thread issues the chunk's tcgen05.mma
// instructions and commits to the mbarrier, and all wait for it (bounded)
// before the buffers are refilled.  The epilogue reads the accumulator back
// with tcgen05.ld, warp w holding rows 32w..32w+31, and applies the same
// per-element arithmetic as k_gemm (expf-based SiLU), so the two backends
// differ only in the order of the FP32 accumulation.
constexpr int GT_KC = 64, GT_THREADS = 128;

__device__ __forceinline__ void stage_chunk(unsigned char *dst, const __nv_bfloat16 *src, int r0, int rows, int nvalid,
                                            int k0, int K)
{
    constexpr int ncm = GT_KC / 8;
    for (int q = threadIdx.x; q < rows * ncm; q += blockDim.x) {
        const int r = q / ncm, c = q - r * ncm;
        const int gr = r0 + r, gk = k0 + 8 * c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < nvalid && gk < K) v = *reinterpret_cast<const uint4 *>(src + (size_t)gr * K + gk);
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * ncm + c) * 128 + (r & 7) * 16) = v;
    }
}

__global__ void __launch_bounds__(GT_THREADS, 1) k_gemm_tc(const __nv_bfloat16 *__restrict__ A,
                                                           const __nv_bfloat16 *__restrict__ B, int M, int N, int K,
                                                           int epi, const float *__restrict__ bias,
                                                           const float *__restrict__ gateZ, float *__restrict__ C32,
                                                           __nv_bfloat16 *__restrict__ C16,
                                                           __nv_bfloat16 *__restrict__ C16T, int tcols, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int Np = (N + 15) & ~15;
    unsigned char *sa = sm, *sb = sm + TC_M * GT_KC * 2;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sb + (size_t)Np * GT_KC * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M;
    const uint32_t mb = smem_u32(mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)),
                     "r"(tcols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc_idesc(TC_M, Np), sbo = (uint32_t)(GT_KC / 8) * 128u;
    uint32_t parity = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K && ok; k0 += GT_KC) {
        stage_chunk(sa, A, m0, TC_M, M, k0, K);
        stage_chunk(sb, B, 0, Np, N, k0, K);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int nks = min(GT_KC, K - k0) >> 4;
            for (int ks = 0; ks < nks; ++ks) {
                const uint64_t ad = tc_desc(smem_u32(sa) + ks * 256, 128, sbo);
                const uint64_t bd = tc_desc(smem_u32(sb) + ks * 256, 128, sbo);
                const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mb)
                         : "memory");
        }
        if (__syncthreads_or(tc_wait(mb, parity) ? 0 : 1)) {
            ok = false;
            if (tid == 0) atomicOr(err, 1);
            tc_wait(mb, parity);   // second bounded wait for MMAs still in flight
        }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok) {
        const int r = m0 + 32 * warp + lane;
        const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < Np; c0 += 16) {
            uint32_t u[16];
            tmem_ld16_issue(tb + (uint32_t)c0, u);
            tmem_wait(u);
            if (r >= M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + j;
                if (c >= N) break;
                float v = __uint_as_float(u[j]);
                const size_t o = (size_t)r * N + c;
                if (epi == EPI_F32) {
                    C32[o] = v;
                } else if (epi == EPI_BIAS) {
                    C32[o] = v + bias[c];
                } else if (epi == EPI_BIAS_SILU) {
                    v += bias[c];
                    C32[o] = v;
                    const __nv_bfloat16 h = __float2bfloat16_rn(silu(v));
                    C16[o] = h;
                    C16T[(size_t)c * M + r] = h;
                } else {   // EPI_GATE
                    const __nv_bfloat16 h = __float2bfloat16_rn(v * dsilu(gateZ[o]));
                    C16[o] = h;
                    C16T[(size_t)c * M + r] = h;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(tcols) : "memory");
}

struct Member {
    float *w[3], *b[3];                 // FP32 masters
    float *mw[3], *vw[3], *mb[3], *vb[3];
    float *gw[3], *gb[3];
    __nv_bfloat16 *wbf[3], *wbfT[3];
};

}  // namespace sur

using namespace sur;

struct sur_ctx {
    int K = 0, cap = 0;   // members, batch capacity (rows, multiple of 64)
    cudaStream_t st = nullptr;
    bool own_stream = false;
    void *pool = nullptr;
    std::vector<Member> mem;
    float *mu_x, *sd_x, *mu_y, *sd_y;   // standardisation (device)
    float h_mu_y[NOUT], h_sd_y[NOUT];
    // activations, sized for cap rows
    __nv_bfloat16 *X0, *X0T, *A1, *A1T, *A2, *A2T, *dY, *dYT, *dZ1, *dZ1T, *dZ2, *dZ2T;
    float *Z1, *Z2, *Y, *dA, *dY32, *T, *Xin, *loss, *Yall, *Yout, *Sout;
    int64_t adam_t = 0;
    float *h_loss = nullptr;
    int *d_err = nullptr;   // bounded-wait timeouts of the tensor-core GEMM
    int tc = 1;             // forward passes of >= 128 rows on tcgen05 (0: mma.sync)
};

static const int DIMS_IN[3] = {NIN_P, NH, NH};
static const int DIMS_OUT[3] = {NH, NH, NOUT_P};

#define CUS(x)                                                                      \
    do {                                                                            \
        const cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

static size_t gemm_tc_smem(int N) { return (size_t)TC_M * GT_KC * 2 + (size_t)((N + 15) & ~15) * GT_KC * 2 + 16; }

// C = A B^T on the backend in use: tcgen05 (the default) or warp-level mma.sync.
static void gemm(sur_ctx *s, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int epi,
                 const float *bias, const float *gate, float *C32, __nv_bfloat16 *C16, __nv_bfloat16 *C16T)
{
    if (s->tc) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem(NH));
            attr = true;
        }
        const int Np = (N + 15) & ~15;
        const int tcols = Np <= 32 ? 32 : (Np <= 64 ? 64 : (Np <= 128 ? 128 : 256));
        k_gemm_tc<<<(M + TC_M - 1) / TC_M, GT_THREADS, gemm_tc_smem(N), s->st>>>(A, B, M, N, K, epi, bias, gate, C32,
                                                                                 C16, C16T, tcols, s->d_err);
        return;
    }
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<<<grid, 128, 0, s->st>>>(A, B, M, N, K, epi, bias, gate, C32, C16, C16T);
}

// Forward pass of member k on the first M rows of X0 (standardised inputs
// already in s->X0 / X0T); output Y [M][48] FP32 (standardised).
static void forward(sur_ctx *s, int k, int M, float *Yout)
{
    Member &m = s->mem[k];
    gemm(s, s->X0, m.wbf[0], M, NH, NIN_P, EPI_BIAS_SILU, m.b[0], nullptr, s->Z1, s->A1, s->A1T);
    gemm(s, s->A1, m.wbf[1], M, NH, NH, EPI_BIAS_SILU, m.b[1], nullptr, s->Z2, s->A2, s->A2T);
    gemm(s, s->A2, m.wbf[2], M, NOUT_P, NH, EPI_BIAS, m.b[2], nullptr, Yout, nullptr, nullptr);
}

// Forward pass of member k on the tensor cores (M a multiple of 128): the
// fused persistent kernel, one CTA per SM at most.
static void forward_fused(sur_ctx *s, int k, int M, float *Yout)
{
    static bool attr = false;
    static int nsm = 0;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        attr = true;
    }
    Member &m = s->mem[k];
    const int ntiles = M / TC_M;
    const int grid = std::min(ntiles, std::max(nsm, 1));
    k_mlp_fwd_tc<<<grid, FW_THREADS, FW_SMEM, s->st>>>(s->X0, m.wbf[0], m.wbf[1], m.wbf[2], m.b[0], m.b[1], m.b[2], Yout,
                                                ntiles, s->d_err);
}

// Loss and gradients of member k for n valid rows (M padded rows).
static void backward(sur_ctx *s, int k, int n, int M)
{
    Member &m = s->mem[k];
    k_loss<<<(M * NOUT_P + 255) / 256, 256, 0, s->st>>>(s->Y, s->T, n, M, s->loss, s->dY, s->dYT, s->dY32);
    // layer 3: dW3 = dY^T A2, db3 = colsum dY, dA2 = dY W3
    gemm(s, s->dYT, s->A2T, NOUT_P, NH, M, EPI_F32, nullptr, nullptr, m.gw[2], nullptr, nullptr);
    k_colsum<<<NOUT_P, 256, 0, s->st>>>(s->dY32, nullptr, M, NOUT_P, m.gb[2]);
    gemm(s, s->dY, m.wbfT[2], M, NH, NOUT_P, EPI_GATE, nullptr, s->Z2, nullptr, s->dZ2, s->dZ2T);
    // layer 2
    gemm(s, s->dZ2T, s->A1T, NH, NH, M, EPI_F32, nullptr, nullptr, m.gw[1], nullptr, nullptr);
    k_colsum<<<NH, 256, 0, s->st>>>(nullptr, s->dZ2, M, NH, m.gb[1]);
    gemm(s, s->dZ2, m.wbfT[1], M, NH, NH, EPI_GATE, nullptr, s->Z1, nullptr, s->dZ1, s->dZ1T);
    // layer 1 (no input gradient)
    gemm(s, s->dZ1T, s->X0T, NH, NIN_P, M, EPI_F32, nullptr, nullptr, m.gw[0], nullptr, nullptr);
    k_colsum<<<NH, 256, 0, s->st>>>(nullptr, s->dZ1, M, NH, m.gb[0]);
}

static void adam(sur_ctx *s, int k, float lr)
{
    Member &m = s->mem[k];
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - (float)std::pow(0.9, (double)s->adam_t), c2 = 1.f - (float)std::pow(0.999, (double)s->adam_t);
    for (int l = 0; l < 3; ++l) {
        const int nw = DIMS_OUT[l] * DIMS_IN[l];
        k_adam<<<(nw + 255) / 256, 256, 0, s->st>>>(m.w[l], m.mw[l], m.vw[l], m.gw[l], nw, DIMS_IN[l], lr, b1, b2,
                                                    eps, c1, c2, m.wbf[l], m.wbfT[l], DIMS_OUT[l]);
        k_adam<<<(DIMS_OUT[l] + 255) / 256, 256, 0, s->st>>>(m.b[l], m.mb[l], m.vb[l], m.gb[l], DIMS_OUT[l], 1, lr,
                                                             b1, b2, eps, c1, c2, nullptr, nullptr, 1);
    }
}

static int upload_inputs(sur_ctx *s, const float *X, int n, int M)
{
    CUS(cudaMemcpyAsync(s->Xin, X, sizeof(float) * NIN * (size_t)n, cudaMemcpyHostToDevice, s->st));
    k_inputs<<<(M + 127) / 128, 128, 0, s->st>>>(s->Xin, n, M, s->mu_x, s->sd_x, s->X0, s->X0T);
    return DPD_OK;
}

// Xavier-style uniform initialisation from a splitmix64 stream (host).
static uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int set_weights_host(sur_ctx *s, int k, const float *const W[3], const float *const b[3])
{
    Member &m = s->mem[k];
    for (int l = 0; l < 3; ++l) {
        const int ni = DIMS_IN[l], no = DIMS_OUT[l];
        std::vector<float> w((size_t)no * ni);
        std::memcpy(w.data(), W[l], sizeof(float) * w.size());
        std::vector<__nv_bfloat16> wb(w.size()), wt(w.size());
        for (int r = 0; r < no; ++r)
            for (int c = 0; c < ni; ++c) {
                wb[(size_t)r * ni + c] = __float2bfloat16_rn(w[(size_t)r * ni + c]);
                wt[(size_t)c * no + r] = wb[(size_t)r * ni + c];
            }
        CUS(cudaMemcpyAsync(m.w[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, s->st));
        CUS(cudaMemcpyAsync(m.wbf[l], wb.data(), 2 * wb.size(), cudaMemcpyHostToDevice, s->st));
        CUS(cudaMemcpyAsync(m.wbfT[l], wt.data(), 2 * wt.size(), cudaMemcpyHostToDevice, s->st));
        CUS(cudaMemcpyAsync(m.b[l], b[l], sizeof(float) * no, cudaMemcpyHostToDevice, s->st));
    }
    CUS(cudaStreamSynchronize(s->st));
    return DPD_OK;
}

extern "C" {

int sur_create(int n_members, int max_rows, uint64_t seed, void *stream, sur_ctx **out)
{
    if (!out || n_members < 1 || n_members > 64 || max_rows < 1 || max_rows > (1 << 20)) return DPD_ERR_INVALID_ARG;
    *out = nullptr;
    sur_ctx *s = new (std::nothrow) sur_ctx();
    if (!s) return DPD_ERR_OOM;
    s->K = n_members;
    s->cap = (max_rows + 127) & ~127;
    if (stream) s->st = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return DPD_ERR_CUDA; }
        s->own_stream = true;
    }
    const size_t M = (size_t)s->cap;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off += (b + 255) & ~size_t(255); return o; };
    std::vector<size_t> offs;
    // per member: for each layer: w, mw, vw, gw (f32), wbf, wbfT (bf16), b, mb, vb, gb
    struct LO { size_t w, mw, vw, gw, wbf, wbfT, b, mb, vb, gb; };
    std::vector<LO> lo((size_t)s->K * 3);
    for (int k = 0; k < s->K; ++k)
        for (int l = 0; l < 3; ++l) {
            const size_t nw = (size_t)DIMS_OUT[l] * DIMS_IN[l], nb = DIMS_OUT[l];
            LO &o = lo[(size_t)k * 3 + l];
            o.w = take(4 * nw); o.mw = take(4 * nw); o.vw = take(4 * nw); o.gw = take(4 * nw);
            o.wbf = take(2 * nw); o.wbfT = take(2 * nw);
            o.b = take(4 * nb); o.mb = take(4 * nb); o.vb = take(4 * nb); o.gb = take(4 * nb);
        }
    const size_t o_mu = take(4 * 256), o_X0 = take(2 * M * NIN_P), o_X0T = take(2 * M * NIN_P),
                 o_A1 = take(2 * M * NH), o_A1T = take(2 * M * NH), o_A2 = take(2 * M * NH), o_A2T = take(2 * M * NH),
                 o_dY = take(2 * M * NOUT_P), o_dYT = take(2 * M * NOUT_P), o_dZ1 = take(2 * M * NH),
                 o_dZ1T = take(2 * M * NH), o_dZ2 = take(2 * M * NH), o_dZ2T = take(2 * M * NH),
                 o_Z1 = take(4 * M * NH), o_Z2 = take(4 * M * NH), o_Y = take(4 * M * NOUT_P),
                 o_dA = take(4 * M * NH), o_dY32 = take(4 * M * NOUT_P), o_T = take(4 * M * NOUT),
                 o_Xin = take(4 * M * NIN), o_loss = take(64), o_Yall = take(4 * M * NOUT_P * (size_t)s->K),
                 o_Yout = take(4 * M * NOUT), o_Sout = take(4 * M * NOUT), o_err = take(4);
    if (cudaMalloc(&s->pool, off) != cudaSuccess || cudaMallocHost((void **)&s->h_loss, 64) != cudaSuccess) {
        sur_destroy(s);
        return DPD_ERR_OOM;
    }
    cudaMemsetAsync(s->pool, 0, off, s->st);
    char *p = (char *)s->pool;
    s->mem.resize(s->K);
    for (int k = 0; k < s->K; ++k)
        for (int l = 0; l < 3; ++l) {
            const LO &o = lo[(size_t)k * 3 + l];
            Member &m = s->mem[k];
            m.w[l] = (float *)(p + o.w); m.mw[l] = (float *)(p + o.mw); m.vw[l] = (float *)(p + o.vw);
            m.gw[l] = (float *)(p + o.gw); m.wbf[l] = (__nv_bfloat16 *)(p + o.wbf);
            m.wbfT[l] = (__nv_bfloat16 *)(p + o.wbfT); m.b[l] = (float *)(p + o.b); m.mb[l] = (float *)(p + o.mb);
            m.vb[l] = (float *)(p + o.vb); m.gb[l] = (float *)(p + o.gb);
        }
    s->mu_x = (float *)(p + o_mu); s->sd_x = s->mu_x + 64; s->mu_y = s->mu_x + 128; s->sd_y = s->mu_x + 192;
    s->X0 = (__nv_bfloat16 *)(p + o_X0); s->X0T = (__nv_bfloat16 *)(p + o_X0T);
    s->A1 = (__nv_bfloat16 *)(p + o_A1); s->A1T = (__nv_bfloat16 *)(p + o_A1T);
    s->A2 = (__nv_bfloat16 *)(p + o_A2); s->A2T = (__nv_bfloat16 *)(p + o_A2T);
    s->dY = (__nv_bfloat16 *)(p + o_dY); s->dYT = (__nv_bfloat16 *)(p + o_dYT);
    s->dZ1 = (__nv_bfloat16 *)(p + o_dZ1); s->dZ1T = (__nv_bfloat16 *)(p + o_dZ1T);
    s->dZ2 = (__nv_bfloat16 *)(p + o_dZ2); s->dZ2T = (__nv_bfloat16 *)(p + o_dZ2T);
    s->Z1 = (float *)(p + o_Z1); s->Z2 = (float *)(p + o_Z2); s->Y = (float *)(p + o_Y); s->dA = (float *)(p + o_dA);
    s->dY32 = (float *)(p + o_dY32); s->T = (float *)(p + o_T); s->Xin = (float *)(p + o_Xin);
    s->loss = (float *)(p + o_loss); s->Yall = (float *)(p + o_Yall); s->Yout = (float *)(p + o_Yout);
    s->Sout = (float *)(p + o_Sout);
    s->d_err = (int *)(p + o_err);
    // identity standardisation until training sets it
    std::vector<float> ones(256, 1.f);
    cudaMemcpyAsync(s->sd_x, ones.data(), 4 * 64, cudaMemcpyHostToDevice, s->st);
    cudaMemcpyAsync(s->sd_y, ones.data(), 4 * 64, cudaMemcpyHostToDevice, s->st);
    for (int c = 0; c < NOUT; ++c) { s->h_mu_y[c] = 0.f; s->h_sd_y[c] = 1.f; }
    // initial weights: uniform(-a, a), a = sqrt(6 / (fan_in + fan_out)); biases 0
    uint64_t st = seed;
    for (int k = 0; k < s->K; ++k) {
        std::vector<float> W[3], B[3];
        for (int l = 0; l < 3; ++l) {
            const int ni = DIMS_IN[l], no = DIMS_OUT[l];
            const int fi = l == 0 ? NIN : ni, fo = l == 2 ? NOUT : no;
            const float a = std::sqrt(6.0f / (float)(fi + fo));
            W[l].assign((size_t)no * ni, 0.f);
            B[l].assign(no, 0.f);
            for (int r = 0; r < (l == 2 ? NOUT : no); ++r)
                for (int c = 0; c < (l == 0 ? NIN : ni); ++c)
                    W[l][(size_t)r * ni + c] = a * (2.0f * (float)((splitmix(st) >> 40) * (1.0 / 16777216.0)) - 1.0f);
        }
        const float *wp[3] = {W[0].data(), W[1].data(), W[2].data()}, *bp[3] = {B[0].data(), B[1].data(), B[2].data()};
        const int rc = set_weights_host(s, k, wp, bp);
        if (rc) { sur_destroy(s); return rc; }
    }
    *out = s;
    return DPD_OK;
}

void sur_destroy(sur_ctx *s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->pool) cudaFree(s->pool);
    if (s->h_loss) cudaFreeHost(s->h_loss);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
}

int sur_set_weights(sur_ctx *s, int member, const float *W1, const float *b1, const float *W2, const float *b2,
                    const float *W3, const float *b3)
{
    if (!s || member < 0 || member >= s->K || !W1 || !W2 || !W3 || !b1 || !b2 || !b3) return DPD_ERR_INVALID_ARG;
    const float *wp[3] = {W1, W2, W3}, *bp[3] = {b1, b2, b3};
    return set_weights_host(s, member, wp, bp);
}

int sur_set_scaling(sur_ctx *s, const float mu_x[4], const float sd_x[4], const float mu_y[40], const float sd_y[40])
{
    if (!s || !mu_x || !sd_x || !mu_y || !sd_y) return DPD_ERR_INVALID_ARG;
    for (int c = 0; c < NIN; ++c)
        if (!(sd_x[c] > 0)) return DPD_ERR_INVALID_ARG;
    for (int c = 0; c < NOUT; ++c)
        if (!(sd_y[c] > 0)) return DPD_ERR_INVALID_ARG;
    CUS(cudaMemcpyAsync(s->mu_x, mu_x, 16, cudaMemcpyHostToDevice, s->st));
    CUS(cudaMemcpyAsync(s->sd_x, sd_x, 16, cudaMemcpyHostToDevice, s->st));
    CUS(cudaMemcpyAsync(s->mu_y, mu_y, 160, cudaMemcpyHostToDevice, s->st));
    CUS(cudaMemcpyAsync(s->sd_y, sd_y, 160, cudaMemcpyHostToDevice, s->st));
    std::memcpy(s->h_mu_y, mu_y, 160);
    std::memcpy(s->h_sd_y, sd_y, 160);
    CUS(cudaStreamSynchronize(s->st));
    return DPD_OK;
}

int sur_gradients(sur_ctx *s, int member, const float *X, const float *Y, int n, float *loss, float *gW1, float *gb1,
                  float *gW2, float *gb2, float *gW3, float *gb3)
{
    if (!s || member < 0 || member >= s->K || !X || !Y || n < 1 || n > s->cap) return DPD_ERR_INVALID_ARG;
    const int M = (n + 63) & ~63;
    int rc = upload_inputs(s, X, n, M);
    if (rc) return rc;
    // standardised targets
    std::vector<float> t((size_t)n * NOUT);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < NOUT; ++c) t[(size_t)r * NOUT + c] = (Y[(size_t)r * NOUT + c] - s->h_mu_y[c]) / s->h_sd_y[c];
    CUS(cudaMemcpyAsync(s->T, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, s->st));
    CUS(cudaMemsetAsync(s->loss, 0, 4, s->st));
    forward(s, member, M, s->Y);
    backward(s, member, n, M);
    CUS(cudaGetLastError());
    Member &m = s->mem[member];
    float *dst[6] = {gW1, gb1, gW2, gb2, gW3, gb3};
    const float *src[6] = {m.gw[0], m.gb[0], m.gw[1], m.gb[1], m.gw[2], m.gb[2]};
    const size_t cnt[6] = {(size_t)NH * NIN_P, NH, (size_t)NH * NH, NH, (size_t)NOUT_P * NH, NOUT_P};
    for (int i = 0; i < 6; ++i)
        if (dst[i]) CUS(cudaMemcpyAsync(dst[i], src[i], 4 * cnt[i], cudaMemcpyDeviceToHost, s->st));
    CUS(cudaMemcpyAsync(s->h_loss, s->loss, 4, cudaMemcpyDeviceToHost, s->st));
    CUS(cudaStreamSynchronize(s->st));
    if (loss) *loss = s->h_loss[0] / (float)(n * NOUT);
    return DPD_OK;
}

int sur_train(sur_ctx *s, const float *X, const float *Y, int n, int epochs, int batch, float lr, float *final_loss)
{
    if (!s || !X || !Y || n < 2 || epochs < 0 || batch < 1 || !(lr > 0) || n > s->cap) return DPD_ERR_INVALID_ARG;
    // standardisation from the training set
    float mx[NIN], sx[NIN], my[NOUT], sy[NOUT];
    for (int c = 0; c < NIN; ++c) {
        double a = 0, b = 0;
        for (int r = 0; r < n; ++r) {
            double x = X[(size_t)r * NIN + c];
            if (c == 1 || c == 2) x = std::log(std::fmax(x, 1e-30));
            a += x;
            b += x * x;
        }
        a /= n;
        mx[c] = (float)a;
        sx[c] = (float)std::sqrt(std::fmax(b / n - a * a, 1e-12));
    }
    for (int c = 0; c < NOUT; ++c) {
        double a = 0, b = 0;
        for (int r = 0; r < n; ++r) { a += Y[(size_t)r * NOUT + c]; b += (double)Y[(size_t)r * NOUT + c] * Y[(size_t)r * NOUT + c]; }
        a /= n;
        my[c] = (float)a;
        sy[c] = (float)std::sqrt(std::fmax(b / n - a * a, 1e-12));
    }
    int rc = sur_set_scaling(s, mx, sx, my, sy);
    if (rc) return rc;
    batch = std::min(batch, n);
    const int Mb = (batch + 63) & ~63;
    // pre-standardise all targets once; minibatches are contiguous row ranges
    // of a per-epoch permutation gathered on the host
    std::vector<float> Ts((size_t)n * NOUT);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < NOUT; ++c) Ts[(size_t)r * NOUT + c] = (Y[(size_t)r * NOUT + c] - my[c]) / sy[c];
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::vector<float> xb((size_t)batch * NIN), tb((size_t)batch * NOUT);
    uint64_t st = 0x5EEDull + (uint64_t)n;
    double last = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(st) % (uint64_t)(i + 1)]);
        double esum = 0;
        int ecnt = 0;
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            for (int q = 0; q < batch; ++q) {
                std::memcpy(&xb[(size_t)q * NIN], &X[(size_t)perm[b0 + q] * NIN], 4 * NIN);
                std::memcpy(&tb[(size_t)q * NOUT], &Ts[(size_t)perm[b0 + q] * NOUT], 4 * NOUT);
            }
            if ((rc = upload_inputs(s, xb.data(), batch, Mb))) return rc;
            CUS(cudaMemcpyAsync(s->T, tb.data(), 4 * tb.size(), cudaMemcpyHostToDevice, s->st));
            ++s->adam_t;
            CUS(cudaMemsetAsync(s->loss, 0, 4, s->st));
            for (int k = 0; k < s->K; ++k) {
                forward(s, k, Mb, s->Y);
                backward(s, k, batch, Mb);
                adam(s, k, lr);
            }
            CUS(cudaGetLastError());
            if (e == epochs - 1) {
                CUS(cudaMemcpyAsync(s->h_loss, s->loss, 4, cudaMemcpyDeviceToHost, s->st));
                CUS(cudaStreamSynchronize(s->st));
                esum += s->h_loss[0] / (double)(batch * NOUT * s->K);
                ++ecnt;
            } else {
                CUS(cudaStreamSynchronize(s->st));   // host buffers are reused next batch
            }
        }
        if (ecnt) last = esum / ecnt;
    }
    if (final_loss) *final_loss = (float)last;
    return DPD_OK;
}

int sur_bench_forward(sur_ctx *s, int n, int reps, double *ms_per_pass)
{
    if (!s || !ms_per_pass || n < 1 || n > s->cap || reps < 1) return DPD_ERR_INVALID_ARG;
    const bool tc = s->tc && n >= TC_M;
    const int M = tc ? (n + TC_M - 1) / TC_M * TC_M : (n + 63) & ~63;
    cudaEvent_t e0, e1;
    CUS(cudaEventCreate(&e0));
    CUS(cudaEventCreate(&e1));
    if (tc) CUS(cudaMemsetAsync(s->d_err, 0, 4, s->st));
    CUS(cudaEventRecord(e0, s->st));
    for (int r = 0; r < reps; ++r)
        for (int k = 0; k < s->K; ++k) {
            if (tc) forward_fused(s, k, M, s->Yall + (size_t)k * M * NOUT_P);
            else forward(s, k, M, s->Yall + (size_t)k * M * NOUT_P);
        }
    CUS(cudaEventRecord(e1, s->st));
    CUS(cudaGetLastError());
    CUS(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_pass = ms / reps;
    return DPD_OK;
}

int sur_set_backend(sur_ctx *s, int use_tcgen05)
{
    if (!s || (use_tcgen05 != 0 && use_tcgen05 != 1)) return DPD_ERR_INVALID_ARG;
    s->tc = use_tcgen05;
    return DPD_OK;
}

int sur_predict(sur_ctx *s, const float *X, int n, float *Y, float *spread)
{
    if (!s || !X || !Y || n < 1 || n > s->cap) return DPD_ERR_INVALID_ARG;
    const bool tc = s->tc && n >= TC_M;
    const int M = tc ? (n + TC_M - 1) / TC_M * TC_M : (n + 63) & ~63;
    int rc = upload_inputs(s, X, n, M);
    if (rc) return rc;
    if (tc) CUS(cudaMemsetAsync(s->d_err, 0, 4, s->st));
    for (int k = 0; k < s->K; ++k) {
        if (tc) forward_fused(s, k, M, s->Yall + (size_t)k * M * NOUT_P);
        else forward(s, k, M, s->Yall + (size_t)k * M * NOUT_P);
    }
    k_predict_out<<<(n * NOUT + 255) / 256, 256, 0, s->st>>>(s->Yall, s->K, n, M, s->mu_y, s->sd_y, s->Yout,
                                                            spread ? s->Sout : nullptr);
    CUS(cudaGetLastError());
    CUS(cudaMemcpyAsync(Y, s->Yout, 4 * (size_t)n * NOUT, cudaMemcpyDeviceToHost, s->st));
    if (spread) CUS(cudaMemcpyAsync(spread, s->Sout, 4 * (size_t)n * NOUT, cudaMemcpyDeviceToHost, s->st));
    if (tc) CUS(cudaMemcpyAsync(s->h_loss + 8, s->d_err, 4, cudaMemcpyDeviceToHost, s->st));
    CUS(cudaStreamSynchronize(s->st));
    if (tc && *reinterpret_cast<int *>(s->h_loss + 8)) return DPD_ERR_TIMEOUT;
    return DPD_OK;
}


static double ls_slope(const double *lnk, const double *y, int n)
{
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int i = 0; i < n; ++i) {
        sx += lnk[i];
        sy += y[i];
        sxx += lnk[i] * lnk[i];
        sxy += lnk[i] * y[i];
    }
    return (n * sxy - sx * sy) / (n * sxx - sx * sx);
}

int sur_targets(int n_snap, int n_shells, int nbins, double dr, const double *E, const double *g, const double *T,
                const double *vcom, double out[40])
{
    if (n_snap < 1 || n_shells < 64 || nbins < 1 || !(dr > 0) || !E || !g || !T || !vcom || !out)
        return DPD_ERR_INVALID_ARG;
    std::vector<double> Em(n_shells, 0.0), gm(nbins, 0.0);
    for (int k = 0; k < n_shells; ++k) {
        for (int s = 0; s < n_snap; ++s) Em[k] += E[(size_t)s * n_shells + k];
        Em[k] /= n_snap;
    }
    for (int b = 0; b < nbins; ++b) {
        double sum = 0;
        int c = 0;
        for (int s = 0; s < n_snap; ++s) {
            const double v = g[(size_t)s * nbins + b];
            if (!std::isnan(v)) { sum += v; ++c; }
        }
        gm[b] = c ? sum / c : 0.0;
    }
    for (int b = 0; b < 32; ++b) out[b] = std::log(std::max(0.5 * (Em[2 * b] + Em[2 * b + 1]), 1e-300));
    // g over r = 0 (g = 1) and the bin centres
    const double ie = std::exp(-1.0);
    double xi = (nbins - 0.5) * dr, area = 0.0;
    bool found = false;
    double r_prev = 0.0, g_prev = 1.0;
    for (int b = 0; b < nbins; ++b) {
        const double r = (b + 0.5) * dr, gv = gm[b];
        area += 0.5 * (gv + g_prev) * (r - r_prev);
        if (!found && gv <= ie) {
            const double f = (g_prev - ie) / std::max(g_prev - gv, 1e-300);
            xi = r_prev + f * (r - r_prev);
            found = true;
        }
        r_prev = r;
        g_prev = gv;
    }
    out[32] = xi;
    out[33] = area;
    double t = 0, vc = 0;
    for (int s = 0; s < n_snap; ++s) { t += T[s]; vc += vcom[s]; }
    out[34] = t / n_snap;
    double lnk[64], y[64];
    for (int i = 0; i < 10; ++i) { lnk[i] = std::log((double)(i + 1)); y[i] = std::log(Em[i] / Em[0]); }
    out[35] = ls_slope(lnk, y, 10);
    for (int i = 0; i < 31; ++i) { lnk[i] = std::log((double)(30 + i)); y[i] = std::log(Em[29 + i] / Em[0]); }
    out[36] = ls_slope(lnk, y, 31);
    int kmax = 0;
    for (int k = 1; k < n_shells; ++k)
        if (Em[k] > Em[kmax]) kmax = k;
    out[37] = kmax + 1;
    out[38] = std::log(std::max(Em[0], 1e-300));
    out[39] = vc / n_snap;
    return DPD_OK;
}

// One fallback run of the protocol for the row (phi, gamma, zeta, f_p).
static int sur_simulate_row(void *stream, const float *x, const sur_protocol *pr, uint64_t seed, uint32_t replica,
                            double out[40])
{
    dpd_params p;
    std::memset(&p, 0, sizeof p);
    const long long nd = std::max(1LL, std::llround(2.0 * (double)x[0] * pr->L * pr->L));
    p.L = pr->L;
    p.n_beads = 2 * nd;
    p.a = 25.0;
    p.gamma = x[1];
    p.kBT = 1.0;
    p.rc = 1.0;
    p.k_bond = 100.0;
    p.r0 = 0.5;
    p.f_p = x[3];
    p.zeta = x[2];
    p.dt = 0.01;
    p.mass = 1.0;
    p.seed = seed;
    p.replica = replica;
    p.exclude_bonded = 1;
    dpd_ctx *c = nullptr;
    int rc = dpd_create(&p, stream, &c);
    if (rc) return rc;
    const int nsh = pr->M / 2, nbins = (int)(pr->L / 2 / pr->dr);
    std::vector<double> E((size_t)pr->n_snap * nsh), g((size_t)pr->n_snap * std::max(nbins, 1)), T(pr->n_snap),
        vc(pr->n_snap);
    rc = dpd_init_random(c, seed);
    if (!rc) rc = dpd_step(c, pr->burn);
    for (int s = 0; s < pr->n_snap && !rc; ++s) {
        rc = dpd_step(c, pr->every);
        if (!rc) rc = dpd_energy_spectrum(c, pr->M, 0.0, &E[(size_t)s * nsh]);
        if (!rc) rc = dpd_velocity_correlation(c, pr->dr, nbins, &g[(size_t)s * nbins], nullptr, nullptr, nullptr);
        if (!rc) rc = dpd_temperature(c, &T[s]);
        if (!rc) rc = dpd_agent_speed(c, &vc[s]);
    }
    dpd_destroy(c);
    if (!rc) rc = sur_targets(pr->n_snap, nsh, nbins, pr->dr, E.data(), g.data(), T.data(), vc.data(), out);
    return rc;
}

int sur_query(sur_ctx *s, const float *X, int n, float threshold, const sur_protocol *proto, float *Y,
              float *spread, int32_t *used_fallback)
{
    if (!s || !X || !Y || !used_fallback || !proto || n < 1 || n > s->cap) return DPD_ERR_INVALID_ARG;
    if (!(proto->L >= 3.0) || !(proto->dr > 0) || proto->burn < 0 || proto->n_snap < 1 || proto->every < 0 ||
        proto->M < 128 || (proto->M & 1) || (int)(proto->L / 2 / proto->dr) < 1)
        return DPD_ERR_INVALID_ARG;
    std::vector<float> S((size_t)n * NOUT);
    int rc = sur_predict(s, X, n, Y, S.data());
    if (rc) return rc;
    for (int i = 0; i < n && !rc; ++i) {
        float rel = 0.f;
        for (int t = 0; t < NOUT; ++t)
            rel = std::max(rel, S[(size_t)i * NOUT + t] / (std::fabs(Y[(size_t)i * NOUT + t]) + 1.0f));
        used_fallback[i] = rel > threshold ? 1 : 0;
        if (used_fallback[i]) {
            double out[NOUT];
            rc = sur_simulate_row(s->st, X + 4 * (size_t)i, proto, proto->seed + (uint64_t)i, (uint32_t)i, out);
            for (int t = 0; t < NOUT && !rc; ++t) Y[(size_t)i * NOUT + t] = (float)out[t];
        }
    }
    if (spread) std::memcpy(spread, S.data(), sizeof(float) * (size_t)n * NOUT);
    return rc;
}

}  // extern "C"
