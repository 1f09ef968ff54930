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
};

static const int DIMS_IN[3] = {NIN_P, NH, NH};
static const int DIMS_OUT[3] = {NH, NH, NOUT_P};

#define CUS(x)                                                                      \
    do {                                                                            \
        const cudaError_t e_ = (x);                                                 \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? DPD_ERR_OOM : DPD_ERR_CUDA; \
    } while (0)

static void gemm(sur_ctx *s, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int epi,
                 const float *bias, const float *gate, float *C32, __nv_bfloat16 *C16, __nv_bfloat16 *C16T)
{
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
    s->cap = (max_rows + 63) & ~63;
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
                 o_Yout = take(4 * M * NOUT), o_Sout = take(4 * M * NOUT);
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

int sur_predict(sur_ctx *s, const float *X, int n, float *Y, float *spread)
{
    if (!s || !X || !Y || n < 1 || n > s->cap) return DPD_ERR_INVALID_ARG;
    const int M = (n + 63) & ~63;
    int rc = upload_inputs(s, X, n, M);
    if (rc) return rc;
    for (int k = 0; k < s->K; ++k) forward(s, k, M, s->Yall + (size_t)k * M * NOUT_P);
    k_predict_out<<<(n * NOUT + 255) / 256, 256, 0, s->st>>>(s->Yall, s->K, n, M, s->mu_y, s->sd_y, s->Yout,
                                                            spread ? s->Sout : nullptr);
    CUS(cudaGetLastError());
    CUS(cudaMemcpyAsync(Y, s->Yout, 4 * (size_t)n * NOUT, cudaMemcpyDeviceToHost, s->st));
    if (spread) CUS(cudaMemcpyAsync(spread, s->Sout, 4 * (size_t)n * NOUT, cudaMemcpyDeviceToHost, s->st));
    CUS(cudaStreamSynchronize(s->st));
    return DPD_OK;
}

}  // extern "C"
