// Learned interpolation: the 112-128-128-16 ReLU MLP that predicts a fine point's row of
// P from its features, trained on the least-squares rows of Algorithm 2 (Eq. (3.6)).
// The paper has no learned interpolation; the definitions (features, bfloat16-rounded
// product inputs with FP32 sums, masked MSE, Adam of Kingma & Ba with beta1 = 0.9,
// beta2 = 0.999, eps = 1e-8, He-uniform initialisation from SplitMix64) are those of the
// interface declared in include/bamg.h.
//
// Forward products run on the tensor cores (mma.sync m16n8k16, bf16 in, FP32 accumulate):
// one warp computes 16 rows x N outputs, the weights staged once per block in shared
// memory with a padded row stride.  The training backward's products (input gradients
// through the ReLU masks, weight gradients summed over the batch) use the same instruction
// with the incoming gradient rounded to bf16; bias gradients and Adam stay in FP32.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "kernels.cuh"

namespace bamg {

// ------------------------------------------------------------------ parameter layout
// One flat FP32 buffer [W1 | b1 | W2 | b2 | W3 | b3]; W_l is out x in, row-major.  The
// bfloat16 copies of W1, W2, W3 sit in one flat buffer in the same order.
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + (int64_t)MLP_H * MLP_F;
constexpr int64_t OFF_W2 = OFF_B1 + MLP_H;
constexpr int64_t OFF_B2 = OFF_W2 + (int64_t)MLP_H * MLP_H;
constexpr int64_t OFF_W3 = OFF_B2 + MLP_H;
constexpr int64_t OFF_B3 = OFF_W3 + (int64_t)MLP_S * MLP_H;
constexpr int64_t NPARAM = OFF_B3 + MLP_S;
constexpr int64_t BOFF_W1 = 0;
constexpr int64_t BOFF_W2 = BOFF_W1 + (int64_t)MLP_H * MLP_F;
constexpr int64_t BOFF_W3 = BOFF_W2 + (int64_t)MLP_H * MLP_H;
constexpr int64_t NBF = BOFF_W3 + (int64_t)MLP_S * MLP_H;

int64_t mlp_param_count() { return NPARAM; }

// index of a flat parameter in the bf16 copy, or -1 for a bias
__device__ __forceinline__ int64_t bf_index(int64_t q) {
    if (q < OFF_B1) return BOFF_W1 + q;
    if (q >= OFF_W2 && q < OFF_B2) return BOFF_W2 + (q - OFF_W2);
    if (q >= OFF_W3 && q < OFF_B3) return BOFF_W3 + (q - OFF_W3);
    return -1;
}

// He-uniform weights W = (2u - 1) sqrt(6 / fan_in), u = SplitMix64 uniform of
// (seed, stream = layer, index); biases zero.
__global__ void k_mlp_init(uint64_t seed, float* __restrict__ P) {
    pdl_begin();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    int layer = -1;
    int64_t idx = 0;
    int fan = 1;
    if (q < OFF_B1) {
        layer = 0, idx = q, fan = MLP_F;
    } else if (q >= OFF_W2 && q < OFF_B2) {
        layer = 1, idx = q - OFF_W2, fan = MLP_H;
    } else if (q >= OFF_W3 && q < OFF_B3) {
        layer = 2, idx = q - OFF_W3, fan = MLP_H;
    }
    if (layer < 0) {
        P[q] = 0.f;
        return;
    }
    const double u = counter_uniform(seed, (uint64_t)layer, (uint64_t)idx);
    P[q] = (float)((2.0 * u - 1.0) * sqrt(6.0 / (double)fan));
}

__global__ void k_mlp_to_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wb) {
    pdl_begin();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    const int64_t b = bf_index(q);
    if (b >= 0) Wb[b] = __float2bfloat16_rn(P[q]);
}

// ------------------------------------------------------------------ forward (tensor cores)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}
template <typename TA>
__device__ __forceinline__ uint32_t load_pair(const TA* p);  // elements p[0], p[1] as bf16x2
template <>
__device__ __forceinline__ uint32_t load_pair<float>(const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return pack_bf16(v.x, v.y);
}
template <>
__device__ __forceinline__ uint32_t load_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Y = act(A W^T + b): A is M x K (row-major, element type TA, rounded to bf16 on load), W
// is N x K bf16, b FP32.  relu: Yb (bf16, M x N) = max(0, .); else Yf (FP32) = the sum.
// Block: 4 warps x 16 rows.  K a multiple of 16, N a multiple of 8, N <= 128, K <= 128.
constexpr int FWD_WARPS = 4;
template <typename TA, int N, int K>
__global__ void __launch_bounds__(FWD_WARPS * 32)
    k_mlp_layer(int64_t M, const TA* __restrict__ A, const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                bool relu, __nv_bfloat16* __restrict__ Yb, float* __restrict__ Yf) {
    pdl_begin();
    constexpr int LDW = K + 8;  // padded stride (bf16 elements): conflict-free fragment loads
    __shared__ __align__(16) __nv_bfloat16 sW[N * LDW];
    __shared__ float sb[N];
    for (int idx = threadIdx.x; idx < N * K / 2; idx += blockDim.x) {
        const int n = (2 * idx) / K, k = (2 * idx) % K;
        *reinterpret_cast<uint32_t*>(&sW[n * LDW + k]) = *reinterpret_cast<const uint32_t*>(&W[(int64_t)n * K + k]);
    }
    for (int n = threadIdx.x; n < N; n += blockDim.x) sb[n] = bias[n];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t r0 = ((int64_t)blockIdx.x * FWD_WARPS + warp) * 16;
    if (r0 >= M) return;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    const bool va = ra < M, vb = rb < M;
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        const uint32_t a0 = va ? load_pair<TA>(A + ra * K + kk + 2 * t) : 0u;
        const uint32_t a1 = vb ? load_pair<TA>(A + rb * K + kk + 2 * t) : 0u;
        const uint32_t a2 = va ? load_pair<TA>(A + ra * K + kk + 2 * t + 8) : 0u;
        const uint32_t a3 = vb ? load_pair<TA>(A + rb * K + kk + 2 * t + 8) : 0u;
#pragma unroll
        for (int nt = 0; nt < N / 8; ++nt) {
            const __nv_bfloat16* wr = sW + (nt * 8 + g) * LDW + kk + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 8);
            mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        float v0 = acc[nt][0] + sb[c], v1 = acc[nt][1] + sb[c + 1];
        float v2 = acc[nt][2] + sb[c], v3 = acc[nt][3] + sb[c + 1];
        if (relu) {
            v0 = fmaxf(v0, 0.f), v1 = fmaxf(v1, 0.f), v2 = fmaxf(v2, 0.f), v3 = fmaxf(v3, 0.f);
            if (va) *reinterpret_cast<uint32_t*>(Yb + ra * N + c) = pack_bf16(v0, v1);
            if (vb) *reinterpret_cast<uint32_t*>(Yb + rb * N + c) = pack_bf16(v2, v3);
        } else {
            if (va) *reinterpret_cast<float2*>(Yf + ra * N + c) = make_float2(v0, v1);
            if (vb) *reinterpret_cast<float2*>(Yf + rb * N + c) = make_float2(v2, v3);
        }
    }
}

// ------------------------------------------------------------------ backward
// dY = (2 / rows_in_batch) mask (Y - T), mask = the features' slot-valid flags; the batch
// loss sum mask (Y - T)^2 / rows_in_batch is added to *loss.
__global__ void k_mlp_loss(int64_t M, int64_t Mtot, const float* __restrict__ Y, const float* __restrict__ Tg,
                           const float* __restrict__ Fe, float* __restrict__ dY, double* __restrict__ loss) {
    pdl_begin();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (q < M * MLP_S) {
        const int64_t row = q / MLP_S;
        const int s = (int)(q - row * MLP_S);
        const float mask = Fe[row * MLP_F + MLP_NF_SLOT * s] > 0.f ? 1.f : 0.f;
        const float d = mask * (Y[q] - Tg[q]);
        dY[q] = 2.f * d / (float)Mtot;
        l = (double)d * (double)d / (double)Mtot;
    }
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// The backward products on the tensor cores as well (mma.sync m16n8k16, bf16 in, FP32
// accumulate): the gradient entering a product is rounded to bf16 like the forward's inputs;
// the bias gradients are FP32 sums of the unrounded gradients (k_colsum).

// Dout[m][n] = (sum_k bf16(Din[m][k]) W[k][n]) * (H[m][n] > 0): the gradient at a layer's
// input (W: K x N bf16, the layer's out x in weights) through the ReLU of the layer below
// (H: that layer's bf16 output).  As the forward tile: 4 warps x 16 rows per block, W^T
// staged once per block with a padded stride.  K a multiple of 16, N of 8.
template <int N, int K>
__global__ void __launch_bounds__(FWD_WARPS * 32)
    k_mlp_dgrad(int64_t M, const float* __restrict__ Din, const __nv_bfloat16* __restrict__ W,
                const __nv_bfloat16* __restrict__ Hm, float* __restrict__ Dout) {
    pdl_begin();
    constexpr int LDW = K + 8;
    __shared__ __align__(16) __nv_bfloat16 sWT[N * LDW];  // sWT[n][k] = W[k][n]
    for (int idx = threadIdx.x; idx < N * K; idx += blockDim.x) {
        const int k = idx / N, n = idx - k * N;
        sWT[n * LDW + k] = W[(int64_t)k * N + n];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t r0 = ((int64_t)blockIdx.x * FWD_WARPS + warp) * 16;
    if (r0 >= M) return;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
    const bool va = ra < M, vb = rb < M;
    float acc[N / 8][4];
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        const uint32_t a0 = va ? load_pair<float>(Din + ra * K + kk + 2 * t) : 0u;
        const uint32_t a1 = vb ? load_pair<float>(Din + rb * K + kk + 2 * t) : 0u;
        const uint32_t a2 = va ? load_pair<float>(Din + ra * K + kk + 2 * t + 8) : 0u;
        const uint32_t a3 = vb ? load_pair<float>(Din + rb * K + kk + 2 * t + 8) : 0u;
#pragma unroll
        for (int nt = 0; nt < N / 8; ++nt) {
            const __nv_bfloat16* wr = sWT + (nt * 8 + g) * LDW + kk + 2 * t;
            mma_bf16(acc[nt], a0, a1, a2, a3, *reinterpret_cast<const uint32_t*>(wr),
                     *reinterpret_cast<const uint32_t*>(wr + 8));
        }
    }
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        if (va) {
            const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(Hm + ra * N + c);
            *reinterpret_cast<float2*>(Dout + ra * N + c) =
                make_float2(__low2float(h) > 0.f ? acc[nt][0] : 0.f, __high2float(h) > 0.f ? acc[nt][1] : 0.f);
        }
        if (vb) {
            const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(Hm + rb * N + c);
            *reinterpret_cast<float2*>(Dout + rb * N + c) =
                make_float2(__low2float(h) > 0.f ? acc[nt][2] : 0.f, __high2float(h) > 0.f ? acc[nt][3] : 0.f);
        }
    }
}

// G[n][k] += sum_m bf16(D[m][n]) X[m][k]: a layer's weight gradient from the gradient at its
// output (D: M x N FP32) and its input (X: M x K, bf16 activations or the FP32 features,
// rounded to bf16).  Block (x, y): rows [x WG_ROWS, +WG_ROWS) and the output rows
// n in [16 y, 16 y + 16).  Rows in chunks of WG_MC; both operands staged transposed in shared
// memory (row index m contiguous, so each fragment register is one aligned pair), padded
// so that the fragment loads are free of bank conflicts; the 16 x 8 output tiles of the slab
// spread over the warps; the block's partial sums go to G with atomics.
constexpr int WG_MC = 64, WG_WARPS = 4, WG_ROWS = 256;
template <typename TX, int N, int K>
__global__ void __launch_bounds__(WG_WARPS * 32)
    k_mlp_wgrad(int64_t M, const float* __restrict__ D, const TX* __restrict__ X, float* __restrict__ G) {
    pdl_begin();
    static_assert(N % 16 == 0 && K % 8 == 0, "tile sizes");
    constexpr int LDM = WG_MC + 8;                                  // padded row stride (bf16 elements)
    constexpr int TK = K / 8, TPW = (TK + WG_WARPS - 1) / WG_WARPS;  // output tiles per warp
    __shared__ __align__(16) __nv_bfloat16 sDT[16 * LDM];           // sDT[n - n0][m - m0]
    __shared__ __align__(16) __nv_bfloat16 sXT[K * LDM];            // sXT[k][m - m0]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int n0 = blockIdx.y * 16;
    const int64_t m_begin = (int64_t)blockIdx.x * WG_ROWS;
    const int64_t m_end = m_begin + WG_ROWS < M ? m_begin + WG_ROWS : M;
    float acc[TPW][4];
#pragma unroll
    for (int q = 0; q < TPW; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
    for (int64_t m0 = m_begin; m0 < m_end; m0 += WG_MC) {
        // rows m0 + 2i, m0 + 2i + 1 of D (slab columns) and X, as bf16 pairs along m
        for (int idx = threadIdx.x; idx < (WG_MC / 2) * 16; idx += blockDim.x) {
            const int i = idx >> 4, n = idx & 15;
            const int64_t m = m0 + 2 * i;
            const float d0 = m < m_end ? D[m * N + n0 + n] : 0.f;
            const float d1 = m + 1 < m_end ? D[(m + 1) * N + n0 + n] : 0.f;
            *reinterpret_cast<uint32_t*>(&sDT[n * LDM + 2 * i]) = pack_bf16(d0, d1);
        }
        for (int idx = threadIdx.x; idx < (WG_MC / 2) * K; idx += blockDim.x) {
            const int i = idx / K, k = idx - i * K;
            const int64_t m = m0 + 2 * i;
            float x0 = 0.f, x1 = 0.f;
            if constexpr (sizeof(TX) == 2) {
                if (m < m_end) x0 = __bfloat162float(X[m * K + k]);
                if (m + 1 < m_end) x1 = __bfloat162float(X[(m + 1) * K + k]);
            } else {
                if (m < m_end) x0 = X[m * K + k];
                if (m + 1 < m_end) x1 = X[(m + 1) * K + k];
            }
            *reinterpret_cast<uint32_t*>(&sXT[k * LDM + 2 * i]) = pack_bf16(x0, x1);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            const int tk = warp + q * WG_WARPS;
            if (tk < TK) {
#pragma unroll
                for (int kk = 0; kk < WG_MC; kk += 16) {
                    const __nv_bfloat16* ar = sDT + g * LDM + kk + 2 * t;
                    const __nv_bfloat16* br = sXT + (tk * 8 + g) * LDM + kk + 2 * t;
                    mma_bf16(acc[q], *reinterpret_cast<const uint32_t*>(ar),
                             *reinterpret_cast<const uint32_t*>(ar + 8 * LDM), *reinterpret_cast<const uint32_t*>(ar + 8),
                             *reinterpret_cast<const uint32_t*>(ar + 8 * LDM + 8), *reinterpret_cast<const uint32_t*>(br),
                             *reinterpret_cast<const uint32_t*>(br + 8));
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < TPW; ++q) {
        const int tk = warp + q * WG_WARPS;
        if (tk < TK) {
            const int k = tk * 8 + 2 * t;
            float* gr = G + (int64_t)(n0 + g) * K + k;
            atomicAdd(gr, acc[q][0]);
            atomicAdd(gr + 1, acc[q][1]);
            atomicAdd(gr + 8 * K, acc[q][2]);
            atomicAdd(gr + 8 * K + 1, acc[q][3]);
        }
    }
}

// g[n] += sum_m D[m][n]
__global__ void k_colsum(int64_t M, int N, const float* __restrict__ D, float* __restrict__ g) {
    pdl_begin();
    const int n = blockIdx.x;
    float s = 0.f;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) s += D[m * N + n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        g[n] += tot;
    }
}

// Adam (bias-corrected), then the bf16 copy of the weights.
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                       float* __restrict__ Vo, __nv_bfloat16* __restrict__ Wb, float lr, float c1, float c2) {
    pdl_begin();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    const float g = G[q];
    const float m = 0.9f * Mo[q] + 0.1f * g;
    const float v = 0.999f * Vo[q] + 0.001f * g * g;
    Mo[q] = m;
    Vo[q] = v;
    const float p = P[q] - lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
    P[q] = p;
    const int64_t b = bf_index(q);
    if (b >= 0) Wb[b] = __float2bfloat16_rn(p);
}

// ------------------------------------------------------------------ the model object
struct Model {
    DevBuf<float> P, G, Mo, Vo;
    DevBuf<__nv_bfloat16> Wb;
    int t = 0;
};

Model* mlp_create(uint64_t seed, cudaStream_t s) {
    AllocStream as_(s);
    auto* m = new Model();
    m->P.alloc(NPARAM);
    m->G.alloc(NPARAM);
    m->Mo.alloc(NPARAM);
    m->Vo.alloc(NPARAM);
    m->Wb.alloc(NBF);
    BAMG_LAUNCH(k_mlp_init, blocks_for(NPARAM, 256), 256, 0, s, seed, m->P.get());
    BAMG_LAUNCH(k_mlp_to_bf16, blocks_for(NPARAM, 256), 256, 0, s, m->P.get(), m->Wb.get());
    BAMG_CK(cudaMemsetAsync(m->Mo.get(), 0, sizeof(float) * NPARAM, s));
    BAMG_CK(cudaMemsetAsync(m->Vo.get(), 0, sizeof(float) * NPARAM, s));
    return m;
}
void mlp_destroy(Model* m) { delete m; }

void mlp_set(Model* m, const float* h_params, cudaStream_t s) {
    BAMG_CK(cudaMemcpyAsync(m->P.get(), h_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    BAMG_LAUNCH(k_mlp_to_bf16, blocks_for(NPARAM, 256), 256, 0, s, m->P.get(), m->Wb.get());
    BAMG_CK(cudaMemsetAsync(m->Mo.get(), 0, sizeof(float) * NPARAM, s));
    BAMG_CK(cudaMemsetAsync(m->Vo.get(), 0, sizeof(float) * NPARAM, s));
    m->t = 0;
}
void mlp_get(const Model* m, float* h_params, cudaStream_t s) {
    BAMG_CK(cudaMemcpyAsync(h_params, m->P.get(), sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
}

// Activations of one batch of rows.
struct MlpWork {
    DevBuf<__nv_bfloat16> H1, H2;
    DevBuf<float> Y, dY, D2, D1;
    DevBuf<double> loss;
    void ensure(int64_t rows, bool train) {
        H1.ensure(rows * MLP_H);
        H2.ensure(rows * MLP_H);
        Y.ensure(rows * MLP_S);
        if (train) {
            dY.ensure(rows * MLP_S);
            D2.ensure(rows * MLP_H);
            D1.ensure(rows * MLP_H);
            loss.ensure(1);
        }
    }
};

static void forward_rows(const Model* m, int64_t rows, const float* feat, MlpWork& w, float* Y, cudaStream_t s) {
    const unsigned g = blocks_for(rows, FWD_WARPS * 16);
    const float* P = m->P.get();
    const __nv_bfloat16* Wb = m->Wb.get();
    BAMG_LAUNCH((k_mlp_layer<float, MLP_H, MLP_F>), g, FWD_WARPS * 32, 0, s, rows, feat, Wb + BOFF_W1, P + OFF_B1, true,
                w.H1.get(), (float*)nullptr);
    BAMG_LAUNCH((k_mlp_layer<__nv_bfloat16, MLP_H, MLP_H>), g, FWD_WARPS * 32, 0, s, rows,
                (const __nv_bfloat16*)w.H1.get(), Wb + BOFF_W2, P + OFF_B2, true, w.H2.get(), (float*)nullptr);
    BAMG_LAUNCH((k_mlp_layer<__nv_bfloat16, MLP_S, MLP_H>), g, FWD_WARPS * 32, 0, s, rows,
                (const __nv_bfloat16*)w.H2.get(), Wb + BOFF_W3, P + OFF_B3, false, (__nv_bfloat16*)nullptr, Y);
}

void mlp_forward(const Model* m, int64_t rows, const float* feat, float* Y, cudaStream_t s) {
    if (rows <= 0) return;
    AllocStream as_(s);
    MlpWork w;
    w.ensure(rows, false);
    forward_rows(m, rows, feat, w, Y, s);
}

// Gradients of the batch loss into m->G (zeroed first); the loss sum into w.loss.
static void gradients(Model* m, int64_t rows, const float* feat, const float* target, MlpWork& w, cudaStream_t s) {
    forward_rows(m, rows, feat, w, w.Y.get(), s);
    float* G = m->G.get();
    const __nv_bfloat16* Wb = m->Wb.get();
    BAMG_CK(cudaMemsetAsync(G, 0, sizeof(float) * NPARAM, s));
    BAMG_LAUNCH(k_mlp_loss, blocks_for(rows * MLP_S, 256), 256, 0, s, rows, rows, w.Y.get(), target, feat, w.dY.get(),
                w.loss.get());
    const unsigned zb = (unsigned)((rows + WG_ROWS - 1) / WG_ROWS), gd = blocks_for(rows, FWD_WARPS * 16);
    // layer 3
    BAMG_LAUNCH((k_mlp_wgrad<__nv_bfloat16, MLP_S, MLP_H>), dim3(zb, MLP_S / 16), WG_WARPS * 32, 0, s, rows,
                (const float*)w.dY.get(), (const __nv_bfloat16*)w.H2.get(), G + OFF_W3);
    BAMG_LAUNCH(k_colsum, MLP_S, 256, 0, s, rows, MLP_S, (const float*)w.dY.get(), G + OFF_B3);
    BAMG_LAUNCH((k_mlp_dgrad<MLP_H, MLP_S>), gd, FWD_WARPS * 32, 0, s, rows, (const float*)w.dY.get(),
                Wb + BOFF_W3, (const __nv_bfloat16*)w.H2.get(), w.D2.get());
    // layer 2
    BAMG_LAUNCH((k_mlp_wgrad<__nv_bfloat16, MLP_H, MLP_H>), dim3(zb, MLP_H / 16), WG_WARPS * 32, 0, s, rows,
                (const float*)w.D2.get(), (const __nv_bfloat16*)w.H1.get(), G + OFF_W2);
    BAMG_LAUNCH(k_colsum, MLP_H, 256, 0, s, rows, MLP_H, (const float*)w.D2.get(), G + OFF_B2);
    BAMG_LAUNCH((k_mlp_dgrad<MLP_H, MLP_H>), gd, FWD_WARPS * 32, 0, s, rows, (const float*)w.D2.get(),
                Wb + BOFF_W2, (const __nv_bfloat16*)w.H1.get(), w.D1.get());
    // layer 1
    BAMG_LAUNCH((k_mlp_wgrad<float, MLP_H, MLP_F>), dim3(zb, MLP_H / 16), WG_WARPS * 32, 0, s, rows,
                (const float*)w.D1.get(), feat, G + OFF_W1);
    BAMG_LAUNCH(k_colsum, MLP_H, 256, 0, s, rows, MLP_H, (const float*)w.D1.get(), G + OFF_B1);
}

double mlp_gradients(Model* m, int64_t rows, const float* feat, const float* target, float* h_grad, cudaStream_t s) {
    BAMG_REQUIRE(rows > 0, BAMG_EINVAL, "mlp_gradients: no rows");
    AllocStream as_(s);
    MlpWork w;
    w.ensure(rows, true);
    BAMG_CK(cudaMemsetAsync(w.loss.get(), 0, sizeof(double), s));
    gradients(m, rows, feat, target, w, s);
    double l = 0.0;
    BAMG_CK(cudaMemcpyAsync(&l, w.loss.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
    if (h_grad) BAMG_CK(cudaMemcpyAsync(h_grad, m->G.get(), sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    return l;
}

void mlp_train(Model* m, int64_t rows, const float* feat, const float* target, int epochs, int batch, double lr,
               double* h_loss, cudaStream_t s) {
    BAMG_REQUIRE(rows > 0 && epochs >= 0 && batch > 0, BAMG_EINVAL, "mlp_train: bad sizes");
    AllocStream as_(s);
    MlpWork w;
    w.ensure(std::min<int64_t>(rows, batch), true);
    for (int e = 0; e < epochs; ++e) {
        BAMG_CK(cudaMemsetAsync(w.loss.get(), 0, sizeof(double), s));
        int64_t nb = 0;
        for (int64_t r0 = 0; r0 < rows; r0 += batch, ++nb) {
            const int64_t br = std::min<int64_t>(batch, rows - r0);
            gradients(m, br, feat + r0 * MLP_F, target + r0 * MLP_S, w, s);
            m->t += 1;
            const float c1 = (float)(1.0 - std::pow(0.9, m->t)), c2 = (float)(1.0 - std::pow(0.999, m->t));
            BAMG_LAUNCH(k_adam, blocks_for(NPARAM, 256), 256, 0, s, m->P.get(), (const float*)m->G.get(),
                        m->Mo.get(), m->Vo.get(), m->Wb.get(), (float)lr, c1, c2);
        }
        if (h_loss) {
            double l = 0.0;
            BAMG_CK(cudaMemcpyAsync(&l, w.loss.get(), sizeof(double), cudaMemcpyDeviceToHost, s));
            BAMG_CK(cudaStreamSynchronize(s));
            h_loss[e] = l / (double)nb;  // mean of the batch losses
        }
    }
    BAMG_CK(cudaStreamSynchronize(s));
}

}  // namespace bamg
