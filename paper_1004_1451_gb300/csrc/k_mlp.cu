// Learned interpolation: the 112-128-128-16 ReLU MLP that predicts a fine point's row of
// P from its features, trained on the least-squares rows of Algorithm 2 (Eq. (3.6)).
// The paper has no learned interpolation; the definitions (features, bfloat16-rounded
// product inputs with FP32 sums, masked MSE, Adam of Kingma & Ba with beta1 = 0.9,
// beta2 = 0.999, eps = 1e-8, He-uniform initialisation from SplitMix64) are those of the
// interface declared in include/bamg.h.
//
// Forward products run on the tensor cores (mma.sync m16n8k16, bf16 in, FP32 accumulate):
// one warp computes 16 rows x N outputs, the weights staged once per block in shared
// memory with a padded row stride.  The training backward products (weight gradients
// summed over the batch, input gradients) are small FP32-accumulating SIMT tiles.
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

// ------------------------------------------------------------------ backward (SIMT)
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

// G[n][k] += sum_m D[m][n] X[m][k] (D: M x N FP32, X: M x K bf16 or FP32 rounded to bf16)
// for rows [blockIdx.z * 128, +128); 32 x 32 output tile per block, 2 x 2 per thread.
template <typename TX>
__global__ void __launch_bounds__(256) k_gemm_tn(int64_t M, int N, int K, const float* __restrict__ D,
                                                 const TX* __restrict__ X, float* __restrict__ G) {
    pdl_begin();
    __shared__ float sD[32][33], sX[32][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int n0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int64_t m_begin = (int64_t)blockIdx.z * 128, m_end = min(M, m_begin + 128);
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int64_t m0 = m_begin; m0 < m_end; m0 += 32) {
        for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
            const int mm = idx >> 5, cc = idx & 31;
            const int64_t m = m0 + mm;
            sD[mm][cc] = (m < m_end && n0 + cc < N) ? D[m * N + n0 + cc] : 0.f;
            float xv = 0.f;
            if (m < m_end && k0 + cc < K) {
                if constexpr (sizeof(TX) == 2)
                    xv = __bfloat162float(X[m * K + k0 + cc]);
                else
                    xv = __bfloat162float(__float2bfloat16_rn(X[m * K + k0 + cc]));
            }
            sX[mm][cc] = xv;
        }
        __syncthreads();
#pragma unroll 8
        for (int mm = 0; mm < 32; ++mm) {
            const float d0 = sD[mm][ty], d1 = sD[mm][ty + 16];
            const float x0 = sX[mm][tx], x1 = sX[mm][tx + 16];
            acc[0][0] += d0 * x0, acc[0][1] += d0 * x1, acc[1][0] += d1 * x0, acc[1][1] += d1 * x1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int n = n0 + ty + 16 * a, k = k0 + tx + 16 * b;
            if (n < N && k < K) atomicAdd(&G[(int64_t)n * K + k], acc[a][b]);
        }
}

// O[m][k] = (sum_n D[m][n] W[n][k]) * (H[m][k] > 0): D FP32 M x N, W bf16 N x K, H bf16.
__global__ void __launch_bounds__(256) k_gemm_nn_relu(int64_t M, int N, int K, const float* __restrict__ D,
                                                      const __nv_bfloat16* __restrict__ W,
                                                      const __nv_bfloat16* __restrict__ Hm, float* __restrict__ O) {
    pdl_begin();
    __shared__ float sD[32][33], sW[32][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 32;
    const int k0 = blockIdx.x * 32;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int n0 = 0; n0 < N; n0 += 32) {
        for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
            const int a = idx >> 5, b = idx & 31;
            const int64_t m = m0 + a;
            sD[a][b] = (m < M && n0 + b < N) ? D[m * N + n0 + b] : 0.f;
            sW[a][b] = (n0 + a < N && k0 + b < K) ? __bfloat162float(W[(int64_t)(n0 + a) * K + k0 + b]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int nn = 0; nn < 32; ++nn) {
            const float d0 = sD[ty][nn], d1 = sD[ty + 16][nn];
            const float w0 = sW[nn][tx], w1 = sW[nn][tx + 16];
            acc[0][0] += d0 * w0, acc[0][1] += d0 * w1, acc[1][0] += d1 * w0, acc[1][1] += d1 * w1;
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t m = m0 + ty + 16 * a;
            const int k = k0 + tx + 16 * b;
            if (m < M && k < K) {
                const float h = __bfloat162float(Hm[m * K + k]);
                O[m * K + k] = h > 0.f ? acc[a][b] : 0.f;
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
    const unsigned zb = (unsigned)((rows + 127) / 128);
    // layer 3
    BAMG_LAUNCH(k_gemm_tn<__nv_bfloat16>, dim3(MLP_H / 32, 1, zb), 256, 0, s, rows, MLP_S, MLP_H,
                (const float*)w.dY.get(), (const __nv_bfloat16*)w.H2.get(), G + OFF_W3);
    BAMG_LAUNCH(k_colsum, MLP_S, 256, 0, s, rows, MLP_S, (const float*)w.dY.get(), G + OFF_B3);
    BAMG_LAUNCH(k_gemm_nn_relu, dim3(MLP_H / 32, blocks_for(rows, 32)), 256, 0, s, rows, MLP_S, MLP_H,
                (const float*)w.dY.get(), Wb + BOFF_W3, (const __nv_bfloat16*)w.H2.get(), w.D2.get());
    // layer 2
    BAMG_LAUNCH(k_gemm_tn<__nv_bfloat16>, dim3(MLP_H / 32, MLP_H / 32, zb), 256, 0, s, rows, MLP_H, MLP_H,
                (const float*)w.D2.get(), (const __nv_bfloat16*)w.H1.get(), G + OFF_W2);
    BAMG_LAUNCH(k_colsum, MLP_H, 256, 0, s, rows, MLP_H, (const float*)w.D2.get(), G + OFF_B2);
    BAMG_LAUNCH(k_gemm_nn_relu, dim3(MLP_H / 32, blocks_for(rows, 32)), 256, 0, s, rows, MLP_H, MLP_H,
                (const float*)w.D2.get(), Wb + BOFF_W2, (const __nv_bfloat16*)w.H1.get(), w.D1.get());
    // layer 1
    BAMG_LAUNCH(k_gemm_tn<float>, dim3(MLP_F / 32 + (MLP_F % 32 ? 1 : 0), MLP_H / 32, zb), 256, 0, s, rows, MLP_H,
                MLP_F, (const float*)w.D1.get(), feat, G + OFF_W1);
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
