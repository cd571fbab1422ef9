// Coarsest level (Algorithm 3, first branch; Section 4.2): the eigenpairs of
// B_L x = lambda T_L x with the smallest |lambda|, and the minimal-norm inverse B_L^+.
// Order n <= 64, matrices in shared memory, 256 threads per block.
//
// Eigenvalues (FP32; they only serve as shifts): shift-and-invert Arnoldi on the explicit
// operator K = (B - sigma T)^{-1} T, then the Francis double-shift QR iteration on the
// small Hessenberg matrix (Golub & Van Loan, Matrix Computations, Sec. 7.5).
// Eigenvectors, one block per selected eigenvalue: inverse iteration in complex
// arithmetic on the pencil (B - sigma T) and a Rayleigh-type quotient, in FP64 (or in
// FP32 for the mixed-precision setup).  B^+: a bordered FP64 LU solve, the right-hand
// sides split over several blocks.  Factorisations use the whole block; triangular
// solves run in single warps (registers and shuffles, no block barriers).
#include <cfloat>
#include <cstdio>
#include <cstdlib>

#include <atomic>

#include "kernels.cuh"

namespace bamg {

constexpr int CN = 64;
constexpr int LDP = CN + 1;  // padded row stride of shared matrices (no bank conflicts on columns)
constexpr int CT = 256;      // threads per block

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
template <typename F>
__device__ __forceinline__ F absv(F x) {
    return x < F(0) ? -x : x;
}

// ---------------------------------------------------------------- block-parallel real LU
// In-place LU with partial pivoting of the n x n row-major A (shared, stride LDP);
// perm[k] = pivot row of step k; pivots smaller than floorv in magnitude become
// +-floorv.  On return the strict lower part holds L (unit diagonal), dinv[k] = 1 / u_kk,
// and the strict upper part holds the rows of U scaled by dinv (a unit upper factor),
// so that a solve needs no division.  Rank-one updates use a 16 x 16 thread grid.
template <typename F>
__device__ void blu_factor(F* A, int n, int* perm, F* dinv, F floorv) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {  // pivot search; one thread forms the (floored) pivot's reciprocal
            F best = F(-1);
            int br = k;
            for (int r = k + tid; r < n; r += 32) {
                const F v = absv(A[r * LDP + k]);
                if (v > best) {
                    best = v;
                    br = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const F ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) {
                perm[k] = br;
                F p = A[br * LDP + k];
                if (absv(p) < floorv) p = p >= F(0) ? floorv : -floorv;
                dinv[k] = F(1) / p;
                A[br * LDP + k] = p;  // lands on the diagonal with the row swap
            }
        }
        __syncthreads();
        const int br = perm[k];
        if (br != k) {
            for (int c = tid; c < n; c += CT) {
                const F t = A[k * LDP + c];
                A[k * LDP + c] = A[br * LDP + c];
                A[br * LDP + c] = t;
            }
            __syncthreads();
        }
        const F inv = dinv[k];
        // rank-one update, a 4 x 4 register tile per thread (n <= 64)
        F u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = k + 1 + tx + 16 * j;
            u[j] = c < n ? A[k * LDP + c] : F(0);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = k + 1 + ty + 16 * i;
            if (r < n) {
                const F l = A[r * LDP + k] * inv;
                F a[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = k + 1 + tx + 16 * j;
                    a[j] = c < n ? A[r * LDP + c] : F(0);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = k + 1 + tx + 16 * j;
                    if (c < n) A[r * LDP + c] = a[j] - l * u[j];
                }
            }
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < n; r += CT) A[r * LDP + k] *= inv;
    }
    __syncthreads();
    for (int r = ty; r < n; r += 16)
        for (int c = r + 1 + tx; c < n; c += 16) A[r * LDP + c] *= dinv[r];
    __syncthreads();
}

// One warp solves A X = R for the NC columns c0 .. c0 + NC - 1 (those < m) of the
// row-major R (row stride ldr) at once: the independent columns hide the latency of the
// shuffles.  Row interchanges, then forward and back substitution eliminating one column
// of L (of U) at a time, as in the plain algorithm.
template <typename F, int NC>
__device__ void warp_lu_solve_cols(const F* A, int n, const int* src, const F* dinv, F* R, int ldr, int c0, int m) {
    const int lane = lane_id();
    F x0[NC], x1[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const bool cj = c0 + j < m;
        x0[j] = lane < n && cj ? R[src[lane] * ldr + c0 + j] : F(0);
        x1[j] = lane + 32 < n && cj ? R[src[lane + 32] * ldr + c0 + j] : F(0);
    }
    __syncwarp();
    for (int q = 0; q + 1 < n; ++q) {  // unit lower
        const bool a0 = lane > q && lane < n, a1 = lane + 32 > q && lane + 32 < n;
        const F l0 = a0 ? A[lane * LDP + q] : F(0), l1 = a1 ? A[(lane + 32) * LDP + q] : F(0);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F y = __shfl_sync(0xffffffffu, q < 32 ? x0[j] : x1[j], q & 31);
            if (a0) x0[j] = x0[j] - l0 * y;
            if (a1) x1[j] = x1[j] - l1 * y;
        }
    }
    const F d0 = lane < n ? dinv[lane] : F(0), d1 = lane + 32 < n ? dinv[lane + 32] : F(0);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (lane < n) x0[j] *= d0;
        if (lane + 32 < n) x1[j] *= d1;
    }
    for (int q = n - 1; q > 0; --q) {  // unit upper
        const bool a0 = lane < q, a1 = lane + 32 < q;
        const F u0 = a0 ? A[lane * LDP + q] : F(0), u1 = a1 ? A[(lane + 32) * LDP + q] : F(0);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F y = __shfl_sync(0xffffffffu, q < 32 ? x0[j] : x1[j], q & 31);
            if (a0) x0[j] = x0[j] - u0 * y;
            if (a1) x1[j] = x1[j] - u1 * y;
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (c0 + j >= m) continue;
        if (lane < n) R[lane * ldr + c0 + j] = x0[j];
        if (lane + 32 < n) R[(lane + 32) * ldr + c0 + j] = x1[j];
    }
    __syncwarp();
}

// One warp solves A x = b for one right-hand side b (stride ldb) with the factor of
// blu_factor; src[i] is the row of b that the interchanges bring to row i
// (lu_row_sources).  Lane l holds x_l and x_{l+32}; the eliminations run one column of
// L (of U) at a time, as in the plain algorithm.  The warp's lanes must all call it.
__device__ void lu_row_sources(int n, const int* perm, int* src) {  // one thread
    for (int i = 0; i < n; ++i) src[i] = i;
    for (int k = 0; k < n; ++k) {
        const int pk = perm[k], t = src[k];
        src[k] = src[pk];
        src[pk] = t;
    }
}
template <typename F>
__device__ void warp_lu_solve(const F* A, int n, const int* src, const F* dinv, F* b, int ldb) {
    const int lane = lane_id();
    F x0 = lane < n ? b[src[lane] * ldb] : F(0);
    F x1 = lane + 32 < n ? b[src[lane + 32] * ldb] : F(0);
    __syncwarp();
    for (int q = 0; q + 1 < n; ++q) {  // unit lower
        const F y = __shfl_sync(0xffffffffu, q < 32 ? x0 : x1, q & 31);
        if (lane > q && lane < n) x0 = x0 - A[lane * LDP + q] * y;
        if (lane + 32 > q && lane + 32 < n) x1 = x1 - A[(lane + 32) * LDP + q] * y;
    }
    if (lane < n) x0 *= dinv[lane];
    if (lane + 32 < n) x1 *= dinv[lane + 32];
    for (int q = n - 1; q > 0; --q) {  // unit upper
        const F y = __shfl_sync(0xffffffffu, q < 32 ? x0 : x1, q & 31);
        if (lane < q) x0 = x0 - A[lane * LDP + q] * y;
        if (lane + 32 < q) x1 = x1 - A[(lane + 32) * LDP + q] * y;
    }
    if (lane < n) b[lane * ldb] = x0;
    if (lane + 32 < n) b[(lane + 32) * ldb] = x1;
    __syncwarp();
}

// ---------------------------------------------------------------- FP32 Hessenberg + QR

__device__ __forceinline__ void house3f(float x, float y, float z, float& v0, float& v1, float& v2, float& beta) {
    const float nrm = sqrtf(x * x + y * y + z * z);
    if (nrm == 0.f) {
        v0 = 1.f;
        v1 = v2 = 0.f;
        beta = 0.f;
        return;
    }
    const float alpha = -copysignf(nrm, x);
    v0 = x - alpha;
    v1 = y;
    v2 = z;
    beta = 2.f / (v0 * v0 + v1 * v1 + v2 * v2);
}

// Eigenvalues of the upper Hessenberg H (destroyed), one warp.  0, or -1 when the
// iteration did not converge within 40 n double-shift steps.
__device__ int hqr_f32(float* H, int n, float* wr, float* wi, int* steps) {
    const int lane = lane_id();
    float hnorm = 0.f;
    for (int idx = lane; idx < n * n; idx += 32) hnorm = fmaxf(hnorm, fabsf(H[(idx / n) * LDP + idx % n]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hnorm = fmaxf(hnorm, __shfl_xor_sync(0xffffffffu, hnorm, o));
    if (hnorm == 0.f) hnorm = 1.f;
    int hi = n - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (total > 40 * n) return -1;
        int l = hi;
        while (l > 0) {
            float s = fabsf(H[(l - 1) * LDP + l - 1]) + fabsf(H[l * LDP + l]);
            if (s == 0.f) s = hnorm;
            if (fabsf(H[l * LDP + l - 1]) <= FLT_EPSILON * s) break;
            --l;
        }
        __syncwarp();
        if (l == hi) {
            if (lane == 0) {
                wr[hi] = H[hi * LDP + hi];
                wi[hi] = 0.f;
            }
            --hi;
            its = 0;
            __syncwarp();
            continue;
        }
        if (l == hi - 1) {
            const float a = H[(hi - 1) * LDP + hi - 1], b = H[(hi - 1) * LDP + hi];
            const float c = H[hi * LDP + hi - 1], d = H[hi * LDP + hi];
            const float p = 0.5f * (a - d), q = p * p + b * c, mid = d + p;
            if (lane == 0) {
                if (q >= 0.f) {
                    const float sq = sqrtf(q);
                    const float l1 = mid + copysignf(sq, mid);
                    const float det = a * d - b * c;
                    wr[hi - 1] = l1;
                    wr[hi] = l1 != 0.f ? det / l1 : mid - sq;
                    wi[hi - 1] = wi[hi] = 0.f;
                } else {
                    const float im = sqrtf(-q);
                    wr[hi - 1] = wr[hi] = mid;
                    wi[hi - 1] = im;
                    wi[hi] = -im;
                }
            }
            hi -= 2;
            its = 0;
            __syncwarp();
            continue;
        }
        float s, t;
        if (its == 10 || its == 20) {
            const float e = fabsf(H[hi * LDP + hi - 1]) + fabsf(H[(hi - 1) * LDP + hi - 2]);
            s = 1.5f * e;
            t = e * e;
        } else {
            s = H[(hi - 1) * LDP + hi - 1] + H[hi * LDP + hi];
            t = H[(hi - 1) * LDP + hi - 1] * H[hi * LDP + hi] - H[(hi - 1) * LDP + hi] * H[hi * LDP + hi - 1];
        }
        ++its;
        ++total;
        float x = H[l * LDP + l] * H[l * LDP + l] + H[l * LDP + l + 1] * H[(l + 1) * LDP + l] - s * H[l * LDP + l] + t;
        float y = H[(l + 1) * LDP + l] * (H[l * LDP + l] + H[(l + 1) * LDP + l + 1] - s);
        float z = H[(l + 1) * LDP + l] * H[(l + 2) * LDP + l + 1];
        __syncwarp();
        for (int k = l; k <= hi - 2; ++k) {
            float v0, v1, v2, beta;
            house3f(x, y, z, v0, v1, v2, beta);
            const int c0 = k - 1 > l ? k - 1 : l;
            for (int c = c0 + lane; c <= hi; c += 32) {
                const float d = beta * (v0 * H[k * LDP + c] + v1 * H[(k + 1) * LDP + c] + v2 * H[(k + 2) * LDP + c]);
                H[k * LDP + c] -= d * v0;
                H[(k + 1) * LDP + c] -= d * v1;
                H[(k + 2) * LDP + c] -= d * v2;
            }
            __syncwarp();
            const int r1 = k + 3 < hi ? k + 3 : hi;
            for (int r = l + lane; r <= r1; r += 32) {
                const float d = beta * (H[r * LDP + k] * v0 + H[r * LDP + k + 1] * v1 + H[r * LDP + k + 2] * v2);
                H[r * LDP + k] -= d * v0;
                H[r * LDP + k + 1] -= d * v1;
                H[r * LDP + k + 2] -= d * v2;
            }
            __syncwarp();
            x = H[(k + 1) * LDP + k];
            y = H[(k + 2) * LDP + k];
            z = (k + 3 <= hi) ? H[(k + 3) * LDP + k] : 0.f;
            __syncwarp();
        }
        {
            float v0, v1, v2, beta;
            house3f(x, y, 0.f, v0, v1, v2, beta);
            const int k = hi - 1;
            for (int c = (k - 1) + lane; c <= hi; c += 32) {
                const float d = beta * (v0 * H[k * LDP + c] + v1 * H[(k + 1) * LDP + c]);
                H[k * LDP + c] -= d * v0;
                H[(k + 1) * LDP + c] -= d * v1;
            }
            __syncwarp();
            for (int r = l + lane; r <= hi; r += 32) {
                const float d = beta * (H[r * LDP + k] * v0 + H[r * LDP + k + 1] * v1);
                H[r * LDP + k] -= d * v0;
                H[r * LDP + k + 1] -= d * v1;
            }
            __syncwarp();
        }
    }
    *steps = total;
    return 0;
}

// Kernel 1: estimates of the eigenvalues of B x = lambda T x closest to zero, in FP32
// (they serve only as shifts).  sigma = -1e-4 max|B|; K = (B - sigma T)^{-1} T is formed
// explicitly (its dominant eigenvalues theta = 1 / (lambda - sigma) belong to the lambda
// of smallest modulus); KRY Arnoldi steps on K with classical Gram-Schmidt applied twice
// (whole block: 4 threads per row for K v, one warp per basis vector for the inner
// products); the eigenvalues of the Hessenberg matrix by the Francis QR iteration (one
// warp); lambda = sigma + 1 / theta.  Selection: eigenvalues with Im >= 0 (a complex pair
// is represented by its member with positive imaginary part) in order of |lambda|; a real
// one takes one vector column, a pair two (Re v, Im v), until k_ev columns are filled.
// sel[3q + {0,1,2}] = (Re, Im, first column); info = {columns, selected, status, steps,
// cycles of the phases}.
constexpr int KRY = 32;
__global__ void __launch_bounds__(CT) k_coarse_eigvals(int n, const double* __restrict__ Bg,
                                                       const double* __restrict__ Tg, int k_ev,
                                                       double* __restrict__ sel, double* __restrict__ lam,
                                                       int32_t* __restrict__ kind, int* __restrict__ info) {
    pdl_begin();
    __shared__ float A[CN * LDP], Km[CN * LDP];
    __shared__ float Vk[(KRY + 1) * CN];
    __shared__ float Hs[KRY * KRY];
    __shared__ float part[4 * CN];
    __shared__ float w[CN], hq[KRY + 1], hcol[KRY + 1], dinv[CN];
    __shared__ float wr[CN], wi[CN], red[CT / 32], s_nn;
    __shared__ int perm[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const long long c_start = clock64();
    // sigma from the largest entry of B
    float mx = 0.f;
    for (int idx = tid; idx < n * n; idx += CT) mx = fmaxf(mx, fabsf((float)Bg[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    mx = 0.f;
    for (int q = 0; q < CT / 32; ++q) mx = fmaxf(mx, red[q]);
    const float sigma = -1e-4f * fmaxf(mx, 1e-30f);
    for (int idx = tid; idx < n * n; idx += CT) {
        const int r = idx / n, c = idx - r * n;
        const float t = (float)Tg[idx];
        Km[r * LDP + c] = t;
        A[r * LDP + c] = (float)Bg[idx] - sigma * t;
    }
    __syncthreads();
    blu_factor<float>(A, n, perm, dinv, 1e-30f);
    {  // Km = (B - sigma T)^{-1} T, one column at a time per warp
        __shared__ int src[CN];
        if (tid == 0) lu_row_sources(n, perm, src);
        __syncthreads();
        warp_lu_solve_cols<float, CN / (CT / 32)>(A, n, src, dinv, Km, LDP, wid * (CN / (CT / 32)), n);
        __syncthreads();
    }
    const long long c_lu = clock64();
    const int kd = n < KRY ? n : KRY;
    if (tid < n) {  // v_0: fixed generic start
        Vk[tid] = 1.f + (float)tid / (float)n;
    }
    for (int idx = tid; idx < KRY * KRY; idx += CT) Hs[idx] = 0.f;
    __syncthreads();
    if (wid == 0) {
        float nn = 0.f;
        for (int r = lane; r < n; r += 32) nn += Vk[r] * Vk[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        if (lane == 0) s_nn = rsqrtf(nn);
    }
    __syncthreads();
    if (tid < n) Vk[tid] *= s_nn;
    __syncthreads();
    const int row = tid & (CN - 1), quarter = tid >> 6;  // K v: 4 threads per row
    int kk = kd;
    for (int k = 0; k < kd; ++k) {
        const float* vk = Vk + k * CN;
        if (row < n) {
            float acc = 0.f;
            const int c1 = min(n, 16 * quarter + 16);
            for (int c = 16 * quarter; c < c1; ++c) acc += Km[row * LDP + c] * vk[c];
            part[quarter * CN + row] = acc;
        }
        __syncthreads();
        if (tid < n) w[tid] = (part[tid] + part[CN + tid]) + (part[2 * CN + tid] + part[3 * CN + tid]);
        if (tid <= k) hcol[tid] = 0.f;
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = wid; q <= k; q += CT / 32) {
                float d = 0.f;
                for (int r = lane; r < n; r += 32) d += Vk[q * CN + r] * w[r];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                if (lane == 0) hq[q] = d;
            }
            __syncthreads();
            if (tid < n) {
                float acc = 0.f;
                for (int q = 0; q <= k; ++q) acc += Vk[q * CN + tid] * hq[q];
                w[tid] -= acc;
            }
            if (tid <= k) hcol[tid] += hq[tid];
            __syncthreads();
        }
        if (wid == 0) {
            float nn = 0.f;
            for (int r = lane; r < n; r += 32) nn += w[r] * w[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
            if (lane == 0) s_nn = sqrtf(nn);
        }
        __syncthreads();
        const float nn = s_nn;
        if (tid <= k) Hs[tid * KRY + k] = hcol[tid];
        if (k + 1 < kd && tid == 0) Hs[(k + 1) * KRY + k] = nn;
        if (!(nn > 1e-6f * fabsf(hcol[0]) + 1e-30f)) {  // invariant subspace found (uniform)
            kk = k + 1;
            break;
        }
        if (k + 1 < kd && tid < n) Vk[(k + 1) * CN + tid] = w[tid] / nn;
        __syncthreads();
    }
    __syncthreads();
    const long long c_arn = clock64();
    if (tid >= 32) return;
    // eigenvalues of the kk x kk Hessenberg matrix (copied to the padded stride)
    for (int idx = lane; idx < kk * kk; idx += 32) {
        const int r = idx / kk, c = idx % kk;
        A[r * LDP + c] = Hs[r * KRY + c];
    }
    __syncwarp();
    int steps = 0;
    const int st = hqr_f32(A, kk, wr, wi, &steps);
    __syncwarp();
    const long long c_qr = clock64();
    if (lane == 0) {
        // lambda = sigma + 1 / theta
        for (int q = 0; q < kk; ++q) {
            const float tr = wr[q], ti = wi[q];
            const float d = tr * tr + ti * ti;
            wr[q] = d > 0.f ? sigma + tr / d : 3.0e38f;
            wi[q] = d > 0.f ? -ti / d : 0.f;
        }
        int order[KRY];
        int m = 0;
        for (int q = 0; q < kk; ++q)
            if (wi[q] >= 0.f) order[m++] = q;
        for (int a = 1; a < m; ++a)
            for (int b = a; b > 0; --b) {
                const float m0 = hypotf(wr[order[b - 1]], wi[order[b - 1]]);
                const float m1 = hypotf(wr[order[b]], wi[order[b]]);
                if (m0 > m1) {
                    const int t = order[b];
                    order[b] = order[b - 1];
                    order[b - 1] = t;
                } else
                    break;
            }
        int col = 0, ns = 0;
        for (int a = 0; a < m && col < k_ev; ++a) {
            const int q = order[a];
            sel[3 * ns + 0] = wr[q];
            sel[3 * ns + 1] = wi[q];
            sel[3 * ns + 2] = (double)col;
            ++ns;
            if (wi[q] == 0.f) {
                lam[col] = wr[q];
                kind[col] = 0;
                col += 1;
            } else {
                lam[col] = lam[col + 1] = wr[q];
                kind[col] = 1;
                kind[col + 1] = 2;
                col += 2;
            }
        }
        if (col > 0) lam[0] = 0.0;
        info[0] = col;
        info[1] = ns;
        info[2] = st;
        info[3] = steps;
        info[4] = (int)(c_lu - c_start);  // phase durations in SM cycles (diagnostics)
        info[5] = (int)(c_arn - c_lu);
        info[6] = (int)(c_qr - c_arn);
        info[7] = (int)(clock64() - c_qr);
    }
}

// ---------------------------------------------------------------- complex inverse iteration
// Kernel 2, one block per selected eigenvalue, in arithmetic F (double, or float for the
// mixed-precision setup): LU of the pencil (B - sigma T) in complex arithmetic with sigma
// the FP32 estimate; four steps of inverse iteration v <- (B - sigma T)^{-1} T v from a
// fixed positive start; the Rayleigh-type quotient lambda = v^H B v / v^H T v (Algorithm
// 3's update, in complex form, accumulated in FP64); and the phase that makes <w, v> real
// and positive (w_i = i + 1) with unit 2-norm.
template <typename F>
__device__ __forceinline__ F pivot_tiny() {
    if constexpr (sizeof(F) == 8)
        return F(1e-300);
    else
        return F(1e-36f);
}

template <typename F>
__global__ void __launch_bounds__(CT) k_coarse_eigvec(int n, const double* __restrict__ Bg,
                                                      const double* __restrict__ Tg, const double* __restrict__ sel,
                                                      double* __restrict__ V, double* __restrict__ lam,
                                                      int* __restrict__ cycles) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smraw[];
    F* Ar = reinterpret_cast<F*>(smraw);
    F* Ai = Ar + CN * LDP;
    F* Bm = Ai + CN * LDP;
    F* Tm = Bm + CN * LDP;
    __shared__ F vr[CN], vi[CN], tr[CN], ti[CN], dr[CN], di[CN], pre[4 * CN], pim[4 * CN];
    __shared__ double red[4 * (CT / 32)];
    __shared__ int perm[CN];
    const long long c_start = clock64();
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5, ty = tid >> 4, tx = tid & 15;
    const F sr = (F)sel[3 * blockIdx.x], si = (F)sel[3 * blockIdx.x + 1];
    const int col = (int)sel[3 * blockIdx.x + 2];
    for (int idx = tid; idx < n * n; idx += CT) {
        const int r = idx / n, c = idx - r * n;
        const F b = (F)Bg[idx], t = (F)Tg[idx];
        Bm[r * LDP + c] = b;
        Tm[r * LDP + c] = t;
        Ar[r * LDP + c] = b - sr * t;
        Ai[r * LDP + c] = -si * t;
    }
    // pivot floor relative to the pencil's largest entry: near an eigenvalue the LU is
    // (nearly) singular by design, and an absolute floor would let the inverse iteration
    // overflow in FP32
    {
        F m = F(0);
        for (int idx = tid; idx < n * n; idx += CT) {
            const int r = idx / n, c = idx - r * n;
            const F a = absv(Ar[r * LDP + c]) + absv(Ai[r * LDP + c]);
            m = m > a ? m : a;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const F q = __shfl_xor_sync(0xffffffffu, m, o);
            m = m > q ? m : q;
        }
        if (lane == 0) pre[wid] = m;
    }
    __syncthreads();
    F amax = F(0);
    for (int q = 0; q < CT / 32; ++q) amax = amax > pre[q] ? amax : pre[q];
    const F pfloor = (sizeof(F) == 8 ? F(1e-15) : F(1e-7)) * (amax > F(0) ? amax : F(1));
    __syncthreads();
    // complex LU with partial pivoting on |Re| + |Im|; dr + i di = 1 / u_kk
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            F best = F(-1);
            int br = k;
            for (int r = k + tid; r < n; r += 32) {
                const F m = absv(Ar[r * LDP + k]) + absv(Ai[r * LDP + k]);
                if (m > best) {
                    best = m;
                    br = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const F ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) {  // the pivot's reciprocal, formed once
                perm[k] = br;
                F pr = Ar[br * LDP + k], pi = Ai[br * LDP + k];
                if (absv(pr) + absv(pi) < pfloor) {
                    pr = pfloor;
                    pi = F(0);
                    Ar[br * LDP + k] = pr;
                    Ai[br * LDP + k] = pi;
                }
                // 1 / (pr + i pi) without squaring (Smith's method: no underflow in FP32)
                if (absv(pr) >= absv(pi)) {
                    const F t = pi / pr, d = F(1) / (pr + pi * t);
                    dr[k] = d;
                    di[k] = -t * d;
                } else {
                    const F t = pr / pi, d = F(1) / (pr * t + pi);
                    dr[k] = t * d;
                    di[k] = -d;
                }
            }
        }
        __syncthreads();
        const int br = perm[k];
        if (br != k) {
            for (int c = tid; c < n; c += CT) {
                F t = Ar[k * LDP + c];
                Ar[k * LDP + c] = Ar[br * LDP + c];
                Ar[br * LDP + c] = t;
                t = Ai[k * LDP + c];
                Ai[k * LDP + c] = Ai[br * LDP + c];
                Ai[br * LDP + c] = t;
            }
            __syncthreads();
        }
        const F qr_ = dr[k], qi_ = di[k];  // 1 / pivot
        F ur[4], ui[4];  // rank-one update, a 4 x 4 register tile per thread
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = k + 1 + tx + 16 * j;
            ur[j] = c < n ? Ar[k * LDP + c] : F(0);
            ui[j] = c < n ? Ai[k * LDP + c] : F(0);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = k + 1 + ty + 16 * i;
            if (r < n) {
                const F ar = Ar[r * LDP + k], ai = Ai[r * LDP + k];
                const F lr = ar * qr_ - ai * qi_, li = ar * qi_ + ai * qr_;
                F xr[4], xi[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = k + 1 + tx + 16 * j;
                    xr[j] = c < n ? Ar[r * LDP + c] : F(0);
                    xi[j] = c < n ? Ai[r * LDP + c] : F(0);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = k + 1 + tx + 16 * j;
                    if (c < n) {
                        Ar[r * LDP + c] = xr[j] - (lr * ur[j] - li * ui[j]);
                        Ai[r * LDP + c] = xi[j] - (lr * ui[j] + li * ur[j]);
                    }
                }
            }
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < n; r += CT) {
            const F ar = Ar[r * LDP + k], ai = Ai[r * LDP + k];
            Ar[r * LDP + k] = ar * qr_ - ai * qi_;
            Ai[r * LDP + k] = ar * qi_ + ai * qr_;
        }
    }
    __syncthreads();
    for (int r = ty; r < n; r += 16)  // rows of U times 1 / u_rr: a unit upper factor
        for (int c = r + 1 + tx; c < n; c += 16) {
            const F ur = Ar[r * LDP + c], ui = Ai[r * LDP + c];
            Ar[r * LDP + c] = ur * dr[r] - ui * di[r];
            Ai[r * LDP + c] = ur * di[r] + ui * dr[r];
        }
    __shared__ int srcp[CN];
    if (tid == 0) lu_row_sources(n, perm, srcp);
    // start vector in [1, 2) drawn per column (SplitMix64, stream = the column): for a
    // multiple eigenvalue (the symmetric pairs of grid walks) each column converges to
    // the projection of its own start onto the eigenspace, so the columns span it
    // instead of repeating one vector
    if (tid < n) {
        vr[tid] = (F)(1.0 + counter_uniform(0x243F6A8885A308D3ull, (uint64_t)blockIdx.x, (uint64_t)tid));
        vi[tid] = F(0);
    }
    __syncthreads();
    const long long c_lu = clock64();
    // four steps of inverse iteration: t = T v by the block (4 threads per row), the
    // interchanges and the two triangular solves in warp 0 (registers and shuffles; lane l
    // holds rows l and l + 32), in the order of operations of the plain solve
    const int row = tid & (CN - 1), quarter = tid >> 6;
    for (int it = 0; it < 4; ++it) {
        if (row < n) {
            F a = F(0), b = F(0);
            const int c1 = min(n, 16 * quarter + 16);
            for (int c = 16 * quarter; c < c1; ++c) {
                const F t = Tm[row * LDP + c];
                a += t * vr[c];
                b += t * vi[c];
            }
            pre[quarter * CN + row] = a;
            pim[quarter * CN + row] = b;
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = lane + 32 * h;
                if (r < n) {
                    tr[r] = (pre[r] + pre[CN + r]) + (pre[2 * CN + r] + pre[3 * CN + r]);
                    ti[r] = (pim[r] + pim[CN + r]) + (pim[2 * CN + r] + pim[3 * CN + r]);
                }
            }
            __syncwarp();
            F xr[2], xi[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // row interchanges
                const int r = lane + 32 * h;
                xr[h] = r < n ? tr[srcp[r]] : F(0);
                xi[h] = r < n ? ti[srcp[r]] : F(0);
            }
            for (int q = 0; q + 1 < n; ++q) {  // unit lower
                const F yr = __shfl_sync(0xffffffffu, q < 32 ? xr[0] : xr[1], q & 31);
                const F yi = __shfl_sync(0xffffffffu, q < 32 ? xi[0] : xi[1], q & 31);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    if (r > q && r < n) {
                        const F lr = Ar[r * LDP + q], li = Ai[r * LDP + q];
                        xr[h] -= lr * yr - li * yi;
                        xi[h] -= lr * yi + li * yr;
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = lane + 32 * h;
                if (r < n) {
                    const F a = xr[h], b = xi[h];
                    xr[h] = a * dr[r] - b * di[r];
                    xi[h] = a * di[r] + b * dr[r];
                }
            }
            for (int q = n - 1; q > 0; --q) {  // unit upper
                const F yr = __shfl_sync(0xffffffffu, q < 32 ? xr[0] : xr[1], q & 31);
                const F yi = __shfl_sync(0xffffffffu, q < 32 ? xi[0] : xi[1], q & 31);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    if (r < q) {
                        const F ur = Ar[r * LDP + q], ui = Ai[r * LDP + q];
                        xr[h] -= ur * yr - ui * yi;
                        xi[h] -= ur * yi + ui * yr;
                    }
                }
            }
            double nn = 0.0;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane + 32 * h < n) nn += (double)xr[h] * xr[h] + (double)xi[h] * xi[h];
            nn = 1.0 / sqrt(warp_sum(nn));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = lane + 32 * h;
                if (r < n) {
                    vr[r] = (F)(xr[h] * nn);
                    vi[r] = (F)(xi[h] * nn);
                }
            }
        }
        __syncthreads();
    }
    // lambda = v^H B v / v^H T v: (B v)_r and (T v)_r with 4 threads per row
    {
        double br_ = 0.0, bi_ = 0.0, tr_ = 0.0, ti_ = 0.0;
        if (row < n) {
            F wbr = F(0), wbi = F(0), wtr = F(0), wti = F(0);
            const int c1 = min(n, 16 * quarter + 16);
            for (int c = 16 * quarter; c < c1; ++c) {
                const F b = Bm[row * LDP + c], t = Tm[row * LDP + c];
                wbr += b * vr[c];
                wbi += b * vi[c];
                wtr += t * vr[c];
                wti += t * vi[c];
            }
            const double xr = vr[row], xi = vi[row];
            br_ = xr * wbr + xi * wbi;
            bi_ = xr * wbi - xi * wbr;
            tr_ = xr * wtr + xi * wti;
            ti_ = xr * wti - xi * wtr;
        }
        br_ = warp_sum(br_);
        bi_ = warp_sum(bi_);
        tr_ = warp_sum(tr_);
        ti_ = warp_sum(ti_);
        if (lane == 0) {
            red[4 * wid] = br_;
            red[4 * wid + 1] = bi_;
            red[4 * wid + 2] = tr_;
            red[4 * wid + 3] = ti_;
        }
    }
    __syncthreads();
    if (tid >= 32) return;
    double sr2 = 0.0, si2 = 0.0;
    for (int r = lane; r < n; r += 32) {
        sr2 += (double)(r + 1) * vr[r];
        si2 += (double)(r + 1) * vi[r];
    }
    sr2 = warp_sum(sr2);
    si2 = warp_sum(si2);
    const double sa = hypot(sr2, si2);
    const double cr = sa > 0.0 ? sr2 / sa : 1.0, ci = sa > 0.0 ? -si2 / sa : 0.0;  // conj(s)/|s|
    double nn = 0.0;
    double ar[2], ai[2];
    for (int q = 0, r = lane; q < 2; ++q, r += 32) {
        ar[q] = ai[q] = 0.0;
        if (r < n) {
            ar[q] = (double)vr[r] * cr - (double)vi[r] * ci;
            ai[q] = (double)vr[r] * ci + (double)vi[r] * cr;
            nn += ar[q] * ar[q] + ai[q] * ai[q];
        }
    }
    nn = 1.0 / sqrt(warp_sum(nn));
    for (int q = 0, r = lane; q < 2; ++q, r += 32)
        if (r < n) {
            V[(int64_t)col * n + r] = ar[q] * nn;
            if (si != F(0)) V[(int64_t)(col + 1) * n + r] = ai[q] * nn;
        }
    if (lane == 0) {
        double nbr = 0.0, nbi = 0.0, ntr = 0.0, nti = 0.0;
        for (int q = 0; q < CT / 32; ++q) {
            nbr += red[4 * q];
            nbi += red[4 * q + 1];
            ntr += red[4 * q + 2];
            nti += red[4 * q + 3];
        }
        // Re of (nbr + i nbi) / (ntr + i nti)
        double lre = (nbr * ntr + nbi * nti) / (ntr * ntr + nti * nti);
        if (col == 0) lre = 0.0;  // the state vector's eigenvalue is exactly zero
        lam[col] = lre;
        if (si != F(0)) lam[col + 1] = lre;
        cycles[2 * blockIdx.x] = (int)(c_lu - c_start);  // diagnostics
        cycles[2 * blockIdx.x + 1] = (int)(clock64() - c_lu);
    }
}

int coarse_eig(int n, const double* dB, const double* dT, int k_ev, double* d_lam, double* d_V, int32_t* d_kind,
               bool fp32_vectors, cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_eig: coarsest order must be 1..64");
    BAMG_REQUIRE(k_ev >= 1 && k_ev <= 16, BAMG_EINVAL, "coarse_eig: 1 <= k_ev <= 16");
    // the attribute is per device (idempotent; several host threads may get here)
    static std::atomic<bool> attr[256] = {};
    int dev = 0;
    BAMG_CK(cudaGetDevice(&dev));
    BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
    const size_t smem64 = 4 * CN * LDP * sizeof(double), smem32 = 4 * CN * LDP * sizeof(float);
    if (!attr[dev]) {
        BAMG_CK(cudaFuncSetAttribute(k_coarse_eigvec<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem64));
        BAMG_CK(cudaFuncSetAttribute(k_coarse_eigvec<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem32));
        attr[dev] = true;
    }
    TmpBuf<double> sel(3 * (k_ev + 1), s);
    TmpBuf<int> info(8, s);
    BAMG_LAUNCH(k_coarse_eigvals, 1, CT, 0, s, n, dB, dT, k_ev, sel.get(), d_lam, d_kind, info.get());
    int h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    const bool dbg = getenv("BAMG_DEBUG") != nullptr;
    if (dbg)
        fprintf(stderr,
                "[bamg] coarse eigenvalues: n=%d QR double-shift steps=%d status=%d cycles lu+K=%d arnoldi=%d qr=%d "
                "tail=%d\n",
                n, h[3], h[2], h[4], h[5], h[6], h[7]);
    if (h[2] != 0) {
        // The FP32 QR iteration on the shift-invert Arnoldi matrix did not converge (seen on
        // birth-death chains whose coarsest eigenvalues cluster near 0 by many orders of
        // magnitude): the coarsest level then supplies the state vector alone, by inverse
        // iteration at shift 0 (the eigenvalue it belongs to is exactly 0).
        const double one_sel[3] = {0.0, 0.0, 0.0};
        const double zero = 0.0;
        const int32_t real_kind = 0;
        BAMG_CK(cudaMemcpyAsync(sel.get(), one_sel, sizeof(one_sel), cudaMemcpyHostToDevice, s));
        BAMG_CK(cudaMemcpyAsync(d_lam, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
        BAMG_CK(cudaMemcpyAsync(d_kind, &real_kind, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        h[0] = 1;
        h[1] = 1;
        if (dbg) fprintf(stderr, "[bamg] coarse eigenvalues: QR did not converge; state vector only\n");
    }
    if (h[1] > 0) {
        TmpBuf<int> cyc(2 * h[1], s);
        if (fp32_vectors)
            BAMG_LAUNCH(k_coarse_eigvec<float>, h[1], CT, smem32, s, n, dB, dT, sel.get(), d_V, d_lam, cyc.get());
        else
            BAMG_LAUNCH(k_coarse_eigvec<double>, h[1], CT, smem64, s, n, dB, dT, sel.get(), d_V, d_lam, cyc.get());
        if (dbg) {
            int hc[64] = {0};
            BAMG_CK(cudaMemcpyAsync(hc, cyc.get(), sizeof(int) * 2 * h[1], cudaMemcpyDeviceToHost, s));
            BAMG_CK(cudaStreamSynchronize(s));
            fprintf(stderr, "[bamg] coarse eigenvectors (%s): %d blocks, cycles lu=%d iterate=%d\n",
                    fp32_vectors ? "fp32" : "fp64", h[1], hc[0], hc[1]);
        }
    }
    return h[0];
}

// ---------------------------------------------------------------- minimal-norm inverse
// B has rank n-1 with left null vector 1.  y = its right null vector (two steps of
// inverse iteration on the LU of B with a pivot floor); with z = 1/sqrt(n) the bordered
// matrix M = B + z y^T is nonsingular and B^+ = M^{-1} (I - z z^T): M w = (I - z z^T) b
// forces y^T w = 0, so w is the solution of B w = (I - z z^T) b orthogonal to null(B).
// Every block factors B and M (the factorisations are identical) and solves its own
// PINV_COLS columns of (I - z z^T).  Arithmetic F: FP64, or FP32 for the mixed-precision
// V-cycle, which applies B^+ in FP32.
constexpr int PINV_COLS = 8;
template <typename F>
__global__ void __launch_bounds__(CT) k_coarse_pinv(int n, const double* __restrict__ Bg, double* __restrict__ Pg,
                                                    int* __restrict__ info) {
    pdl_begin();
    __shared__ F A[CN * LDP];
    __shared__ F R[CN * PINV_COLS];
    __shared__ F y[CN], dinv[CN], red[CT / 32];
    __shared__ int perm[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const long long c_start = clock64();
    const int c0 = blockIdx.x * PINV_COLS, mc = min(PINV_COLS, n - c0);
    F mx = F(0);
    for (int idx = tid; idx < n * n; idx += CT) {
        const int r = idx / n, c = idx - r * n;
        const F b = (F)Bg[idx];
        A[r * LDP + c] = b;
        mx = mx > absv(b) ? mx : absv(b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const F t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = mx > t ? mx : t;
    }
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    mx = F(0);
    for (int q = 0; q < CT / 32; ++q) mx = mx > red[q] ? mx : red[q];
    const F rel_floor = sizeof(F) == 8 ? F(1e-14) : F(1e-6f);
    __shared__ int src[CN];
    blu_factor<F>(A, n, perm, dinv, rel_floor * (mx > F(0) ? mx : F(1)));
    if (tid == 0) lu_row_sources(n, perm, src);
    if (tid < n) y[tid] = F(1);
    __syncthreads();
    if (wid == 0) {  // two steps of inverse iteration, in one warp
        for (int it = 0; it < 2; ++it) {
            warp_lu_solve<F>(A, n, src, dinv, y, 1);
            double nn = 0.0;
            for (int r = lane; r < n; r += 32) nn += (double)y[r] * y[r];
            const F sc = (F)(1.0 / sqrt(warp_sum(nn)));
            for (int r = lane; r < n; r += 32) y[r] *= sc;
            __syncwarp();
        }
    }
    __syncthreads();
    const F zs = (F)(1.0 / sqrt((double)n)), ninv = (F)(1.0 / (double)n);
    for (int idx = tid; idx < n * n; idx += CT) {
        const int r = idx / n, c = idx - r * n;
        A[r * LDP + c] = (F)Bg[idx] + zs * y[c];
    }
    for (int idx = tid; idx < n * mc; idx += CT) {
        const int r = idx / mc, c = idx - r * mc;
        R[r * mc + c] = (r == c0 + c ? F(1) : F(0)) - ninv;
    }
    __syncthreads();
    const long long c_null = clock64();
    blu_factor<F>(A, n, perm, dinv, pivot_tiny<F>());
    if (tid == 0) lu_row_sources(n, perm, src);
    __syncthreads();
    const long long c_lu = clock64();
    if (wid < mc) warp_lu_solve<F>(A, n, src, dinv, R + wid, mc);  // one right-hand side per warp
    __syncthreads();
    const long long c_solve = clock64();
    int bad = 0;
    for (int idx = tid; idx < n * mc; idx += CT) {
        const int r = idx / mc, c = idx - r * mc;
        const double v = (double)R[idx];
        if (!(fabs(v) < INFINITY)) bad = 1;
        Pg[r * n + c0 + c] = v;
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        info[4 * blockIdx.x] = bad;
        info[4 * blockIdx.x + 1] = (int)(c_null - c_start);  // diagnostics: cycles per phase
        info[4 * blockIdx.x + 2] = (int)(c_lu - c_null);
        info[4 * blockIdx.x + 3] = (int)(c_solve - c_lu);
    }
}

int coarse_pinv(int n, const double* dB, double* dP, bool fp32, cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_pinv: coarsest order must be 1..64");
    const int nb = (n + PINV_COLS - 1) / PINV_COLS;
    TmpBuf<int> info(4 * nb, s);
    if (fp32)
        BAMG_LAUNCH(k_coarse_pinv<float>, nb, CT, 0, s, n, dB, dP, info.get());
    else
        BAMG_LAUNCH(k_coarse_pinv<double>, nb, CT, 0, s, n, dB, dP, info.get());
    int h[4 * (CN / PINV_COLS)] = {0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(int) * 4 * nb, cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    if (getenv("BAMG_DEBUG"))
        fprintf(stderr, "[bamg] coarse pinv (%s): n=%d blocks=%d cycles null=%d lu=%d solve=%d\n", fp32 ? "fp32" : "fp64",
                n, nb, h[1], h[2], h[3]);
    for (int b = 0; b < nb; ++b)
        if (h[4 * b]) return BAMG_ENUMERIC;
    return 0;
}

}  // namespace bamg
