// Coarsest level (Algorithm 3, first branch; Section 4.2): the eigenpairs of
// B_L x = lambda T_L x with the smallest |lambda|, and the minimal-norm inverse B_L^+.
// Order n <= 64, one thread block per task, matrices in shared memory.
//
// Eigenpairs: the eigenvalues of T^{-1} B from an LU solve, a Householder reduction to
// Hessenberg form and the implicit double-shift QR iteration (Francis; Golub & Van Loan,
// Matrix Computations, Sec. 7.5), all in FP32 because they only serve as shifts; then,
// per selected eigenvalue, FP64 inverse iteration in complex arithmetic on the pencil
// (B - sigma T) and a Rayleigh-type quotient give the eigenvector and the eigenvalue to
// FP64 accuracy.  B^+: a bordered FP64 LU solve.
#include <cfloat>
#include <cstdio>
#include <cstdlib>

#include "kernels.cuh"

namespace bamg {

constexpr int CN = 64;
constexpr int LDP = CN + 1;  // padded row stride of shared matrices (no bank conflicts on columns)
constexpr int CT = 256;  // threads per block

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------- block-parallel real LU
// In-place LU with partial pivoting of the n x n row-major A (shared memory); perm[k] =
// pivot row of step k.  Pivots smaller than floorv in magnitude become +-floorv.
__device__ void blu_factor(double* A, int n, int* perm, double floorv) {
    const int tid = threadIdx.x;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int br = k;
            for (int r = k + tid; r < n; r += 32) {
                const double v = fabs(A[r * LDP + k]);
                if (v > best) {
                    best = v;
                    br = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) perm[k] = br;
        }
        __syncthreads();
        const int br = perm[k];
        if (br != k)
            for (int c = tid; c < n; c += blockDim.x) {
                const double t = A[k * LDP + c];
                A[k * LDP + c] = A[br * LDP + c];
                A[br * LDP + c] = t;
            }
        __syncthreads();
        double p = A[k * LDP + k];
        if (fabs(p) < floorv) p = p >= 0.0 ? floorv : -floorv;
        for (int r = k + 1 + tid; r < n; r += blockDim.x) A[r * LDP + k] /= p;
        __syncthreads();
        if (tid == 0) A[k * LDP + k] = p;
        const int m = n - k - 1;
        for (int idx = tid; idx < m * m; idx += blockDim.x) {
            const int r = k + 1 + idx / m, c = k + 1 + idx % m;
            A[r * LDP + c] -= A[r * LDP + k] * A[k * LDP + c];
        }
        __syncthreads();
    }
}

// Solves A X = R for the m right-hand sides stored row-major (n x m) in R, in place.
__device__ void blu_solve(const double* A, int n, const int* perm, double* R, int m) {
    const int tid = threadIdx.x;
    for (int k = 0; k < n; ++k) {
        const int pk = perm[k];
        if (pk != k) {
            for (int c = tid; c < m; c += blockDim.x) {
                const double t = R[k * m + c];
                R[k * m + c] = R[pk * m + c];
                R[pk * m + c] = t;
            }
            __syncthreads();
        }
    }
    for (int q = 0; q < n; ++q) {
        const int rows = n - q - 1;
        for (int idx = tid; idx < rows * m; idx += blockDim.x) {
            const int r = q + 1 + idx / m, c = idx % m;
            R[r * m + c] -= A[r * LDP + q] * R[q * m + c];
        }
        __syncthreads();
    }
    for (int q = n - 1; q >= 0; --q) {
        for (int c = tid; c < m; c += blockDim.x) R[q * m + c] /= A[q * LDP + q];
        __syncthreads();
        for (int idx = tid; idx < q * m; idx += blockDim.x) {
            const int r = idx / m, c = idx % m;
            R[r * m + c] -= A[r * LDP + q] * R[q * m + c];
        }
        __syncthreads();
    }
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

// FP32 LU with partial pivoting (block-parallel) and the solve T M = B for n right-hand
// sides, used only to obtain shifts.
__device__ void blu_factor_f32(float* A, int n, int* perm) {
    const int tid = threadIdx.x;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            float best = -1.f;
            int br = k;
            for (int r = k + tid; r < n; r += 32) {
                const float v = fabsf(A[r * LDP + k]);
                if (v > best) {
                    best = v;
                    br = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) perm[k] = br;
        }
        __syncthreads();
        const int br = perm[k];
        if (br != k)
            for (int c = tid; c < n; c += blockDim.x) {
                const float t = A[k * LDP + c];
                A[k * LDP + c] = A[br * LDP + c];
                A[br * LDP + c] = t;
            }
        __syncthreads();
        float p = A[k * LDP + k];
        if (fabsf(p) < 1e-30f) p = p >= 0.f ? 1e-30f : -1e-30f;
        const float pinv = 1.f / p;
        for (int r = k + 1 + tid; r < n; r += blockDim.x) A[r * LDP + k] *= pinv;
        __syncthreads();
        if (tid == 0) A[k * LDP + k] = p;
        const int m = n - k - 1;
        for (int idx = tid; idx < m * m; idx += blockDim.x) {
            const int r = k + 1 + idx / m, c = k + 1 + idx % m;
            A[r * LDP + c] -= A[r * LDP + k] * A[k * LDP + c];
        }
        __syncthreads();
    }
}


// Kernel 1: estimates of the eigenvalues of B x = lambda T x closest to zero, in FP32
// (they serve only as shifts): shift-and-invert Arnoldi on K = (B - sigma T)^{-1} T with
// sigma = -1e-4 max|B| (K's dominant eigenvalues theta = 1/(lambda - sigma) belong to
// the lambda of smallest modulus), KRY steps with classical Gram-Schmidt applied twice,
// the eigenvalues of the small Hessenberg matrix by the Francis QR iteration, then
// lambda = sigma + 1/theta.  Selection: eigenvalues with Im >= 0 (a complex pair is
// represented by its member with positive imaginary part) in order of |lambda|; a real
// one takes one vector column, a pair two (Re v, Im v), until k_ev columns are filled.
// sel[3q + {0,1,2}] = (Re, Im, first column); info = {columns, selected, status, steps}.
constexpr int KRY = 32;
__global__ void __launch_bounds__(CT) k_coarse_eigvals(int n, const double* __restrict__ Bg,
                                                       const double* __restrict__ Tg, int k_ev,
                                                       double* __restrict__ sel, double* __restrict__ lam,
                                                       int32_t* __restrict__ kind, int* __restrict__ info) {
    __shared__ float A[CN * LDP], Tm[CN * LDP];
    __shared__ float Vk[(KRY + 1) * CN];
    __shared__ float w[CN], hcol[KRY + 1];
    __shared__ int perm[CN];
    __shared__ float wr[CN], wi[CN], red[CT / 32];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    // sigma from the largest entry of B
    float mx = 0.f;
    for (int idx = tid; idx < n * n; idx += blockDim.x) mx = fmaxf(mx, fabsf((float)Bg[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    mx = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) mx = fmaxf(mx, red[q]);
    const float sigma = -1e-4f * fmaxf(mx, 1e-30f);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        const float t = (float)Tg[idx];
        Tm[r * LDP + c] = t;
        A[r * LDP + c] = (float)Bg[idx] - sigma * t;
    }
    __syncthreads();
    blu_factor_f32(A, n, perm);
    const int kd = n < KRY ? n : KRY;
    if (tid >= 32) return;  // the Arnoldi process runs in one warp
    // v_0: fixed generic start, unit norm
    {
        float nn = 0.f;
        for (int r = lane; r < n; r += 32) {
            const float v = 1.f + (float)r / (float)n;
            Vk[r] = v;
            nn += v * v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        nn = rsqrtf(nn);
        for (int r = lane; r < n; r += 32) Vk[r] *= nn;
        __syncwarp();
    }
    __shared__ float Hs[KRY * KRY];
    for (int idx = lane; idx < KRY * KRY; idx += 32) Hs[idx] = 0.f;
    int kk = kd;
    for (int k = 0; k < kd; ++k) {
        const float* vk = Vk + k * CN;
        // w = T v_k
        for (int r = lane; r < n; r += 32) {
            float sacc = 0.f;
            for (int c = 0; c < n; ++c) sacc += Tm[r * LDP + c] * vk[c];
            w[r] = sacc;
        }
        __syncwarp();
        // w <- (B - sigma T)^{-1} w
        for (int q = 0; q < n; ++q) {
            const int pq = perm[q];
            if (pq != q && lane == 0) {
                const float t = w[q];
                w[q] = w[pq];
                w[pq] = t;
            }
            __syncwarp();
        }
        for (int q = 0; q < n; ++q) {
            const float yq = w[q];
            for (int r = q + 1 + lane; r < n; r += 32) w[r] -= A[r * LDP + q] * yq;
            __syncwarp();
        }
        for (int q = n - 1; q >= 0; --q) {
            if (lane == 0) w[q] /= A[q * LDP + q];
            __syncwarp();
            const float yq = w[q];
            for (int r = lane; r < q; r += 32) w[r] -= A[r * LDP + q] * yq;
            __syncwarp();
        }
        // classical Gram-Schmidt, twice
        for (int q = 0; q <= k; ++q) hcol[q] = 0.f;
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
            for (int q = 0; q <= k; ++q) {
                float d = 0.f;
                for (int r = lane; r < n; r += 32) d += Vk[q * CN + r] * w[r];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                for (int r = lane; r < n; r += 32) w[r] -= d * Vk[q * CN + r];
                if (lane == 0) hcol[q] += d;
                __syncwarp();
            }
        }
        float nn = 0.f;
        for (int r = lane; r < n; r += 32) nn += w[r] * w[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
        nn = sqrtf(nn);
        for (int q = lane; q <= k; q += 32) Hs[q * KRY + k] = hcol[q];
        if (k + 1 < kd && lane == 0) Hs[(k + 1) * KRY + k] = nn;
        __syncwarp();
        if (!(nn > 1e-6f * fabsf(hcol[0]) + 1e-30f)) {  // invariant subspace found
            kk = k + 1;
            break;
        }
        if (k + 1 < kd)
            for (int r = lane; r < n; r += 32) Vk[(k + 1) * CN + r] = w[r] / nn;
        __syncwarp();
    }
    // eigenvalues of the kk x kk Hessenberg matrix (stored with the padded row stride)
    for (int idx = lane; idx < kk * kk; idx += 32) {
        const int r = idx / kk, c = idx % kk;
        Tm[r * LDP + c] = Hs[r * KRY + c];
    }
    __syncwarp();
    int steps = 0;
    const int st = hqr_f32(Tm, kk, wr, wi, &steps);
    __syncwarp();
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
    }
}

// ---------------------------------------------------------------- complex inverse iteration
// Kernel 2, one block per selected eigenvalue: LU of the pencil (B - sigma T) in
// complex FP64 with sigma the FP32 estimate; four steps of inverse iteration
// v <- (B - sigma T)^{-1} T v from a fixed positive start; the Rayleigh-type quotient
// lambda = v^H B v / v^H T v (Algorithm 3's update, in complex form); and the phase that
// makes <w, v> real and positive (w_i = i + 1) with unit 2-norm.
__global__ void __launch_bounds__(CT) k_coarse_eigvec(int n, const double* __restrict__ Bg,
                                                      const double* __restrict__ Tg, const double* __restrict__ sel,
                                                      double* __restrict__ V, double* __restrict__ lam) {
    extern __shared__ double sm[];
    double* Ar = sm;
    double* Ai = sm + CN * LDP;
    __shared__ double vr[CN], vi[CN], tr[CN], ti[CN], red[4 * (CT / 32)];
    __shared__ int perm[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const double sr = sel[3 * blockIdx.x], si = sel[3 * blockIdx.x + 1];
    const int col = (int)sel[3 * blockIdx.x + 2];
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const double t = Tg[idx];
        Ar[(idx / n) * LDP + idx % n] = Bg[idx] - sr * t;
        Ai[(idx / n) * LDP + idx % n] = -si * t;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int br = k;
            for (int r = k + tid; r < n; r += 32) {
                const double m = fabs(Ar[r * LDP + k]) + fabs(Ai[r * LDP + k]);
                if (m > best) {
                    best = m;
                    br = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ob > best || (ob == best && orr < br)) {
                    best = ob;
                    br = orr;
                }
            }
            if (tid == 0) perm[k] = br;
        }
        __syncthreads();
        const int br = perm[k];
        if (br != k)
            for (int c = tid; c < n; c += blockDim.x) {
                double t = Ar[k * LDP + c];
                Ar[k * LDP + c] = Ar[br * LDP + c];
                Ar[br * LDP + c] = t;
                t = Ai[k * LDP + c];
                Ai[k * LDP + c] = Ai[br * LDP + c];
                Ai[br * LDP + c] = t;
            }
        __syncthreads();
        double pr = Ar[k * LDP + k], pi = Ai[k * LDP + k];
        if (fabs(pr) + fabs(pi) < 1e-300) {
            pr = 1e-300;
            pi = 0.0;
        }
        const double inv = 1.0 / (pr * pr + pi * pi);
        const double qr_ = pr * inv, qi_ = -pi * inv;  // 1 / pivot
        for (int r = k + 1 + tid; r < n; r += blockDim.x) {
            const double ar = Ar[r * LDP + k], ai = Ai[r * LDP + k];
            Ar[r * LDP + k] = ar * qr_ - ai * qi_;
            Ai[r * LDP + k] = ar * qi_ + ai * qr_;
        }
        __syncthreads();
        if (tid == 0) {
            Ar[k * LDP + k] = pr;
            Ai[k * LDP + k] = pi;
        }
        const int m = n - k - 1;
        for (int idx = tid; idx < m * m; idx += blockDim.x) {
            const int r = k + 1 + idx / m, c = k + 1 + idx % m;
            const double lr = Ar[r * LDP + k], li = Ai[r * LDP + k];
            const double ur = Ar[k * LDP + c], ui = Ai[k * LDP + c];
            Ar[r * LDP + c] -= lr * ur - li * ui;
            Ai[r * LDP + c] -= lr * ui + li * ur;
        }
        __syncthreads();
    }
    for (int r = tid; r < n; r += blockDim.x) {
        vr[r] = 1.0 + (double)r / (double)n;
        vi[r] = 0.0;
    }
    __syncthreads();
    for (int it = 0; it < 4; ++it) {
        // t = T v (rows in parallel)
        for (int r = tid; r < n; r += blockDim.x) {
            double a = 0.0, b = 0.0;
            for (int c = 0; c < n; ++c) {
                const double t = Tg[r * n + c];
                a += t * vr[c];
                b += t * vi[c];
            }
            tr[r] = a;
            ti[r] = b;
        }
        __syncthreads();
        if (tid < 32) {  // one warp: column-oriented substitutions on t
            for (int k = 0; k < n; ++k) {
                const int pk = perm[k];
                if (pk != k && lane == 0) {
                    double t = tr[k];
                    tr[k] = tr[pk];
                    tr[pk] = t;
                    t = ti[k];
                    ti[k] = ti[pk];
                    ti[pk] = t;
                }
                __syncwarp();
            }
            for (int q = 0; q < n; ++q) {
                const double yr = tr[q], yi = ti[q];
                for (int r = q + 1 + lane; r < n; r += 32) {
                    tr[r] -= Ar[r * LDP + q] * yr - Ai[r * LDP + q] * yi;
                    ti[r] -= Ar[r * LDP + q] * yi + Ai[r * LDP + q] * yr;
                }
                __syncwarp();
            }
            for (int q = n - 1; q >= 0; --q) {
                if (lane == 0) {
                    const double ur = Ar[q * LDP + q], ui = Ai[q * LDP + q];
                    const double d = 1.0 / (ur * ur + ui * ui);
                    const double a = tr[q], b = ti[q];
                    tr[q] = (a * ur + b * ui) * d;
                    ti[q] = (b * ur - a * ui) * d;
                }
                __syncwarp();
                const double yr = tr[q], yi = ti[q];
                for (int r = lane; r < q; r += 32) {
                    tr[r] -= Ar[r * LDP + q] * yr - Ai[r * LDP + q] * yi;
                    ti[r] -= Ar[r * LDP + q] * yi + Ai[r * LDP + q] * yr;
                }
                __syncwarp();
            }
            double nn = 0.0;
            for (int r = lane; r < n; r += 32) nn += tr[r] * tr[r] + ti[r] * ti[r];
            nn = 1.0 / sqrt(warp_sum(nn));
            for (int r = lane; r < n; r += 32) {
                vr[r] = tr[r] * nn;
                vi[r] = ti[r] * nn;
            }
            __syncwarp();
        }
        __syncthreads();
    }
    // lambda = v^H B v / v^H T v
    double br_ = 0.0, bi_ = 0.0, tr_ = 0.0, ti_ = 0.0;
    for (int r = tid; r < n; r += blockDim.x) {
        double wbr = 0.0, wbi = 0.0, wtr = 0.0, wti = 0.0;
        for (int c = 0; c < n; ++c) {
            const double b = Bg[r * n + c], t = Tg[r * n + c];
            wbr += b * vr[c];
            wbi += b * vi[c];
            wtr += t * vr[c];
            wti += t * vi[c];
        }
        br_ += vr[r] * wbr + vi[r] * wbi;
        bi_ += vr[r] * wbi - vi[r] * wbr;
        tr_ += vr[r] * wtr + vi[r] * wti;
        ti_ += vr[r] * wti - vi[r] * wtr;
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
    for (int r = lane; r < n; r += 32) {
        const double a = vr[r] * cr - vi[r] * ci, b = vr[r] * ci + vi[r] * cr;
        vr[r] = a;
        vi[r] = b;
        nn += a * a + b * b;
    }
    nn = 1.0 / sqrt(warp_sum(nn));
    for (int r = lane; r < n; r += 32) {
        V[(int64_t)col * n + r] = vr[r] * nn;
        if (si != 0.0) V[(int64_t)(col + 1) * n + r] = vi[r] * nn;
    }
    if (lane == 0) {
        double nbr = 0.0, nbi = 0.0, ntr = 0.0, nti = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            nbr += red[4 * w];
            nbi += red[4 * w + 1];
            ntr += red[4 * w + 2];
            nti += red[4 * w + 3];
        }
        // Re of (nbr + i nbi) / (ntr + i nti)
        double lre = (nbr * ntr + nbi * nti) / (ntr * ntr + nti * nti);
        if (col == 0) lre = 0.0;  // the state vector's eigenvalue is exactly zero
        lam[col] = lre;
        if (si != 0.0) lam[col + 1] = lre;
    }
}

int coarse_eig(int n, const double* dB, const double* dT, int k_ev, double* d_lam, double* d_V, int32_t* d_kind,
               cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_eig: coarsest order must be 1..64");
    BAMG_REQUIRE(k_ev >= 1 && k_ev <= 16, BAMG_EINVAL, "coarse_eig: 1 <= k_ev <= 16");
    static bool attr = false;
    const size_t smem = 2 * CN * LDP * sizeof(double);
    if (!attr) {
        BAMG_CK(cudaFuncSetAttribute(k_coarse_eigvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    TmpBuf<double> sel(3 * (k_ev + 1), s);
    TmpBuf<int> info(4, s);
    BAMG_LAUNCH(k_coarse_eigvals, 1, CT, 0, s, n, dB, dT, k_ev, sel.get(), d_lam, d_kind, info.get());
    int h[4] = {0, 0, 0, 0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    if (getenv("BAMG_DEBUG")) fprintf(stderr, "[bamg] coarse QR: n=%d double-shift steps=%d status=%d\n", n, h[3], h[2]);
    if (h[2] != 0) return BAMG_ENUMERIC;
    if (h[1] > 0) BAMG_LAUNCH(k_coarse_eigvec, h[1], CT, smem, s, n, dB, dT, sel.get(), d_V, d_lam);
    return h[0];
}

// ---------------------------------------------------------------- minimal-norm inverse
// B has rank n-1 with left null vector 1.  y = its right null vector (two steps of
// inverse iteration on the LU of B with a pivot floor); with z = 1/sqrt(n) the bordered
// matrix M = B + z y^T is nonsingular and B^+ = M^{-1} (I - z z^T): M w = (I - z z^T) b
// forces y^T w = 0, so w is the solution of B w = (I - z z^T) b orthogonal to null(B).
__global__ void __launch_bounds__(CT) k_coarse_pinv(int n, const double* __restrict__ Bg, double* __restrict__ Pg,
                                                    int* __restrict__ info) {
    extern __shared__ double sm[];
    double* A = sm;
    double* R = sm + CN * LDP;
    __shared__ double y[CN], red[CT / 32];
    __shared__ int perm[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    double mx = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        A[(idx / n) * LDP + idx % n] = Bg[idx];
        mx = fmax(mx, fabs(Bg[idx]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    __syncthreads();
    blu_factor(A, n, perm, 1e-14 * fmax(mx, 1e-300));
    for (int r = tid; r < n; r += blockDim.x) R[r] = 1.0;
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        blu_solve(A, n, perm, R, 1);
        if (tid < 32) {
            double nn = 0.0;
            for (int r = lane; r < n; r += 32) nn += R[r] * R[r];
            nn = sqrt(warp_sum(nn));
            for (int r = lane; r < n; r += 32) R[r] /= nn;
        }
        __syncthreads();
    }
    for (int r = tid; r < n; r += blockDim.x) y[r] = R[r];
    __syncthreads();
    const double zs = 1.0 / sqrt((double)n);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx / n, c = idx % n;
        A[r * LDP + c] = Bg[idx] + zs * y[c];
        R[idx] = (r == c ? 1.0 : 0.0) - 1.0 / (double)n;
    }
    __syncthreads();
    blu_factor(A, n, perm, 1e-300);
    blu_solve(A, n, perm, R, n);
    int bad = 0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const double v = R[idx];
        if (!(fabs(v) < INFINITY)) bad = 1;
        Pg[idx] = v;
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) info[0] = bad;
}

int coarse_pinv(int n, const double* dB, double* dP, cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_pinv: coarsest order must be 1..64");
    static bool attr = false;
    const size_t smem = 2 * CN * LDP * sizeof(double);
    if (!attr) {
        BAMG_CK(cudaFuncSetAttribute(k_coarse_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    TmpBuf<int> info(1, s);
    BAMG_LAUNCH(k_coarse_pinv, 1, CT, smem, s, n, dB, dP, info.get());
    int h = 0;
    BAMG_CK(cudaMemcpyAsync(&h, info.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    return h ? BAMG_ENUMERIC : 0;
}

}  // namespace bamg
