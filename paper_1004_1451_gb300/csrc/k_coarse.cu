// Coarsest level (Algorithm 3, first branch; Section 4.2): the eigenpairs of
// B_L x = lambda T_L x with the smallest |lambda|, and the minimal-norm inverse B_L^+.
// Order n <= 64, matrices in shared memory, 256 threads per block.
//
// Eigenvalues (FP32; they only serve as shifts): shift-and-invert Arnoldi on the explicit
// operator K = (B - sigma T)^{-1} T, then the Francis double-shift QR iteration on the
// small Hessenberg matrix (Golub & Van Loan, Matrix Computations, Sec. 7.5).
// Eigenvectors, one block per selected eigenvalue: inverse iteration in complex
// arithmetic on the pencil (B - sigma T) and a Rayleigh-type quotient, in FP64 (or in
// FP32 for the mixed-precision setup, through the explicit (B - sigma T)^{-1} T).  B^+: one LU of the bordered matrix B + z z^T
// (z = 1/sqrt(n)), the right-hand sides split over several blocks.  Factorisations use the
// whole block (rows in place, the pivot found by a warp reduction); triangular solves run
// in single warps (shuffles, no block barriers).
#include <cfloat>
#include <cstdio>
#include <cstdlib>

#include <atomic>
#include <type_traits>

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

// ---------------------------------------------------------------- block LU, rows in place
// Partial pivoting with the rows left where they are: step k takes as pivot the not yet
// pivoted row of largest magnitude in column k and records it as src[k]; the other
// unpivoted rows get their multiplier in column k and update their columns > k.  On return
// row src[i] of A holds pivot row i: multipliers left of column i, the upper factor times
// dinv[i] (= 1 / u_ii) right of it, so a solve reads equation i from row src[i] (and its
// right-hand side entry b[src[i]]).  n <= 64, A in shared memory with row stride LDP = 65.
//
// Per step: warp 0 finds the pivot with one warp reduction over a 32-bit key (the
// magnitude's float bits with the low 6 mantissa bits replaced by 63 - row: magnitudes
// within 2^-17 count as equal and the lowest row wins; a NaN counts as infinite, so a valid
// row is always taken and the NaN reaches the factors, where the callers' finiteness checks
// see it); then all CT threads update, 4 per row, consecutive threads on consecutive rows
// (a column's rows sit on distinct banks).  The multipliers of a step are parked in `mult`
// and written to their column by warp 0 in the next step, when no thread reads that column.
// Every thread of the block calls it (block barriers inside).
__device__ __forceinline__ unsigned pivot_key(float mag, int row) {
    const unsigned bits = mag == mag ? __float_as_uint(mag) : 0x7f800000u;
    return (bits & ~63u) | (unsigned)(63 - row);
}

// Real A (F = float or double); pivots below floorv in magnitude become +-floorv.
template <typename F>
__device__ void block_lu_factor(F* A, int n, int* src, F* dinv, F floorv) {
    __shared__ int step_of[CN];  // pivot step of each row, -1 while unpivoted
    __shared__ F mult[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const int r = tid & (CN - 1), q = tid >> 6;  // this thread's row and its column phase (CT = 4 CN)
    if (tid < CN) step_of[tid] = tid < n ? -1 : CN;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (wid == 0) {
            const bool ua = step_of[lane] < 0, ub = step_of[lane + 32] < 0;
            if (k > 0) {  // the previous step's multipliers into column k - 1
                if (ua) A[lane * LDP + k - 1] = mult[lane];
                if (ub) A[(lane + 32) * LDP + k - 1] = mult[lane + 32];
            }
            const unsigned ka = ua ? pivot_key((float)absv(A[lane * LDP + k]), lane) : 0u;
            const unsigned kb = ub ? pivot_key((float)absv(A[(lane + 32) * LDP + k]), lane + 32) : 0u;
            const unsigned best = __reduce_max_sync(0xffffffffu, ka > kb ? ka : kb);
            if (lane == 0) {
                const int pr = 63 - (int)(best & 63u);
                F pv = A[pr * LDP + k];
                if (absv(pv) < floorv) pv = pv >= F(0) ? floorv : -floorv;
                A[pr * LDP + k] = pv;
                src[k] = pr;
                dinv[k] = F(1) / pv;
                step_of[pr] = k;
            }
        }
        __syncthreads();
        if (step_of[r] < 0) {
            const F l = A[r * LDP + k] * dinv[k];
            if (q == 0) mult[r] = l;
            const F* prow = A + src[k] * LDP;
            F* row = A + r * LDP;
            int c = k + 1 + q;
            for (; c + 12 < n; c += 16) {  // 4 columns at once, loads before stores
                F pc[4], x[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    pc[j] = prow[c + 4 * j];
                    x[j] = row[c + 4 * j];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) row[c + 4 * j] = x[j] - l * pc[j];
            }
            for (; c < n; c += 4) row[c] -= l * prow[c];
        }
        __syncthreads();
    }
    // unit upper factor: the part of row src[i] right of column i times dinv[i]
    const int sr = step_of[r];
    if (sr < n) {
        const F d = dinv[sr];
        for (int c = sr + 1 + ((q - sr - 1) & 3); c < n; c += 4) A[r * LDP + c] *= d;
    }
    __syncthreads();
}

// 1 / (pr + i pi) without squaring (Smith's method: no overflow or underflow in FP32)
template <typename F>
__device__ __forceinline__ void cplx_recip(F pr, F pi, F& dr, F& di) {
    if (absv(pr) >= absv(pi)) {
        const F t = pi / pr, d = F(1) / (pr + pi * t);
        dr = d;
        di = -t * d;
    } else {
        const F t = pr / pi, d = F(1) / (pr * t + pi);
        dr = t * d;
        di = -d;
    }
}

// Complex A = Ar + i Ai, pivoting on |Re| + |Im|; pivots below floorv become floorv; dr + i di
// = 1 / u_ii.  Same layout and contract as block_lu_factor.
template <typename F>
__device__ void block_lu_factor_cplx(F* Ar, F* Ai, int n, int* src, F* dr, F* di, F floorv) {
    __shared__ int step_of[CN];
    __shared__ F mr[CN], mi[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const int r = tid & (CN - 1), q = tid >> 6;
    if (tid < CN) step_of[tid] = tid < n ? -1 : CN;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (wid == 0) {
            const bool ua = step_of[lane] < 0, ub = step_of[lane + 32] < 0;
            if (k > 0) {
                if (ua) {
                    Ar[lane * LDP + k - 1] = mr[lane];
                    Ai[lane * LDP + k - 1] = mi[lane];
                }
                if (ub) {
                    Ar[(lane + 32) * LDP + k - 1] = mr[lane + 32];
                    Ai[(lane + 32) * LDP + k - 1] = mi[lane + 32];
                }
            }
            const int ia = lane * LDP + k, ib = (lane + 32) * LDP + k;
            const unsigned ka = ua ? pivot_key((float)(absv(Ar[ia]) + absv(Ai[ia])), lane) : 0u;
            const unsigned kb = ub ? pivot_key((float)(absv(Ar[ib]) + absv(Ai[ib])), lane + 32) : 0u;
            const unsigned best = __reduce_max_sync(0xffffffffu, ka > kb ? ka : kb);
            if (lane == 0) {
                const int pr = 63 - (int)(best & 63u);
                F ppr = Ar[pr * LDP + k], ppi = Ai[pr * LDP + k];
                if (absv(ppr) + absv(ppi) < floorv) {
                    ppr = floorv;
                    ppi = F(0);
                }
                Ar[pr * LDP + k] = ppr;
                Ai[pr * LDP + k] = ppi;
                F qr, qi;
                cplx_recip(ppr, ppi, qr, qi);
                src[k] = pr;
                dr[k] = qr;
                di[k] = qi;
                step_of[pr] = k;
            }
        }
        __syncthreads();
        if (step_of[r] < 0) {
            const F ar = Ar[r * LDP + k], ai = Ai[r * LDP + k], qr = dr[k], qi = di[k];
            const F lr = ar * qr - ai * qi, li = ar * qi + ai * qr;
            if (q == 0) {
                mr[r] = lr;
                mi[r] = li;
            }
            const F* pur = Ar + src[k] * LDP;
            const F* pui = Ai + src[k] * LDP;
            F* xr_ = Ar + r * LDP;
            F* xi_ = Ai + r * LDP;
            int c = k + 1 + q;
            for (; c + 4 < n; c += 8) {  // 2 columns at once, loads before stores
                const F ur0 = pur[c], ui0 = pui[c], ur1 = pur[c + 4], ui1 = pui[c + 4];
                const F x0 = xr_[c], y0 = xi_[c], x1 = xr_[c + 4], y1 = xi_[c + 4];
                xr_[c] = x0 - (lr * ur0 - li * ui0);
                xi_[c] = y0 - (lr * ui0 + li * ur0);
                xr_[c + 4] = x1 - (lr * ur1 - li * ui1);
                xi_[c + 4] = y1 - (lr * ui1 + li * ur1);
            }
            for (; c < n; c += 4) {
                const F ur = pur[c], ui = pui[c], x = xr_[c], y = xi_[c];
                xr_[c] = x - (lr * ur - li * ui);
                xi_[c] = y - (lr * ui + li * ur);
            }
        }
        __syncthreads();
    }
    const int sr = step_of[r];
    if (sr < n) {
        const F qr = dr[sr], qi = di[sr];
        for (int c = sr + 1 + ((q - sr - 1) & 3); c < n; c += 4) {
            const F ur = Ar[r * LDP + c], ui = Ai[r * LDP + c];
            Ar[r * LDP + c] = ur * qr - ui * qi;
            Ai[r * LDP + c] = ur * qi + ui * qr;
        }
    }
    __syncthreads();
}

// One warp solves A X = R for the NC columns c0 .. c0 + NC - 1 (those < m) of the
// row-major R (row stride ldr) at once, with the factors of block_lu_factor (equation i in
// row src[i] of A and of R): the independent columns hide the latency of the shuffles.
// Forward and back substitution eliminate one column of L (of U) at a time, as in the
// plain algorithm; lane l holds the unknowns l and l + 32.
template <typename F, int NC>
__device__ void warp_lu_solve_cols(const F* A, int n, const int* src, const F* dinv, F* R, int ldr, int c0, int m) {
    const int lane = lane_id();
    const int r0 = lane < n ? src[lane] : 0, r1 = lane + 32 < n ? src[lane + 32] : 0;
    F x0[NC], x1[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const bool cj = c0 + j < m;
        x0[j] = lane < n && cj ? R[r0 * ldr + c0 + j] : F(0);
        x1[j] = lane + 32 < n && cj ? R[r1 * ldr + c0 + j] : F(0);
    }
    __syncwarp();
    for (int q = 0; q + 1 < n; ++q) {  // unit lower
        const bool a0 = lane > q && lane < n, a1 = lane + 32 > q && lane + 32 < n;
        const F l0 = a0 ? A[r0 * LDP + q] : F(0), l1 = a1 ? A[r1 * LDP + q] : F(0);
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
        const F u0 = a0 ? A[r0 * LDP + q] : F(0), u1 = a1 ? A[r1 * LDP + q] : F(0);
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

// One warp solves A x = b for one right-hand side b (stride ldb), in place, with the factors
// of block_lu_factor.  The warp's lanes must all call it.
template <typename F>
__device__ void warp_lu_solve(const F* A, int n, const int* src, const F* dinv, F* b, int ldb) {
    warp_lu_solve_cols<F, 1>(A, n, src, dinv, b, ldb, 0, 1);
}

// One warp solves (Ar + i Ai) X = R for the NC real right-hand sides c0 .. c0 + NC - 1 (those
// < n) of R (row-major, stride LDP), with the factors of block_lu_factor_cplx (equation i in
// row src[i]); X = Xr + i Xi (stride LDP).  The NC independent columns share each step's
// shuffle latency.  Entries of L (U) beyond a lane's range are taken as zero, which leaves
// its unknowns exactly unchanged.
template <typename F, int NC>
__device__ void warp_lu_solve_cols_cplx(const F* Ar, const F* Ai, int n, const int* src, const F* dr, const F* di,
                                        const F* R, F* Xr, F* Xi, int c0) {
    const int lane = lane_id();
    const bool v0 = lane < n, v1 = lane + 32 < n;
    const int r0 = v0 ? src[lane] : 0, r1 = v1 ? src[lane + 32] : 0;
    F ar[NC], ai[NC], br[NC], bi[NC];  // the unknowns lane (a) and lane + 32 (b) of each column
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const bool cj = c0 + j < n;
        ar[j] = v0 && cj ? R[r0 * LDP + c0 + j] : F(0);
        br[j] = v1 && cj ? R[r1 * LDP + c0 + j] : F(0);
        ai[j] = bi[j] = F(0);
    }
    __syncwarp();
    for (int q = 0; q + 1 < n; ++q) {  // unit lower
        const bool a0 = v0 && lane > q, a1 = v1 && lane + 32 > q;
        const F l0r = a0 ? Ar[r0 * LDP + q] : F(0), l0i = a0 ? Ai[r0 * LDP + q] : F(0);
        const F l1r = a1 ? Ar[r1 * LDP + q] : F(0), l1i = a1 ? Ai[r1 * LDP + q] : F(0);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F yr = __shfl_sync(0xffffffffu, q < 32 ? ar[j] : br[j], q & 31);
            const F yi = __shfl_sync(0xffffffffu, q < 32 ? ai[j] : bi[j], q & 31);
            ar[j] -= l0r * yr - l0i * yi;
            ai[j] -= l0r * yi + l0i * yr;
            br[j] -= l1r * yr - l1i * yi;
            bi[j] -= l1r * yi + l1i * yr;
        }
    }
    {
        const F d0r = v0 ? dr[lane] : F(0), d0i = v0 ? di[lane] : F(0);
        const F d1r = v1 ? dr[lane + 32] : F(0), d1i = v1 ? di[lane + 32] : F(0);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F a = ar[j], b = ai[j], c = br[j], d = bi[j];
            ar[j] = a * d0r - b * d0i;
            ai[j] = a * d0i + b * d0r;
            br[j] = c * d1r - d * d1i;
            bi[j] = c * d1i + d * d1r;
        }
    }
    for (int q = n - 1; q > 0; --q) {  // unit upper
        const bool a0 = v0 && lane < q, a1 = v1 && lane + 32 < q;
        const F u0r = a0 ? Ar[r0 * LDP + q] : F(0), u0i = a0 ? Ai[r0 * LDP + q] : F(0);
        const F u1r = a1 ? Ar[r1 * LDP + q] : F(0), u1i = a1 ? Ai[r1 * LDP + q] : F(0);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const F yr = __shfl_sync(0xffffffffu, q < 32 ? ar[j] : br[j], q & 31);
            const F yi = __shfl_sync(0xffffffffu, q < 32 ? ai[j] : bi[j], q & 31);
            ar[j] -= u0r * yr - u0i * yi;
            ai[j] -= u0r * yi + u0i * yr;
            br[j] -= u1r * yr - u1i * yi;
            bi[j] -= u1r * yi + u1i * yr;
        }
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (c0 + j >= n) continue;
        if (v0) {
            Xr[lane * LDP + c0 + j] = ar[j];
            Xi[lane * LDP + c0 + j] = ai[j];
        }
        if (v1) {
            Xr[(lane + 32) * LDP + c0 + j] = br[j];
            Xi[(lane + 32) * LDP + c0 + j] = bi[j];
        }
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

// Kernel 1: estimates of the eigenvalues of B x = lambda T x closest to zero, in FP32
// (they serve only as shifts).  sigma = -1e-4 max|B|; K = (B - sigma T)^{-1} T is formed
// explicitly (its dominant eigenvalues theta = 1 / (lambda - sigma) belong to the lambda
// of smallest modulus); min(n, max(20, 2 k_ev + 6), KRY) Arnoldi steps on K with classical
// Gram-Schmidt applied twice (whole block: 4 threads per row for K v, one warp per basis
// vector for the inner products); the eigenvalues of the Hessenberg matrix by the Francis QR iteration (one
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
    {  // Km = (B - sigma T)^{-1} T: the LU by the block, then several columns per warp
        __shared__ int src[CN];
        block_lu_factor<float>(A, n, src, dinv, 1e-30f);
        __syncthreads();
        warp_lu_solve_cols<float, CN / (CT / 32)>(A, n, src, dinv, Km, LDP, wid * (CN / (CT / 32)), n);
        __syncthreads();
    }
    const long long c_lu = clock64();
    // Krylov dimension: the wanted eigenvalues are the dominant ones of K, so 2 k_ev + 6 steps
    // (at least 20, at most KRY) give them to shift accuracy; the QR work grows with its square
    const int kwant = 2 * k_ev + 6 > 20 ? 2 * k_ev + 6 : 20;
    const int kd = min(n, min(KRY, kwant));
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
        if (st != 0) {
            // The FP32 QR iteration on the shift-invert Arnoldi matrix did not converge (seen
            // on birth-death chains whose coarsest eigenvalues cluster near 0 by many orders of
            // magnitude): the coarsest level then supplies the state vector alone, by inverse
            // iteration at shift 0 (the eigenvalue it belongs to is exactly 0).
            sel[0] = sel[1] = sel[2] = 0.0;
            lam[0] = 0.0;
            kind[0] = 0;
            col = ns = 1;
        }
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
// start drawn per column (FP64: two triangular solves per step in one warp; FP32: the
// matrix K = (B - sigma T)^{-1} T formed once by all warps, eight right-hand sides each,
// then products with K); the Rayleigh-type quotient lambda = v^H B v / v^H T v (Algorithm
// 3's update, in complex form, accumulated in F); and the phase that makes <w, v> real and
// positive (w_i = i + 1) with unit 2-norm.
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
                                                      int* __restrict__ cycles, const int* __restrict__ info) {
    pdl_begin();
    if ((int)blockIdx.x >= info[1]) return;  // past the selected eigenvalues (uniform per block)
    extern __shared__ __align__(16) unsigned char smraw[];
    F* Ar = reinterpret_cast<F*>(smraw);
    F* Ai = Ar + CN * LDP;
    F* Bm = Ai + CN * LDP;
    F* Tm = Bm + CN * LDP;
    __shared__ F vr[CN], vi[CN], tr[CN], ti[CN], dr[CN], di[CN], pre[4 * CN], pim[4 * CN];
    __shared__ typename std::conditional<sizeof(F) == 4, float, double>::type red[4 * (CT / 32)];
    const long long c_start = clock64();
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
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
    // complex LU with partial pivoting on |Re| + |Im|, rows in place: row srcp[i] holds
    // pivot row i, dr + i di = 1 / u_ii
    __shared__ int srcp[CN];
    block_lu_factor_cplx<F>(Ar, Ai, n, srcp, dr, di, pfloor);
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
    if constexpr (sizeof(F) == 4) {
        // FP32: K = (B - sigma T)^{-1} T once (each warp solves 8 of its columns), then the four
        // steps as products v <- K v by the block (4 threads per row); the normalisation in FP32
        F* Kr = Tm + CN * LDP;
        F* Ki = Kr + CN * LDP;
        warp_lu_solve_cols_cplx<F, CN / (CT / 32)>(Ar, Ai, n, srcp, dr, di, Tm, Kr, Ki, wid * (CN / (CT / 32)));
        __syncthreads();
        for (int it = 0; it < 4; ++it) {
            if (row < n) {
                F a = F(0), b = F(0);
                const int c1 = min(n, 16 * quarter + 16);
                for (int c = 16 * quarter; c < c1; ++c) {
                    const F kr = Kr[row * LDP + c], ki = Ki[row * LDP + c];
                    a += kr * vr[c] - ki * vi[c];
                    b += kr * vi[c] + ki * vr[c];
                }
                pre[quarter * CN + row] = a;
                pim[quarter * CN + row] = b;
            }
            __syncthreads();
            if (wid == 0) {
                F xr[2], xi[2], nn = F(0);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    xr[h] = r < n ? (pre[r] + pre[CN + r]) + (pre[2 * CN + r] + pre[3 * CN + r]) : F(0);
                    xi[h] = r < n ? (pim[r] + pim[CN + r]) + (pim[2 * CN + r] + pim[3 * CN + r]) : F(0);
                    nn += xr[h] * xr[h] + xi[h] * xi[h];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
                const F sc = rsqrtf(nn);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    if (r < n) {
                        vr[r] = xr[h] * sc;
                        vi[r] = xi[h] * sc;
                    }
                }
            }
            __syncthreads();
        }
    } else {
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
            int fr[2];  // the rows of A holding this lane's equations
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // row interchanges
                const int r = lane + 32 * h;
                fr[h] = r < n ? srcp[r] : 0;
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
                        const F lr = Ar[fr[h] * LDP + q], li = Ai[fr[h] * LDP + q];
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
                        const F ur = Ar[fr[h] * LDP + q], ui = Ai[fr[h] * LDP + q];
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
    }
    // lambda = v^H B v / v^H T v: (B v)_r and (T v)_r with 4 threads per row, the sums in
    // FP64 (FP32 for the FP32 vectors)
    using Acc = typename std::conditional<sizeof(F) == 4, float, double>::type;
    auto wsum = [](Acc v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    {
        Acc br_ = Acc(0), bi_ = Acc(0), tr_ = Acc(0), ti_ = Acc(0);
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
            const Acc xr = vr[row], xi = vi[row];
            br_ = xr * wbr + xi * wbi;
            bi_ = xr * wbi - xi * wbr;
            tr_ = xr * wtr + xi * wti;
            ti_ = xr * wti - xi * wtr;
        }
        br_ = wsum(br_);
        bi_ = wsum(bi_);
        tr_ = wsum(tr_);
        ti_ = wsum(ti_);
        if (lane == 0) {
            red[4 * wid] = br_;
            red[4 * wid + 1] = bi_;
            red[4 * wid + 2] = tr_;
            red[4 * wid + 3] = ti_;
        }
    }
    __syncthreads();
    if (tid >= 32) return;
    Acc sr2 = Acc(0), si2 = Acc(0);
    for (int r = lane; r < n; r += 32) {
        sr2 += (Acc)(r + 1) * vr[r];
        si2 += (Acc)(r + 1) * vi[r];
    }
    sr2 = wsum(sr2);
    si2 = wsum(si2);
    const Acc sa = hypot(sr2, si2);
    const Acc cr = sa > Acc(0) ? sr2 / sa : Acc(1), ci = sa > Acc(0) ? -si2 / sa : Acc(0);  // conj(s)/|s|
    Acc nn = Acc(0);
    Acc ar[2], ai[2];
    for (int q = 0, r = lane; q < 2; ++q, r += 32) {
        ar[q] = ai[q] = Acc(0);
        if (r < n) {
            ar[q] = (Acc)vr[r] * cr - (Acc)vi[r] * ci;
            ai[q] = (Acc)vr[r] * ci + (Acc)vi[r] * cr;
            nn += ar[q] * ar[q] + ai[q] * ai[q];
        }
    }
    nn = Acc(1) / sqrt(wsum(nn));
    for (int q = 0, r = lane; q < 2; ++q, r += 32)
        if (r < n) {
            V[(int64_t)col * n + r] = (double)(ar[q] * nn);
            if (si != F(0)) V[(int64_t)(col + 1) * n + r] = (double)(ai[q] * nn);
        }
    if (lane == 0) {
        Acc nbr = Acc(0), nbi = Acc(0), ntr = Acc(0), nti = Acc(0);
        for (int q = 0; q < CT / 32; ++q) {
            nbr += red[4 * q];
            nbi += red[4 * q + 1];
            ntr += red[4 * q + 2];
            nti += red[4 * q + 3];
        }
        // Re of (nbr + i nbi) / (ntr + i nti)
        double lre = (double)((nbr * ntr + nbi * nti) / (ntr * ntr + nti * nti));
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
    const size_t smem64 = 4 * CN * LDP * sizeof(double), smem32 = 6 * CN * LDP * sizeof(float);
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
    // one block per selected eigenvalue: k_ev blocks, those past the selection (info[1])
    // return at once, so the launch needs no read of the selection by the host; the columns
    // filled (info[0]) are read while the blocks run
    TmpBuf<int> cyc(2 * k_ev, s);
    if (fp32_vectors)
        BAMG_LAUNCH(k_coarse_eigvec<float>, k_ev, CT, smem32, s, n, dB, dT, sel.get(), d_V, d_lam, cyc.get(),
                    (const int*)info.get());
    else
        BAMG_LAUNCH(k_coarse_eigvec<double>, k_ev, CT, smem64, s, n, dB, dT, sel.get(), d_V, d_lam, cyc.get(),
                    (const int*)info.get());
    int h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    if (getenv("BAMG_DEBUG")) {
        fprintf(stderr,
                "[bamg] coarse eigenvalues: n=%d QR double-shift steps=%d status=%d cycles lu+K=%d arnoldi=%d qr=%d "
                "tail=%d\n",
                n, h[3], h[2], h[4], h[5], h[6], h[7]);
        if (h[2] != 0) fprintf(stderr, "[bamg] coarse eigenvalues: QR did not converge; state vector only\n");
        int hc[64] = {0};
        BAMG_CK(cudaMemcpyAsync(hc, cyc.get(), sizeof(int) * 2 * k_ev, cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
        fprintf(stderr, "[bamg] coarse eigenvectors (%s): %d blocks, cycles lu=%d iterate=%d\n",
                fp32_vectors ? "fp32" : "fp64", h[1], hc[0], hc[1]);
    }
    return h[0];
}

// ---------------------------------------------------------------- minimal-norm inverse
// B has rank n-1 and left null vector 1 (1^T B = 0).  With z = 1/sqrt(n), M = B + z z^T is
// nonsingular, and one factorisation of M gives B^+: M y = z yields the right null vector
// (z^T B = 0 forces z^T y = 1, hence B y = 0), and M w = (I - z z^T) b forces z^T w = 0,
// hence B w = (I - z z^T) b; the minimal-norm solution is w minus its component along y, so
// B^+ b = (I - y y^T / y^T y) M^{-1} (I - z z^T) b.  Every block factors M (identically) and
// solves y and its own PINV_COLS columns, one per warp.  Arithmetic F: FP64,
// or FP32 for the mixed-precision V-cycle, which applies B^+ in FP32.
constexpr int PINV_COLS = 8;
template <typename F>
__global__ void __launch_bounds__(CT) k_coarse_pinv(int n, const double* __restrict__ Bg, double* __restrict__ Pg,
                                                    int* __restrict__ info, int* __restrict__ fail) {
    pdl_begin();
    __shared__ F A[CN * LDP];
    __shared__ F R[CN * PINV_COLS];
    __shared__ F y[CN], dinv[CN];
    __shared__ int src[CN];
    const int tid = threadIdx.x, lane = lane_id(), wid = tid >> 5;
    const long long c_start = clock64();
    const int c0 = blockIdx.x * PINV_COLS, mc = min(PINV_COLS, n - c0);
    const F ninv = (F)(1.0 / (double)n);
    for (int idx = tid; idx < n * n; idx += CT) {
        const int r = idx / n, c = idx - r * n;
        A[r * LDP + c] = (F)Bg[idx] + ninv;  // B + z z^T
    }
    for (int idx = tid; idx < n * mc; idx += CT) {
        const int r = idx / mc, c = idx - r * mc;
        R[r * mc + c] = (r == c0 + c ? F(1) : F(0)) - ninv;  // (I - z z^T) e_c
    }
    if (tid < n) y[tid] = (F)(1.0 / sqrt((double)n));
    __syncthreads();
    block_lu_factor<F>(A, n, src, dinv, pivot_tiny<F>());
    __syncthreads();
    const long long c_lu = clock64();
    if (wid == 0) warp_lu_solve<F>(A, n, src, dinv, y, 1);            // M y = z
    if (wid < mc) warp_lu_solve<F>(A, n, src, dinv, R + wid, mc);     // M w = (I - z z^T) e_c
    __syncthreads();
    const long long c_solve = clock64();
    if (wid < mc) {  // w - y (y^T w) / (y^T y)
        double yw = 0.0, yy = 0.0;
        for (int r = lane; r < n; r += 32) {
            yw += (double)y[r] * (double)R[r * mc + wid];
            yy += (double)y[r] * (double)y[r];
        }
        yw = warp_sum(yw);
        yy = warp_sum(yy);
        const F f = (F)(yy > 0.0 ? yw / yy : 0.0);
        __syncwarp();
        for (int r = lane; r < n; r += 32) R[r * mc + wid] -= f * y[r];
    }
    __syncthreads();
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
        if (fail && bad) atomicOr(fail, 2);
        info[4 * blockIdx.x + 1] = 0;  // diagnostics: cycles per phase
        info[4 * blockIdx.x + 2] = (int)(c_lu - c_start);
        info[4 * blockIdx.x + 3] = (int)(c_solve - c_lu);
    }
}

int coarse_pinv(int n, const double* dB, double* dP, bool fp32, cudaStream_t s, int* d_fail) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_pinv: coarsest order must be 1..64");
    const int nb = (n + PINV_COLS - 1) / PINV_COLS;
    TmpBuf<int> info(4 * nb, s);
    if (fp32)
        BAMG_LAUNCH(k_coarse_pinv<float>, nb, CT, 0, s, n, dB, dP, info.get(), d_fail);
    else
        BAMG_LAUNCH(k_coarse_pinv<double>, nb, CT, 0, s, n, dB, dP, info.get(), d_fail);
    if (d_fail && !getenv("BAMG_DEBUG")) return 0;  // the caller reads the flag later
    int h[4 * (CN / PINV_COLS)] = {0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(int) * 4 * nb, cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    if (getenv("BAMG_DEBUG"))
        fprintf(stderr, "[bamg] coarse pinv (%s): n=%d blocks=%d cycles lu=%d solve=%d\n", fp32 ? "fp32" : "fp64", n,
                nb, h[2], h[3]);
    for (int b = 0; b < nb; ++b)
        if (h[4 * b]) return BAMG_ENUMERIC;
    return 0;
}

}  // namespace bamg
