// Coarsest level (Algorithm 3, first branch; Section 4.2): the eigenpairs of
// B_L x = lambda T_L x with the smallest |lambda|, and the minimal-norm inverse B_L^+.
// Dense FP64, order n <= 64, each kernel run by one warp with the matrices in shared
// memory.  Methods: LU with partial pivoting; Householder reduction to Hessenberg
// form and the implicit double-shift QR iteration for the eigenvalues (Francis; Golub &
// Van Loan, Matrix Computations, Sec. 7.5); inverse iteration in complex arithmetic
// for the eigenvectors; a bordered LU solve for B^+.
#include <cfloat>

#include "kernels.cuh"

namespace bamg {

constexpr int CN = 64;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ---------------------------------------------------------------- real LU
// In-place LU with partial pivoting of the n x n row-major A; perm[k] = pivot row of
// step k.  Pivots smaller than floorv in magnitude are replaced by +-floorv.
__device__ void lu_factor(double* A, int n, int* perm, double floorv) {
    const int lane = lane_id();
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int br = k;
        for (int r = k + lane; r < n; r += 32) {
            const double v = fabs(A[r * n + k]);
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
        if (lane == 0) perm[k] = br;
        if (br != k)
            for (int c = lane; c < n; c += 32) {
                const double t = A[k * n + c];
                A[k * n + c] = A[br * n + c];
                A[br * n + c] = t;
            }
        __syncwarp();
        double p = A[k * n + k];
        if (fabs(p) < floorv) p = p >= 0.0 ? floorv : -floorv;
        __syncwarp();
        if (lane == 0) A[k * n + k] = p;
        for (int r = k + 1 + lane; r < n; r += 32) A[r * n + k] /= p;
        __syncwarp();
        const int m = n - k - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int r = k + 1 + idx / m, c = k + 1 + idx % m;
            A[r * n + c] -= A[r * n + k] * A[k * n + c];
        }
        __syncwarp();
    }
}

// Solves A X = Bm for m right-hand sides stored row-major (n x m) in place.
__device__ void lu_solve(const double* A, int n, const int* perm, double* Bm, int m) {
    const int lane = lane_id();
    for (int k = 0; k < n; ++k) {
        const int pk = perm[k];
        if (pk != k)
            for (int c = lane; c < m; c += 32) {
                const double t = Bm[k * m + c];
                Bm[k * m + c] = Bm[pk * m + c];
                Bm[pk * m + c] = t;
            }
        __syncwarp();
    }
    for (int c = lane; c < m; c += 32) {
        for (int r = 0; r < n; ++r) {
            double s = Bm[r * m + c];
            for (int q = 0; q < r; ++q) s -= A[r * n + q] * Bm[q * m + c];
            Bm[r * m + c] = s;
        }
        for (int r = n - 1; r >= 0; --r) {
            double s = Bm[r * m + c];
            for (int q = r + 1; q < n; ++q) s -= A[r * n + q] * Bm[q * m + c];
            Bm[r * m + c] = s / A[r * n + r];
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- Hessenberg + QR
__device__ void hessenberg(double* H, int n, double* v) {
    const int lane = lane_id();
    for (int k = 0; k + 2 < n; ++k) {
        double ss = 0.0;
        for (int r = k + 1 + lane; r < n; r += 32) ss += H[r * n + k] * H[r * n + k];
        ss = warp_sum(ss);
        const double x0 = H[(k + 1) * n + k];
        if (ss == x0 * x0) continue;  // column already reduced
        const double alpha = -copysign(sqrt(ss), x0);
        const double v0 = x0 - alpha;
        const double vn2 = ss - x0 * x0 + v0 * v0;
        const double beta = 2.0 / vn2;
        for (int r = k + 1 + lane; r < n; r += 32) v[r] = (r == k + 1) ? v0 : H[r * n + k];
        __syncwarp();
        for (int c = k + lane; c < n; c += 32) {
            double d = 0.0;
            for (int r = k + 1; r < n; ++r) d += v[r] * H[r * n + c];
            d *= beta;
            for (int r = k + 1; r < n; ++r) H[r * n + c] -= d * v[r];
        }
        __syncwarp();
        for (int r = lane; r < n; r += 32) {
            double d = 0.0;
            for (int c = k + 1; c < n; ++c) d += H[r * n + c] * v[c];
            d *= beta;
            for (int c = k + 1; c < n; ++c) H[r * n + c] -= d * v[c];
        }
        __syncwarp();
        if (lane == 0) {
            H[(k + 1) * n + k] = alpha;
            for (int r = k + 2; r < n; ++r) H[r * n + k] = 0.0;
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void house3(double x, double y, double z, double& v0, double& v1, double& v2, double& beta) {
    const double nrm = sqrt(x * x + y * y + z * z);
    if (nrm == 0.0) {
        v0 = 1.0;
        v1 = v2 = 0.0;
        beta = 0.0;
        return;
    }
    const double alpha = -copysign(nrm, x);
    v0 = x - alpha;
    v1 = y;
    v2 = z;
    beta = 2.0 / (v0 * v0 + v1 * v1 + v2 * v2);
}

// Eigenvalues of the upper Hessenberg H (destroyed).  Returns 0, or -1 if the
// iteration did not converge within 40 n double-shift steps.
__device__ int hqr(double* H, int n, double* wr, double* wi) {
    const int lane = lane_id();
    double hnorm = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) hnorm = fmax(hnorm, fabs(H[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hnorm = fmax(hnorm, __shfl_xor_sync(0xffffffffu, hnorm, o));
    if (hnorm == 0.0) hnorm = 1.0;
    int hi = n - 1, its = 0, total = 0;
    while (hi >= 0) {
        if (total > 40 * n) return -1;
        int l = hi;
        while (l > 0) {
            double s = fabs(H[(l - 1) * n + l - 1]) + fabs(H[l * n + l]);
            if (s == 0.0) s = hnorm;
            if (fabs(H[l * n + l - 1]) <= DBL_EPSILON * s) break;
            --l;
        }
        __syncwarp();
        if (l == hi) {
            if (lane == 0) {
                wr[hi] = H[hi * n + hi];
                wi[hi] = 0.0;
            }
            --hi;
            its = 0;
            __syncwarp();
            continue;
        }
        if (l == hi - 1) {
            const double a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
            const double c = H[hi * n + hi - 1], d = H[hi * n + hi];
            const double p = 0.5 * (a - d), q = p * p + b * c, mid = d + p;
            if (lane == 0) {
                if (q >= 0.0) {
                    const double sq = sqrt(q);
                    const double l1 = mid + copysign(sq, mid);
                    const double det = a * d - b * c;
                    const double l2 = l1 != 0.0 ? det / l1 : mid - sq;
                    wr[hi - 1] = l1;
                    wr[hi] = l2;
                    wi[hi - 1] = wi[hi] = 0.0;
                } else {
                    const double im = sqrt(-q);
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
        double s, t;
        if (its == 10 || its == 20) {
            const double e = fabs(H[hi * n + hi - 1]) + fabs(H[(hi - 1) * n + hi - 2]);
            s = 1.5 * e;
            t = e * e;
        } else {
            s = H[(hi - 1) * n + hi - 1] + H[hi * n + hi];
            t = H[(hi - 1) * n + hi - 1] * H[hi * n + hi] - H[(hi - 1) * n + hi] * H[hi * n + hi - 1];
        }
        ++its;
        ++total;
        double x = H[l * n + l] * H[l * n + l] + H[l * n + l + 1] * H[(l + 1) * n + l] - s * H[l * n + l] + t;
        double y = H[(l + 1) * n + l] * (H[l * n + l] + H[(l + 1) * n + l + 1] - s);
        double z = H[(l + 1) * n + l] * H[(l + 2) * n + l + 1];
        __syncwarp();
        for (int k = l; k <= hi - 2; ++k) {
            double v0, v1, v2, beta;
            house3(x, y, z, v0, v1, v2, beta);
            const int c0 = k - 1 > l ? k - 1 : l;
            for (int c = c0 + lane; c <= hi; c += 32) {
                const double d = beta * (v0 * H[k * n + c] + v1 * H[(k + 1) * n + c] + v2 * H[(k + 2) * n + c]);
                H[k * n + c] -= d * v0;
                H[(k + 1) * n + c] -= d * v1;
                H[(k + 2) * n + c] -= d * v2;
            }
            __syncwarp();
            const int r1 = k + 3 < hi ? k + 3 : hi;
            for (int r = l + lane; r <= r1; r += 32) {
                const double d = beta * (H[r * n + k] * v0 + H[r * n + k + 1] * v1 + H[r * n + k + 2] * v2);
                H[r * n + k] -= d * v0;
                H[r * n + k + 1] -= d * v1;
                H[r * n + k + 2] -= d * v2;
            }
            __syncwarp();
            x = H[(k + 1) * n + k];
            y = H[(k + 2) * n + k];
            z = (k + 3 <= hi) ? H[(k + 3) * n + k] : 0.0;
            __syncwarp();
        }
        {
            double v0, v1, v2, beta;
            house3(x, y, 0.0, v0, v1, v2, beta);
            const int k = hi - 1;
            for (int c = (k - 1) + lane; c <= hi; c += 32) {
                const double d = beta * (v0 * H[k * n + c] + v1 * H[(k + 1) * n + c]);
                H[k * n + c] -= d * v0;
                H[(k + 1) * n + c] -= d * v1;
            }
            __syncwarp();
            for (int r = l + lane; r <= hi; r += 32) {
                const double d = beta * (H[r * n + k] * v0 + H[r * n + k + 1] * v1);
                H[r * n + k] -= d * v0;
                H[r * n + k + 1] -= d * v1;
            }
            __syncwarp();
        }
    }
    return 0;
}

// Kernel 1: M = T^{-1} B (kept in global memory for the vectors), its eigenvalues, and
// the selection: eigenvalues with Im >= 0 (each complex pair is represented by its
// member with positive imaginary part) sorted by |lambda|; a real one takes one vector
// column, a pair two (Re v, Im v), until k_ev columns are filled.
// sel[3*q + {0,1,2}] = (Re lambda, Im lambda, first column); info = {nvec, nsel, status}.
__global__ void k_coarse_eigvals(int n, const double* __restrict__ Bg, const double* __restrict__ Tg, int k_ev,
                                 double* __restrict__ Mg, double* __restrict__ sel, double* __restrict__ lam,
                                 int32_t* __restrict__ kind, int* __restrict__ info) {
    extern __shared__ double sm[];
    double* A = sm;            // B -> M -> Hessenberg
    double* Tm = sm + CN * CN; // T -> LU(T)
    __shared__ int perm[CN];
    __shared__ double v[CN], wr[CN], wi[CN];
    const int lane = lane_id();
    for (int idx = lane; idx < n * n; idx += 32) {
        A[idx] = Bg[idx];
        Tm[idx] = Tg[idx];
    }
    __syncwarp();
    lu_factor(Tm, n, perm, 1e-300);
    lu_solve(Tm, n, perm, A, n);
    for (int idx = lane; idx < n * n; idx += 32) Mg[idx] = A[idx];
    __syncwarp();
    hessenberg(A, n, v);
    const int st = hqr(A, n, wr, wi);
    __syncwarp();
    if (lane == 0) {
        int order[CN];
        int m = 0;
        for (int q = 0; q < n; ++q)
            if (wi[q] >= 0.0) order[m++] = q;
        for (int a = 1; a < m; ++a)
            for (int b = a; b > 0; --b) {
                const double m0 = hypot(wr[order[b - 1]], wi[order[b - 1]]);
                const double m1 = hypot(wr[order[b]], wi[order[b]]);
                if (m0 > m1) {
                    int t = order[b];
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
            if (wi[q] == 0.0) {
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
    }
}

// ---------------------------------------------------------------- complex inverse iteration
// Kernel 2: one block per selected eigenvalue.  Three steps of inverse iteration with
// (M - sigma I), sigma = lambda + delta (delta = 1e-10 max(1, max|M|) keeps the LU
// finite); then unit 2-norm and the phase that makes <w, v> real positive, w_i = i + 1.
__global__ void k_coarse_eigvec(int n, const double* __restrict__ Mg, const double* __restrict__ sel,
                                double* __restrict__ V) {
    extern __shared__ double sm[];
    double* Ar = sm;
    double* Ai = sm + CN * CN;
    __shared__ double vr[CN], vi[CN];
    __shared__ int perm[CN];
    const int lane = lane_id();
    const double lre = sel[3 * blockIdx.x], lim = sel[3 * blockIdx.x + 1];
    const int col = (int)sel[3 * blockIdx.x + 2];
    double mx = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) mx = fmax(mx, fabs(Mg[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double sr = lre + 1e-10 * fmax(1.0, mx), si = lim;
    for (int idx = lane; idx < n * n; idx += 32) {
        const int r = idx / n, c = idx % n;
        Ar[idx] = Mg[idx] - (r == c ? sr : 0.0);
        Ai[idx] = (r == c ? -si : 0.0);
    }
    __syncwarp();
    // complex LU with partial pivoting on |a|
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int br = k;
        for (int r = k + lane; r < n; r += 32) {
            const double m = hypot(Ar[r * n + k], Ai[r * n + k]);
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
        if (lane == 0) perm[k] = br;
        if (br != k)
            for (int c = lane; c < n; c += 32) {
                double t = Ar[k * n + c];
                Ar[k * n + c] = Ar[br * n + c];
                Ar[br * n + c] = t;
                t = Ai[k * n + c];
                Ai[k * n + c] = Ai[br * n + c];
                Ai[br * n + c] = t;
            }
        __syncwarp();
        double pr = Ar[k * n + k], pi = Ai[k * n + k];
        if (hypot(pr, pi) < 1e-300) {
            pr = 1e-300;
            pi = 0.0;
        }
        const double den = pr * pr + pi * pi;
        __syncwarp();
        if (lane == 0) {
            Ar[k * n + k] = pr;
            Ai[k * n + k] = pi;
        }
        for (int r = k + 1 + lane; r < n; r += 32) {
            const double ar = Ar[r * n + k], ai = Ai[r * n + k];
            Ar[r * n + k] = (ar * pr + ai * pi) / den;
            Ai[r * n + k] = (ai * pr - ar * pi) / den;
        }
        __syncwarp();
        const int m = n - k - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int r = k + 1 + idx / m, c = k + 1 + idx % m;
            const double lr = Ar[r * n + k], li = Ai[r * n + k];
            const double ur = Ar[k * n + c], ui = Ai[k * n + c];
            Ar[r * n + c] -= lr * ur - li * ui;
            Ai[r * n + c] -= lr * ui + li * ur;
        }
        __syncwarp();
    }
    for (int r = lane; r < n; r += 32) {
        vr[r] = 1.0 + (double)r / (double)n;
        vi[r] = 0.0;
    }
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
        if (lane == 0) {
            for (int k = 0; k < n; ++k) {
                const int pk = perm[k];
                if (pk != k) {
                    double t = vr[k];
                    vr[k] = vr[pk];
                    vr[pk] = t;
                    t = vi[k];
                    vi[k] = vi[pk];
                    vi[pk] = t;
                }
            }
            for (int r = 0; r < n; ++r) {
                double sr2 = vr[r], si2 = vi[r];
                for (int q = 0; q < r; ++q) {
                    sr2 -= Ar[r * n + q] * vr[q] - Ai[r * n + q] * vi[q];
                    si2 -= Ar[r * n + q] * vi[q] + Ai[r * n + q] * vr[q];
                }
                vr[r] = sr2;
                vi[r] = si2;
            }
            for (int r = n - 1; r >= 0; --r) {
                double sr2 = vr[r], si2 = vi[r];
                for (int q = r + 1; q < n; ++q) {
                    sr2 -= Ar[r * n + q] * vr[q] - Ai[r * n + q] * vi[q];
                    si2 -= Ar[r * n + q] * vi[q] + Ai[r * n + q] * vr[q];
                }
                const double ur = Ar[r * n + r], ui = Ai[r * n + r];
                const double d = ur * ur + ui * ui;
                vr[r] = (sr2 * ur + si2 * ui) / d;
                vi[r] = (si2 * ur - sr2 * ui) / d;
            }
        }
        __syncwarp();
        double nn = 0.0;
        for (int r = lane; r < n; r += 32) nn += vr[r] * vr[r] + vi[r] * vi[r];
        nn = sqrt(warp_sum(nn));
        for (int r = lane; r < n; r += 32) {
            vr[r] /= nn;
            vi[r] /= nn;
        }
        __syncwarp();
    }
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
    nn = sqrt(warp_sum(nn));
    for (int r = lane; r < n; r += 32) {
        V[(int64_t)col * n + r] = vr[r] / nn;
        if (lim != 0.0) V[(int64_t)(col + 1) * n + r] = vi[r] / nn;
    }
}

int coarse_eig(int n, const double* dB, const double* dT, int k_ev, double* d_lam, double* d_V, int32_t* d_kind,
               cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_eig: coarsest order must be 1..64");
    BAMG_REQUIRE(k_ev >= 1 && k_ev <= 16, BAMG_EINVAL, "coarse_eig: 1 <= k_ev <= 16");
    static bool attr = false;
    const size_t smem = 2 * CN * CN * sizeof(double);
    if (!attr) {
        BAMG_CK(cudaFuncSetAttribute(k_coarse_eigvals, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BAMG_CK(cudaFuncSetAttribute(k_coarse_eigvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    TmpBuf<double> M((size_t)n * n, s), sel(3 * (k_ev + 1), s);
    TmpBuf<int> info(4, s);
    BAMG_LAUNCH(k_coarse_eigvals, 1, 32, smem, s, n, dB, dT, k_ev, M.get(), sel.get(), d_lam, d_kind, info.get());
    int h[4] = {0, 0, 0, 0};
    BAMG_CK(cudaMemcpyAsync(h, info.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    if (h[2] != 0) return BAMG_ENUMERIC;
    if (h[1] > 0) BAMG_LAUNCH(k_coarse_eigvec, h[1], 32, smem, s, n, M.get(), sel.get(), d_V);
    return h[0];
}

// ---------------------------------------------------------------- minimal-norm inverse
// B has rank n-1 with left null vector 1.  y = its right null vector (two steps of
// inverse iteration on the LU of B with a pivot floor); with z = 1/sqrt(n) the bordered
// matrix M = B + z y^T is nonsingular and B^+ = M^{-1} (I - z z^T): M w = (I - z z^T) b
// forces y^T w = 0, so w is the solution of B w = (I - z z^T) b orthogonal to null(B).
__global__ void k_coarse_pinv(int n, const double* __restrict__ Bg, double* __restrict__ Pg, int* __restrict__ info) {
    extern __shared__ double sm[];
    double* A = sm;
    double* R = sm + CN * CN;
    __shared__ double y[CN];
    __shared__ int perm[CN];
    const int lane = lane_id();
    double mx = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) {
        A[idx] = Bg[idx];
        mx = fmax(mx, fabs(Bg[idx]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncwarp();
    lu_factor(A, n, perm, 1e-14 * fmax(mx, 1e-300));
    for (int r = lane; r < n; r += 32) R[r] = 1.0;
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
        lu_solve(A, n, perm, R, 1);
        double nn = 0.0;
        for (int r = lane; r < n; r += 32) nn += R[r] * R[r];
        nn = sqrt(warp_sum(nn));
        for (int r = lane; r < n; r += 32) R[r] /= nn;
        __syncwarp();
    }
    for (int r = lane; r < n; r += 32) y[r] = R[r];
    __syncwarp();
    const double zs = 1.0 / sqrt((double)n);
    for (int idx = lane; idx < n * n; idx += 32) {
        const int r = idx / n, c = idx % n;
        A[idx] = Bg[idx] + zs * y[c];
        R[idx] = (r == c ? 1.0 : 0.0) - 1.0 / (double)n;
    }
    __syncwarp();
    lu_factor(A, n, perm, 1e-300);
    lu_solve(A, n, perm, R, n);
    int bad = 0;
    for (int idx = lane; idx < n * n; idx += 32) {
        const double v = R[idx];
        if (!(fabs(v) < INFINITY)) bad = 1;
        Pg[idx] = v;
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) info[0] = bad;
}

int coarse_pinv(int n, const double* dB, double* dP, cudaStream_t s) {
    BAMG_REQUIRE(n >= 1 && n <= CN, BAMG_EINVAL, "coarse_pinv: coarsest order must be 1..64");
    static bool attr = false;
    const size_t smem = 2 * CN * CN * sizeof(double);
    if (!attr) {
        BAMG_CK(cudaFuncSetAttribute(k_coarse_pinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    TmpBuf<int> info(1, s);
    BAMG_LAUNCH(k_coarse_pinv, 1, 32, smem, s, n, dB, dP, info.get());
    int h = 0;
    BAMG_CK(cudaMemcpyAsync(&h, info.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    return h ? BAMG_ENUMERIC : 0;
}

}  // namespace bamg
