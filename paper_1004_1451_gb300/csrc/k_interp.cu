// Interpolation and coarse operators: full coarsening (Section 5.1), the coarse
// neighbourhoods of Eq. (3.5), the greedy least-squares fit of Algorithm 2 / Eq. (3.6),
// the averaging restriction Q of Section 4, and the Petrov-Galerkin products
// B_{l+1} = Q B P, T_{l+1} = Q T P (Section 1 step 3, Algorithm 3).
#include <cfloat>

#include <atomic>
#include <chrono>

#include "kernels.cuh"

namespace bamg {

// ================================================================ scan
constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_B = SCAN_T * SCAN_I;

__global__ void k_scan_local(const int32_t* __restrict__ in, int32_t* __restrict__ out, int n,
                             int32_t* __restrict__ bsum) {
    pdl_begin();
    __shared__ int32_t wsum[SCAN_T / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_I;
    int32_t v[SCAN_I];
    int32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tsum += v[k];
    }
    int32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < SCAN_T / 32 ? wsum[lane] : 0;
        int32_t incl = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < SCAN_T / 32) wsum[lane] = incl - w;
        if (lane == SCAN_T / 32 - 1) bsum[blockIdx.x] = incl;
    }
    __syncthreads();
    int32_t run = x - tsum + wsum[warp];
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_sums(int32_t* __restrict__ bsum, int nb, int32_t* __restrict__ total,
                            int32_t* __restrict__ h_total) {
    pdl_begin();
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int32_t v = i < nb ? bsum[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            int32_t incl = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            wsum[lane] = incl - w;
        }
        __syncthreads();
        const int32_t excl = carry + wsum[warp] + x - v;
        __syncthreads();
        if (i < nb) bsum[i] = excl;
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total = carry;
        if (h_total) {
            *(volatile int32_t*)h_total = carry;
            __threadfence_system();
        }
    }
}

__global__ void k_scan_add(int32_t* __restrict__ out, int n, const int32_t* __restrict__ bsum) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_B];
}

// Arrays of up to SCAN_ONE_MAX entries: one block walks the tiles in order with a running
// carry (one launch instead of three).  out[n] = total; out may alias in.
constexpr int SCAN_ONE_T = 1024, SCAN_ONE_MAX = 32768;
__global__ void __launch_bounds__(SCAN_ONE_T) k_scan_one(const int32_t* in, int32_t* out, int n,
                                                         int32_t* __restrict__ h_total) {
    pdl_begin();
    __shared__ int32_t wsum[SCAN_ONE_T / 32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += (int64_t)SCAN_ONE_T * SCAN_I) {
        const int64_t base = t0 + (int64_t)threadIdx.x * SCAN_I;
        int32_t v[SCAN_I];
        int32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < SCAN_I; ++k) {
            v[k] = (base + k < n) ? in[base + k] : 0;
            tsum += v[k];
        }
        int32_t x = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int32_t w = wsum[lane];
            int32_t incl = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            wsum[lane] = incl - w;
        }
        __syncthreads();
        int32_t run = carry + wsum[warp] + x - tsum;
#pragma unroll
        for (int k = 0; k < SCAN_I; ++k) {
            if (base + k < n) out[base + k] = run;
            run += v[k];
        }
        __syncthreads();  // every thread has read carry and wsum
        if (threadIdx.x == SCAN_ONE_T - 1) carry = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        if (h_total) {
            *(volatile int32_t*)h_total = carry;
            __threadfence_system();
        }
    }
}

// ---------------------------------------------------------------- counts read by the host
// A word of mapped pinned host memory per host thread and device: a kernel stores a count
// there and the host polls it, instead of a device-to-host copy and a stream synchronisation
// (whose completion path left the GPU idle for about 20 us per read in the setup).
struct HostWord {
    int32_t* h = nullptr;
    int32_t* d = nullptr;
};
static HostWord& host_word() {
    thread_local HostWord w[64];
    int dev = 0;
    BAMG_CK(cudaGetDevice(&dev));
    BAMG_REQUIRE(dev >= 0 && dev < 64, BAMG_EINVAL, "device ordinal out of range");
    HostWord& hw = w[dev];
    if (!hw.h) {
        BAMG_CK(cudaHostAlloc((void**)&hw.h, 64, cudaHostAllocMapped | cudaHostAllocPortable));
        BAMG_CK(cudaHostGetDevicePointer((void**)&hw.d, hw.h, 0));
    }
    return hw;
}
constexpr int32_t HOST_WORD_EMPTY = INT32_MIN;
// The count a kernel queued on s stores in the word: polled, with the stream's state checked
// now and then so that an error or a stream that finished without storing is reported; a
// bounded wait (BAMG_ETIMEOUT after 60 s).
static int32_t host_word_wait(const HostWord& hw, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (uint64_t k = 0;; ++k) {
        const int32_t v = *(volatile int32_t*)hw.h;
        if (v != HOST_WORD_EMPTY) return v;
        if ((k & 1023) == 1023) {
            const cudaError_t e = cudaStreamQuery(s);
            if (e != cudaSuccess && e != cudaErrorNotReady) BAMG_CK(e);
            if (e == cudaSuccess && *(volatile int32_t*)hw.h == HOST_WORD_EMPTY)
                throw Error(BAMG_ECUDA, "a count the host waits for was not stored");
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
                throw Error(BAMG_ETIMEOUT, "waiting for a count from the device");
        }
    }
}
__global__ void k_word_copy(const int32_t* __restrict__ d_p, int32_t* __restrict__ h) {
    pdl_begin();
    *(volatile int32_t*)h = *d_p;
    __threadfence_system();
}

void exclusive_scan(const int32_t* d_in, int32_t* d_out, int n, cudaStream_t s, int32_t* h_total) {
    if (n <= 0) {
        BAMG_CK(cudaMemsetAsync(d_out, 0, sizeof(int32_t), s));
        if (h_total) BAMG_LAUNCH(k_word_copy, 1, 1, 0, s, (const int32_t*)d_out, h_total);
        return;
    }
    if (n <= SCAN_ONE_MAX) {
        BAMG_LAUNCH(k_scan_one, 1, SCAN_ONE_T, 0, s, d_in, d_out, n, h_total);
        return;
    }
    const int nb = (int)blocks_for(n, SCAN_B);
    TmpBuf<int32_t> bsum(nb, s);
    BAMG_LAUNCH(k_scan_local, nb, SCAN_T, 0, s, d_in, d_out, n, bsum.get());
    BAMG_LAUNCH(k_scan_sums, 1, 1024, 0, s, bsum.get(), nb, d_out + n, h_total);
    BAMG_LAUNCH(k_scan_add, blocks_for(n, 256), 256, 0, s, d_out, n, bsum.get());
}

// exclusive scan of n counts into d_out (n + 1 entries), returning the total to the host
int32_t exclusive_scan_total(const int32_t* d_in, int32_t* d_out, int n, cudaStream_t s) {
    HostWord& hw = host_word();
    *(volatile int32_t*)hw.h = HOST_WORD_EMPTY;
    exclusive_scan(d_in, d_out, n, s, hw.d);
    return host_word_wait(hw, s);
}
// the same scan with the total left on its way to the host word (scan_total_wait collects it)
static void exclusive_scan_total_begin(const int32_t* d_in, int32_t* d_out, int n, cudaStream_t s) {
    HostWord& hw = host_word();
    *(volatile int32_t*)hw.h = HOST_WORD_EMPTY;
    exclusive_scan(d_in, d_out, n, s, hw.d);
}
static int32_t scan_total_wait(cudaStream_t s) { return host_word_wait(host_word(), s); }

int32_t read_int(const int32_t* d_p, cudaStream_t s) {
    HostWord& hw = host_word();
    *(volatile int32_t*)hw.h = HOST_WORD_EMPTY;
    BAMG_LAUNCH(k_word_copy, 1, 1, 0, s, d_p, hw.d);
    return host_word_wait(hw, s);
}

// ================================================================ coarsening
__global__ void k_coarsen_grid(int nx, int ny, uint8_t* __restrict__ cf, int32_t* __restrict__ cidx) {
    pdl_begin();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nx * ny) return;
    const int ix = (int)(i % nx), iy = (int)(i / nx);
    const bool c = (ix % 2 == 0) && (iy % 2 == 0);
    cf[i] = c ? 1 : 0;
    cidx[i] = c ? (ix / 2) + (iy / 2) * ((nx + 1) / 2) : -1;
}
void coarsen_grid(int nx, int ny, uint8_t* cf, int32_t* cidx, cudaStream_t s) {
    BAMG_LAUNCH(k_coarsen_grid, blocks_for((int64_t)nx * ny, 256), 256, 0, s, nx, ny, cf, cidx);
}

__global__ void k_coarse_to_fine(int n, const uint8_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                                 int32_t* __restrict__ c2f) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cf[i]) c2f[cidx[i]] = i;
}
void coarse_to_fine(int n, const uint8_t* cf, const int32_t* cidx, int32_t* c2f, cudaStream_t s) {
    if (n) BAMG_LAUNCH(k_coarse_to_fine, blocks_for(n, 256), 256, 0, s, n, cf, cidx, c2f);
}

// ================================================================ least-squares interpolation
constexpr int LS_WARPS = 4;
constexpr int VIS_CAP = 256;    // nodes recorded by one neighbourhood search (first pass)
constexpr int VIS_CAP2 = 2048;  // second pass, for the points whose search overflowed
constexpr int LS2_BLOCKS = 608;
constexpr int MMAX = 16;
constexpr int CMAX = 4;
constexpr int KMAX = 32;

// Solves the SPD system A x = b of order m <= CMAX by Cholesky; false if not SPD.
template <typename T>
__device__ __forceinline__ bool chol_solve(T (&A)[CMAX][CMAX], const T (&b)[CMAX], int m, T (&x)[CMAX]) {
    T L[CMAX][CMAX];
    T y[CMAX];
#pragma unroll
    for (int j = 0; j < CMAX; ++j) {
        if (j < m) {
            T s = A[j][j];
#pragma unroll
            for (int k = 0; k < CMAX; ++k)
                if (k < j) s -= L[j][k] * L[j][k];
            if (!(s > T(0))) return false;
            const T d = sqrt(s);
            L[j][j] = d;
#pragma unroll
            for (int i = 0; i < CMAX; ++i) {
                if (i > j && i < m) {
                    T t = A[i][j];
#pragma unroll
                    for (int k = 0; k < CMAX; ++k)
                        if (k < j) t -= L[i][k] * L[j][k];
                    L[i][j] = t / d;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CMAX; ++j) {
        if (j < m) {
            T t = b[j];
#pragma unroll
            for (int k = 0; k < CMAX; ++k)
                if (k < j) t -= L[j][k] * y[k];
            y[j] = t / L[j][j];
        }
    }
#pragma unroll
    for (int j = CMAX - 1; j >= 0; --j) {
        if (j < m) {
            T t = y[j];
#pragma unroll
            for (int k = 0; k < CMAX; ++k)
                if (k > j && k < m) t -= L[k][j] * x[k];
            x[j] = t / L[j][j];
        }
    }
    return true;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// b_rc, or 0 when column c is not in row r
template <typename T>
__device__ __forceinline__ T entry_of(int r, int c, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      const T* __restrict__ bv) {
    for (int p = rp[r]; p < rp[r + 1]; ++p)
        if (ci[p] == c) return bv[p];
    return T(0);
}

// Features of fine point i for the learned interpolation (one warp; lane s < ncand holds
// candidate `node` with path length `depth`, g_jj = gss and g_ij = bs): per slot
// [1, d / 3, g_ij / g_jj, g_ij / sqrt(g_ii g_jj), -b_ij / b_ii, -b_ji / b_jj] (ratios with a
// zero denominator are 0), zeros for empty slots, then [m / 16, sum_{j != i} |b_ij| / b_ii],
// zero-padded to MLP_F.
template <typename T>
__device__ void learned_features(int i, int lane, int node, int ncand, int depth, T gss, T bs, const T* xi,
                                 const T* s_w, int ncols, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, const T* __restrict__ bv, float* f) {
    T gii = T(0);
    for (int k = 0; k < ncols; ++k) gii += s_w[k] * xi[k] * xi[k];
    T bii_l = T(0), off_l = T(0);
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
        const T v = bv[p];
        if (ci[p] == i)
            bii_l += v;
        else
            off_l += v < T(0) ? -v : v;
    }
    const T bii = warp_sum_t(bii_l), off = warp_sum_t(off_l);
    if (lane < MLP_S) {
        float o[MLP_NF_SLOT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (lane < ncand && node >= 0) {
            const T bij = entry_of<T>(i, node, rp, ci, bv);
            const T bji = entry_of<T>(node, i, rp, ci, bv);
            const T bjj = entry_of<T>(node, node, rp, ci, bv);
            o[0] = 1.f;
            o[1] = (float)((double)depth / 3.0);
            o[2] = gss != T(0) ? (float)(bs / gss) : 0.f;
            o[3] = gii * gss != T(0) ? (float)(bs / sqrt(gii * gss)) : 0.f;
            o[4] = (float)(-bij / bii);
            o[5] = (float)(-bji / bjj);
        }
#pragma unroll
        for (int e = 0; e < MLP_NF_SLOT; ++e) f[MLP_NF_SLOT * lane + e] = o[e];
    }
    for (int k = MLP_NF_SLOT * MLP_S + lane; k < MLP_F; k += 32) {
        float v = 0.f;
        if (k == MLP_NF_SLOT * MLP_S) v = (float)((double)ncand / (double)MLP_S);
        if (k == MLP_NF_SLOT * MLP_S + 1) v = (float)(off / bii);
        f[k] = v;
    }
}

// One warp per point.  Fine points: breadth-first search to depth z over the row
// pattern of B (edges i -> j for b_ij != 0, i != j), continued up to depth 3 while no
// coarse point has been found, and stopped early once mmax coarse points are known at
// the depths already completed; candidates = coarse points found, ranked by (depth,
// coarse index) and cut to mmax; then the greedy steps of
// Algorithm 2 with one lane per candidate: each lane forms its (|J|+1)-square weighted
// normal equations (plus the Tikhonov term), solves them by Cholesky and evaluates the
// functional of Eq. (3.6) directly; the lane with the smallest value (lowest slot on
// ties) joins J.
// Visited set of a neighbourhood search: open addressing over 2 CAP slots (load <= 1/2),
// keys are node indices, -1 = empty.
__device__ __forceinline__ unsigned vis_hash(int v, int nslots) { return ((unsigned)v * 2654435761u) & (nslots - 1); }
__device__ __forceinline__ bool vis_contains(const int* hs, int nslots, int v) {
    for (unsigned h = vis_hash(v, nslots);; h = (h + 1) & (nslots - 1)) {
        const int k = hs[h];
        if (k == v) return true;
        if (k == -1) return false;
    }
}
__device__ __forceinline__ void vis_insert(int* hs, int nslots, int v) {
    for (unsigned h = vis_hash(v, nslots);; h = (h + 1) & (nslots - 1)) {
        const int prev = atomicCAS(&hs[h], -1, v);
        if (prev == -1 || prev == v) return;
    }
}

template <typename T, int CAP, bool EXTRA>
__device__ bool ls_point(int i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ bv, const uint8_t* __restrict__ cf, const int32_t* __restrict__ cidx, const T* __restrict__ X,
                         int ncols, int ld, const T* s_w, int z, int mmax, int c, double ridge,
                         int32_t* __restrict__ pcol, T* __restrict__ pval, int32_t* __restrict__ pcnt, int* vis,
                         unsigned long long* key, uint8_t* dist, int* cand, uint8_t* cdep, T* xi, T (*xj)[KMAX],
                         int* hs, bool defer, const LsOut& ex) {
    constexpr int HS = 2 * CAP;  // visited-set slots
    const int lane = threadIdx.x & 31;
    const int64_t prow = (int64_t)i * c;
    if (cf[i]) {
        if (lane < c) {
            pcol[prow + lane] = lane == 0 ? cidx[i] : -1;
            pval[prow + lane] = lane == 0 ? T(1) : T(0);
        }
        if (lane == 0) pcnt[i] = 1;
        if (EXTRA) {
            if (ex.feat)
                for (int k = lane; k < MLP_F; k += 32) ex.feat[(int64_t)i * MLP_F + k] = 0.f;
            if (ex.target && lane < MLP_S) ex.target[(int64_t)i * MLP_S + lane] = 0.f;
            if (ex.cand && lane < MLP_S) ex.cand[(int64_t)i * MLP_S + lane] = -1;
        }
        return false;
    }
    // ---- neighbourhood search (Eq. (3.5))
    __syncwarp();
    for (int e = lane; e < HS; e += 32) hs[e] = -1;
    __syncwarp();
    if (lane == 0) {
        vis[0] = i;
        dist[0] = 0;
        vis_insert(hs, HS, i);
    }
    __syncwarp();
    int nvis = 1, fs = 0, fe = 1, ncvis = 0;
    bool ovf = false;
    for (int d = 1; d <= 3; ++d) {
        // beyond z only while no coarse point has been reached (the extension of R30);
        // and no deeper once mmax coarse points are known: deeper ones would rank after them
        if ((d > z && ncvis > 0) || ncvis >= mmax) break;
        bool fonly = false;  // visited list full: record only coarse nodes for the rest of this depth
        // the frontier's rows, 32 frontier nodes at a time: the lanes load the row pointers
        // together, lay the rows end to end (warp prefix sum), and take 32 entries of the
        // concatenation per batch (the same entries in the same order as row by row)
        for (int f0 = fs; f0 < fe; f0 += 32) {
            const int fu = f0 + lane;
            const int u = fu < fe ? vis[fu] : -1;
            const int ra = u >= 0 ? rp[u] : 0;
            const int rlen = u >= 0 ? rp[u + 1] - ra : 0;
            int incl = rlen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            for (int e0 = 0; e0 < total; e0 += 32) {
                const int e = e0 + lane;
                int k = 0;  // the lane whose row holds entry e: the first with incl > e
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const int ic = __shfl_sync(0xffffffffu, incl, k + st - 1);
                    if (ic <= e) k += st;
                }
                const int ka = __shfl_sync(0xffffffffu, ra, k);
                const int kx = __shfl_sync(0xffffffffu, incl - rlen, k);
                const int v = e < total ? ci[ka + e - kx] : -1;
                const bool vc = v >= 0 && cf[v] != 0;  // loaded with v: the count below reads it from dist
                const bool isnew = v >= 0 && !vis_contains(hs, HS, v);
                const int key = isnew ? v : -1 - lane;
                const unsigned grp = __match_any_sync(0xffffffffu, key);
                const unsigned lt = (1u << lane) - 1u;
                const bool leader = isnew && (grp & lt) == 0u;
                unsigned bal = __ballot_sync(0xffffffffu, leader);
                if (fonly || nvis + __popc(bal) > CAP) {  // list full: keep the coarse nodes only
                    fonly = true;
                    bal = __ballot_sync(0xffffffffu, leader && vc);
                }
                const bool rec = (bal >> lane) & 1u;
                const int pos = nvis + __popc(bal & lt);
                if (rec && pos < CAP) {
                    vis[pos] = v;
                    dist[pos] = (uint8_t)(d | (vc ? 0x80 : 0));  // depth, and the C flag in bit 7
                    vis_insert(hs, HS, v);
                }
                int added = __popc(bal);
                if (nvis + added > CAP) {
                    ovf = true;
                    added = CAP - nvis;
                }
                nvis += added;
                __syncwarp();
            }
        }
        for (int q0 = fe; q0 < nvis; q0 += 32) {  // coarse points recorded at this depth
            const int q = q0 + lane;
            ncvis += __popc(__ballot_sync(0xffffffffu, q < nvis && (dist[q] & 0x80) != 0));
        }
        // a truncated depth (fine nodes not recorded) is exact only if the search ends here
        if (fonly) {
            if (d < 3 && ncvis < mmax && !(d >= z && ncvis > 0)) ovf = true;
            break;
        }
        fs = fe;
        fe = nvis;
    }
    if (ovf && defer) return true;  // the second pass redoes this point with a larger list
    // ---- candidates: coarse points ranked by (depth, coarse index).  The coarse entries
    // are compacted to the front of key (and their nodes to the front of vis; the point
    // itself at vis[0] is no longer needed), then ranked among themselves.
    int ntot = 0;
    for (int q0 = 1; q0 < nvis; q0 += 32) {
        const int q = q0 + lane;
        int v = -1;
        bool isc = false;
        unsigned long long kq = 0;
        if (q < nvis) {
            v = vis[q];
            isc = (dist[q] & 0x80) != 0;
            if (isc) kq = ((unsigned long long)(dist[q] & 0x7f) << 32) | (unsigned)cidx[v];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, isc);
        __syncwarp();  // every lane has read vis[q] before the compacted writes below
        if (isc) {
            const int pos = ntot + __popc(bal & ((1u << lane) - 1u));
            key[pos] = kq;
            vis[pos] = v;
        }
        ntot += __popc(bal);
        __syncwarp();
    }
    for (int q0 = 0; q0 < ntot; q0 += 32) {
        const int q = q0 + lane;
        if (q < ntot) {
            const unsigned long long kq = key[q];
            int rank = 0;
            for (int q2 = 0; q2 < ntot; ++q2) rank += key[q2] < kq;
            if (rank < mmax) {
                cand[rank] = vis[q];
                cdep[rank] = (uint8_t)(kq >> 32);
            }
        }
    }
    const int ncand = ntot < mmax ? ntot : mmax;
    for (int k = lane; k < KMAX; k += 32) xi[k] = k < ncols ? X[(int64_t)i * ld + k] : T(0);
    __syncwarp();
    // ---- greedy least squares (Algorithm 2)
    const int node = lane < ncand ? cand[lane] : -1;
    const T* xs = node >= 0 ? X + (int64_t)node * ld : nullptr;
    T gss = T(0), bs = T(0);
    if (node >= 0)
        for (int k = 0; k < ncols; ++k) {
            const T wk = s_w[k], v = xs[k];
            gss += wk * v * v;
            bs += wk * v * xi[k];
        }
    if (EXTRA && ex.cand && lane < MLP_S) ex.cand[(int64_t)i * MLP_S + lane] = node;
    if (EXTRA && ex.feat) learned_features<T>(i, lane, node, ncand, lane < ncand ? cdep[lane] : 0, gss, bs, xi, s_w, ncols, rp,
                                     ci, bv, ex.feat + (int64_t)i * MLP_F);
    if (EXTRA && !ex.greedy) return false;
    T gsj[CMAX], GJJ[CMAX][CMAX], bJ[CMAX], pbest[CMAX];
    int J[CMAX];
#pragma unroll
    for (int a = 0; a < CMAX; ++a) {
        gsj[a] = bJ[a] = pbest[a] = T(0);
        J[a] = -1;
#pragma unroll
        for (int b = 0; b < CMAX; ++b) GJJ[a][b] = T(0);
    }
    bool used = false;
    int nJ = 0;
    const T INF = (T)INFINITY;
#pragma unroll
    for (int t = 0; t < CMAX; ++t) {
        if (t >= c) break;
        T L = INF;
        T pl[CMAX];
#pragma unroll
        for (int a = 0; a < CMAX; ++a) pl[a] = T(0);
        if (node >= 0 && !used) {
            T A[CMAX][CMAX], rhs[CMAX];
            T tr = gss;
#pragma unroll
            for (int a = 0; a < CMAX; ++a) {
#pragma unroll
                for (int b = 0; b < CMAX; ++b) A[a][b] = (a < t && b < t) ? GJJ[a][b] : T(0);
                rhs[a] = a < t ? bJ[a] : T(0);
                if (a < t) tr += GJJ[a][a];
            }
#pragma unroll
            for (int a = 0; a < CMAX; ++a) {
                if (a < t) {
                    A[a][t] = gsj[a];
                    A[t][a] = gsj[a];
                }
            }
            A[t][t] = gss;
            rhs[t] = bs;
            const T delta = (T)ridge * tr / (T)(t + 1);
#pragma unroll
            for (int a = 0; a < CMAX; ++a)
                if (a <= t) A[a][a] += delta;
            if (chol_solve<T>(A, rhs, t + 1, pl)) {
                T acc = T(0);
                for (int k = 0; k < ncols; ++k) {
                    T r = xi[k] - pl[t] * xs[k];
#pragma unroll
                    for (int a = 0; a < CMAX; ++a)
                        if (a < t) r -= pl[a] * xj[a][k];
                    acc += s_w[k] * r * r;
                }
                L = (acc == acc) ? acc : INF;
            }
        }
        T bestL = L;
        int bestLane = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T oL = __shfl_xor_sync(0xffffffffu, bestL, o);
            const int oLane = __shfl_xor_sync(0xffffffffu, bestLane, o);
            if (oL < bestL || (oL == bestL && oLane < bestLane)) {
                bestL = oL;
                bestLane = oLane;
            }
        }
        if (!(bestL < INF)) break;
        const T w_gss = __shfl_sync(0xffffffffu, gss, bestLane);
        const T w_bs = __shfl_sync(0xffffffffu, bs, bestLane);
        const int w_node = __shfl_sync(0xffffffffu, node, bestLane);
#pragma unroll
        for (int a = 0; a < CMAX; ++a) {
            const T g = __shfl_sync(0xffffffffu, gsj[a], bestLane);
            const T pv = __shfl_sync(0xffffffffu, pl[a], bestLane);
            if (a < t) {
                GJJ[t][a] = g;
                GJJ[a][t] = g;
            }
            pbest[a] = a <= t ? pv : T(0);
        }
        GJJ[t][t] = w_gss;
        bJ[t] = w_bs;
        J[t] = w_node;
        nJ = t + 1;
        if (lane == bestLane) used = true;
        for (int k = lane; k < KMAX; k += 32) xj[t][k] = k < ncols ? X[(int64_t)w_node * ld + k] : T(0);
        __syncwarp();
        if (node >= 0) {
            T g = T(0);
            for (int k = 0; k < ncols; ++k) g += s_w[k] * xs[k] * xj[t][k];
            gsj[t] = g;
        }
    }
    if (lane == 0) {
        int cols[CMAX];
        T vals[CMAX];
#pragma unroll
        for (int a = 0; a < CMAX; ++a) {
            cols[a] = a < nJ ? cidx[J[a]] : 0x7fffffff;
            vals[a] = pbest[a];
        }
        for (int a = 1; a < nJ; ++a)
            for (int b = a; b > 0 && cols[b - 1] > cols[b]; --b) {
                int tc = cols[b];
                cols[b] = cols[b - 1];
                cols[b - 1] = tc;
                T tv = vals[b];
                vals[b] = vals[b - 1];
                vals[b - 1] = tv;
            }
        for (int a = 0; a < c; ++a) {
            pcol[prow + a] = a < nJ ? cols[a] : -1;
            pval[prow + a] = a < nJ ? vals[a] : T(0);
        }
        pcnt[i] = nJ;
    }
    if (EXTRA && ex.target && lane < MLP_S) {  // the LS row on the slots (Algorithm 2's choice)
        float tv = 0.f;
#pragma unroll
        for (int a = 0; a < CMAX; ++a)
            if (a < nJ && node >= 0 && J[a] == node) tv = (float)pbest[a];
        ex.target[(int64_t)i * MLP_S + lane] = tv;
    }
    return ovf;
}

// First pass (list == nullptr): warp per point i; a point whose search overflows the
// CAP-entry list is appended to ovf_list (or flags err when ovf_list is null).  Second
// pass (list != nullptr): persistent warps over the *list_count points of list.
template <typename T, int CAP, int WARPS, bool EXTRA>
__global__ void __launch_bounds__(WARPS * 32, (WARPS > 1 && sizeof(T) == 4) ? 8 : 1)  // FP32: 8 blocks/SM
    k_ls_fit(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ bv,
             const uint8_t* __restrict__ cf, const int32_t* __restrict__ cidx, const T* __restrict__ X, int ncols,
             int ld, const double* __restrict__ w, int z, int mmax, int c, double ridge, int32_t* __restrict__ pcol,
             T* __restrict__ pval, int32_t* __restrict__ pcnt, const int* __restrict__ list,
             const int* __restrict__ list_count, int* __restrict__ ovf_list, int* __restrict__ ovf_count,
             int* __restrict__ err, LsOut ex) {
    pdl_begin();
    __shared__ int s_vis[WARPS][CAP];
    __shared__ unsigned long long s_key[WARPS][CAP];
    __shared__ uint8_t s_dist[WARPS][CAP];
    __shared__ int s_cand[WARPS][MMAX];
    __shared__ uint8_t s_cdep[WARPS][MMAX];
    __shared__ int s_hash[WARPS][2 * CAP];
    __shared__ T s_xi[WARPS][KMAX];
    __shared__ T s_xj[WARPS][CMAX][KMAX];
    __shared__ T s_w[KMAX];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < KMAX) s_w[threadIdx.x] = threadIdx.x < ncols ? (T)w[threadIdx.x] : T(0);
    __syncthreads();
    if (list == nullptr) {
        const int i = blockIdx.x * WARPS + wid;
        if (i >= n) return;
        const bool ovf = ls_point<T, CAP, EXTRA>(i, rp, ci, bv, cf, cidx, X, ncols, ld, s_w, z, mmax, c, ridge, pcol, pval,
                                          pcnt, s_vis[wid], s_key[wid], s_dist[wid], s_cand[wid], s_cdep[wid],
                                          s_xi[wid], s_xj[wid], s_hash[wid], ovf_list != nullptr, ex);
        if (ovf && lane == 0) {
            if (ovf_list)
                ovf_list[atomicAdd(ovf_count, 1)] = i;
            else
                atomicOr(err, 1);
        }
        return;
    }
    const int cnt = *list_count;
    for (int k = blockIdx.x * WARPS + wid; k < cnt; k += gridDim.x * WARPS) {
        const bool ovf = ls_point<T, CAP, EXTRA>(list[k], rp, ci, bv, cf, cidx, X, ncols, ld, s_w, z, mmax, c, ridge, pcol,
                                          pval, pcnt, s_vis[wid], s_key[wid], s_dist[wid], s_cand[wid], s_cdep[wid],
                                          s_xi[wid], s_xj[wid], s_hash[wid], false, ex);
        if (ovf && lane == 0) atomicOr(err, 1);
    }
}

template <typename T>
int interp_ls(int n, const int32_t* rp, const int32_t* ci, const T* bv, const uint8_t* cf, const int32_t* cidx,
              const T* X, int ncols, int ld, const double* d_w, int z, int mmax, int c, double ridge, int32_t* pcol,
              T* pval, int32_t* pcnt, cudaStream_t s, int* d_err, const LsOut& ex) {
    BAMG_REQUIRE(ncols >= 1 && ncols <= KMAX, BAMG_EINVAL, "interp_ls: 1 <= ncols <= 32");
    BAMG_REQUIRE(c >= 1 && c <= CMAX, BAMG_EINVAL, "interp_ls: 1 <= caliber <= 4");
    BAMG_REQUIRE(mmax >= 1 && mmax <= MMAX, BAMG_EINVAL, "interp_ls: 1 <= mmax <= 16");
    BAMG_REQUIRE(z >= 1 && z <= 3, BAMG_EINVAL, "interp_ls: 1 <= z <= 3");
    if (n == 0) return 0;
    // two passes: the common case with a small visited list and 4 warps per block, then the
    // (rare) points whose search overflowed it, with a large list and one warp per block
    TmpBuf<int> olist(n, s), ocount(1, s), err(1, s);
    BAMG_CK(cudaMemsetAsync(ocount.get(), 0, sizeof(int), s));
    int* e = d_err ? d_err : err.get();  // with d_err the caller reads the overflow flag later
    if (!d_err) BAMG_CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    // the optional outputs are compiled into a separate instance (they cost registers)
    const bool extra = ex.feat || ex.target || ex.cand || !ex.greedy;
    if (extra) {
        BAMG_LAUNCH((k_ls_fit<T, VIS_CAP, LS_WARPS, true>), blocks_for(n, LS_WARPS), LS_WARPS * 32, 0, s, n, rp, ci, bv,
                    cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, pcol, pval, pcnt, (const int*)nullptr,
                    (const int*)nullptr, olist.get(), ocount.get(), e, ex);
        BAMG_LAUNCH((k_ls_fit<T, VIS_CAP2, 1, true>), LS2_BLOCKS, 32, 0, s, n, rp, ci, bv, cf, cidx, X, ncols, ld, d_w,
                    z, mmax, c, ridge, pcol, pval, pcnt, (const int*)olist.get(), (const int*)ocount.get(),
                    (int*)nullptr, (int*)nullptr, e, ex);
    } else {
        BAMG_LAUNCH((k_ls_fit<T, VIS_CAP, LS_WARPS, false>), blocks_for(n, LS_WARPS), LS_WARPS * 32, 0, s, n, rp, ci,
                    bv, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, pcol, pval, pcnt, (const int*)nullptr,
                    (const int*)nullptr, olist.get(), ocount.get(), e, ex);
        BAMG_LAUNCH((k_ls_fit<T, VIS_CAP2, 1, false>), LS2_BLOCKS, 32, 0, s, n, rp, ci, bv, cf, cidx, X, ncols, ld,
                    d_w, z, mmax, c, ridge, pcol, pval, pcnt, (const int*)olist.get(), (const int*)ocount.get(),
                    (int*)nullptr, (int*)nullptr, e, ex);
    }
    if (d_err) return 0;
    int h = 0;
    BAMG_CK(cudaMemcpyAsync(&h, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    return h ? BAMG_EOVERFLOW : 0;
}

// ================================================================ learned interpolation
// One thread per fine point: the c valid slots of largest |y| (lower slot on ties) form J;
// weights y, or with refit the minimiser of Eq. (3.6) over J with the Tikhonov term
// delta = ridge tr(G_JJ) / |J| (R25); the row is stored sorted by coarse index.
template <typename T>
__global__ void k_learned_select(int n, const uint8_t* __restrict__ cf, const int32_t* __restrict__ cidx,
                                 const int32_t* __restrict__ cand, const float* __restrict__ Y, const T* __restrict__ X,
                                 int ncols, int ld, const double* __restrict__ w, int c, int refit, double ridge,
                                 int32_t* __restrict__ pcol, T* __restrict__ pval, int32_t* __restrict__ pcnt) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || cf[i]) return;
    const int32_t* cd = cand + (int64_t)i * MLP_S;
    const float* y = Y + (int64_t)i * MLP_S;
    int m = 0;
    while (m < MLP_S && cd[m] >= 0) ++m;
    int slot[CMAX];
    int nJ = 0;
    unsigned used = 0u;
    for (int t = 0; t < c && t < m; ++t) {
        int best = -1;
        float bv = -1.f;
        for (int q = 0; q < m; ++q) {
            const float a = fabsf(y[q]);
            if (!((used >> q) & 1u) && a > bv) {
                bv = a;
                best = q;
            }
        }
        if (best < 0) break;
        used |= 1u << best;
        slot[nJ++] = best;
    }
    T p[CMAX];
#pragma unroll
    for (int a = 0; a < CMAX; ++a) p[a] = (a < nJ) ? (T)y[slot[a < nJ ? a : 0]] : T(0);
    if (refit && nJ > 0) {
        T A[CMAX][CMAX], rhs[CMAX], sol[CMAX];
        T tr = T(0);
#pragma unroll
        for (int a = 0; a < CMAX; ++a) {
            rhs[a] = T(0);
#pragma unroll
            for (int b = 0; b < CMAX; ++b) A[a][b] = T(0);
        }
        const T* xi = X + (int64_t)i * ld;
        for (int a = 0; a < nJ; ++a) {
            const T* xa = X + (int64_t)cd[slot[a]] * ld;
            for (int b = 0; b <= a; ++b) {
                const T* xb = X + (int64_t)cd[slot[b]] * ld;
                T g = T(0);
                for (int k = 0; k < ncols; ++k) g += (T)w[k] * xa[k] * xb[k];
                A[a][b] = g;
                A[b][a] = g;
            }
            T r = T(0);
            for (int k = 0; k < ncols; ++k) r += (T)w[k] * xa[k] * xi[k];
            rhs[a] = r;
            tr += A[a][a];
        }
        const T delta = (T)ridge * tr / (T)nJ;
        for (int a = 0; a < nJ; ++a) A[a][a] += delta;
        if (chol_solve<T>(A, rhs, nJ, sol))
#pragma unroll
            for (int a = 0; a < CMAX; ++a) p[a] = a < nJ ? sol[a] : T(0);
    }
    int cols[CMAX];
#pragma unroll
    for (int a = 0; a < CMAX; ++a) cols[a] = a < nJ ? cidx[cd[slot[a < nJ ? a : 0]]] : 0x7fffffff;
    for (int a = 1; a < nJ; ++a)
        for (int b = a; b > 0 && cols[b - 1] > cols[b]; --b) {
            const int tc = cols[b];
            cols[b] = cols[b - 1];
            cols[b - 1] = tc;
            const T tv = p[b];
            p[b] = p[b - 1];
            p[b - 1] = tv;
        }
    const int64_t prow = (int64_t)i * c;
    for (int a = 0; a < c; ++a) {
        pcol[prow + a] = a < nJ ? cols[a] : -1;
        pval[prow + a] = a < nJ ? p[a] : T(0);
    }
    pcnt[i] = nJ;
}

template <typename T>
int interp_learned(int n, const int32_t* rp, const int32_t* ci, const T* bv, const uint8_t* cf, const int32_t* cidx,
                   const T* X, int ncols, int ld, const double* d_w, int z, int mmax, int c, double ridge,
                   const Model* model, bool refit, int32_t* pcol, T* pval, int32_t* pcnt, cudaStream_t s, int* d_err) {
    BAMG_REQUIRE(model != nullptr, BAMG_EINVAL, "learned interpolation without a model");
    BAMG_REQUIRE(mmax <= MLP_S, BAMG_EINVAL, "learned interpolation: mmax must be <= 16");
    if (n == 0) return 0;
    TmpBuf<float> feat((size_t)n * MLP_F, s), Y((size_t)n * MLP_S, s);
    TmpBuf<int32_t> cand((size_t)n * MLP_S, s);
    LsOut ex;
    ex.feat = feat.get();
    ex.cand = cand.get();
    ex.greedy = false;
    const int e = interp_ls<T>(n, rp, ci, bv, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, pcol, pval, pcnt, s,
                               d_err, ex);
    if (e) return e;
    mlp_forward(model, n, feat.get(), Y.get(), s);
    BAMG_LAUNCH(k_learned_select<T>, blocks_for(n, 128), 128, 0, s, n, cf, cidx, (const int32_t*)cand.get(),
                (const float*)Y.get(), X, ncols, ld, d_w, c, refit ? 1 : 0, ridge, pcol, pval, pcnt);
    return 0;
}

// ================================================================ restriction Q
__global__ void k_q_count(int n, int c, const int32_t* __restrict__ pcol, const int32_t* __restrict__ pcnt,
                          int32_t* __restrict__ qcnt) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int t = 0; t < pcnt[i]; ++t) atomicAdd(qcnt + pcol[(int64_t)i * c + t], 1);
}
__global__ void k_q_fill(int n, int c, const int32_t* __restrict__ pcol, const int32_t* __restrict__ pcnt,
                         const int32_t* __restrict__ qrp, int32_t* __restrict__ cursor, int32_t* __restrict__ qci) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int t = 0; t < pcnt[i]; ++t) {
        const int I = pcol[(int64_t)i * c + t];
        const int pos = atomicAdd(cursor + I, 1);
        qci[qrp[I] + pos] = i;
    }
}
// Sort each row by fine index (the fill order above is arbitrary) and set the
// averaging weights 1/|J_i| (Section 4: identical entries per column, 1^T Q = 1^T).
// Rows of up to Q_SORT_REG entries are sorted in registers (one load and one store per
// entry), longer ones in place; 1 / |J_i| comes from constants where |J_i| <= 4 (every
// caliber the setup allows), the same values as the division.
constexpr int Q_SORT_REG = 16;
template <typename T>
__global__ void k_q_sort(int nc, const int32_t* __restrict__ qrp, int32_t* __restrict__ qci, T* __restrict__ qv,
                         const int32_t* __restrict__ pcnt) {
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    auto inv = [](int p) {  // 1 / p, from constants for the common p <= 4
        switch (p) {
            case 1: return (T)(1.0 / 1.0);
            case 2: return (T)(1.0 / 2.0);
            case 3: return (T)(1.0 / 3.0);
            case 4: return (T)(1.0 / 4.0);
            default: return (T)(1.0 / (double)p);
        }
    };
    const int a = qrp[I], b = qrp[I + 1];
    if (b - a <= Q_SORT_REG) {
        int v[Q_SORT_REG];
#pragma unroll
        for (int k = 0; k < Q_SORT_REG; ++k) v[k] = a + k < b ? qci[a + k] : 0x7fffffff;
#pragma unroll
        for (int k = 1; k < Q_SORT_REG; ++k)  // insertion sort, unrolled: indices stay constant
#pragma unroll
            for (int q = k; q > 0; --q) {
                const int lo = min(v[q - 1], v[q]), hi = max(v[q - 1], v[q]);
                v[q - 1] = lo;
                v[q] = hi;
            }
#pragma unroll
        for (int k = 0; k < Q_SORT_REG; ++k)
            if (a + k < b) {
                qci[a + k] = v[k];
                qv[a + k] = inv(pcnt[v[k]]);
            }
        return;
    }
    for (int p = a + 1; p < b; ++p) {
        const int v = qci[p];
        int q = p;
        while (q > a && qci[q - 1] > v) {
            qci[q] = qci[q - 1];
            --q;
        }
        qci[q] = v;
    }
    for (int p = a; p < b; ++p) qv[p] = inv(pcnt[qci[p]]);
}

template <typename T>
void build_restriction(const EllView<T>& P, int nc, DevBuf<int32_t>& qrp, DevBuf<int32_t>& qci, DevBuf<T>& qv,
                       cudaStream_t s) {
    TmpBuf<int32_t> cnt(nc, s), cursor(nc, s);
    BAMG_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * nc, s));
    BAMG_CK(cudaMemsetAsync(cursor.get(), 0, sizeof(int32_t) * nc, s));
    BAMG_LAUNCH(k_q_count, blocks_for(P.n, 256), 256, 0, s, P.n, P.c, P.pcol, P.pcnt, cnt.get());
    qrp.alloc(nc + 1);
    exclusive_scan(cnt.get(), qrp.get(), nc, s);
    const size_t nq = (size_t)P.n * P.c;  // bound: every row of P has at most c entries
    qci.alloc(nq > 0 ? nq : 1);
    qv.alloc(nq > 0 ? nq : 1);
    BAMG_LAUNCH(k_q_fill, blocks_for(P.n, 256), 256, 0, s, P.n, P.c, P.pcol, P.pcnt, qrp.get(), cursor.get(), qci.get());
    BAMG_LAUNCH(k_q_sort<T>, blocks_for(nc, 128), 128, 0, s, nc, qrp.get(), qci.get(), qv.get(), P.pcnt);
}

// ================================================================ Petrov-Galerkin
// Every product Q[I,i] M[i,j] P[j,J] is enumerated in the order (i, j, slot) for each
// coarse row I, rounded as ((q * m) * p); the products of one (I, J) are then summed in
// that order.  This is the order of the plain definition, so a CPU evaluation of the
// same sum in the same order gives the same bits.
// Products of coarse row I: sum over its Q entries i and the entries (i, j) of B of |P row j|.
// One warp per coarse row: the lanes take the Q entries, then the (i, j) pairs, 32 at a time.
constexpr int GAL_COUNT_WARPS = 4;
__global__ void __launch_bounds__(GAL_COUNT_WARPS * 32)
    k_gal_count(int nc, const int32_t* __restrict__ qrp, const int32_t* __restrict__ qci,
                const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ pcnt,
                int32_t* __restrict__ np) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int I = blockIdx.x * GAL_COUNT_WARPS + (threadIdx.x >> 5);
    if (I >= nc) return;
    const int q0 = qrp[I], q1 = qrp[I + 1];
    int s = 0;
    for (int qc = q0; qc < q1; qc += 32) {
        const int qq = qc + lane;
        const int ii = qq < q1 ? qci[qq] : 0;
        const int rb = qq < q1 ? rp[ii] : 0;
        const int rl = qq < q1 ? rp[ii + 1] - rb : 0;
        int rinc = rl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, rinc, d);
            if (lane >= d) rinc += v;
        }
        const int npairs = __shfl_sync(0xffffffffu, rinc, 31);
        for (int f0 = 0; f0 < npairs; f0 += 32) {
            const int f = f0 + lane;
            int k = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int ic = __shfl_sync(0xffffffffu, rinc, k + st - 1);
                if (ic <= f) k += st;
            }
            k = min(k, 31);
            const int p = __shfl_sync(0xffffffffu, rb, k) + f - __shfl_sync(0xffffffffu, rinc - rl, k);
            if (f < npairs) s += pcnt[ci[p]];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) np[I] = s;
}

template <typename T>
__global__ void k_gal_compact(int nc, const int32_t* __restrict__ poff, const int32_t* __restrict__ ucnt,
                              const int32_t* __restrict__ rpc, const int32_t* __restrict__ uJ, const T* __restrict__ ubv,
                              const T* __restrict__ utv, int32_t* __restrict__ ci, T* __restrict__ bv,
                              T* __restrict__ tv) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int I = blockIdx.x * GAL_COUNT_WARPS + (threadIdx.x >> 5);  // one warp per coarse row
    if (I >= nc) return;
    const int o = poff[I], d = rpc[I], cnt = ucnt[I];
    for (int u = lane; u < cnt; u += 32) {
        ci[d + u] = uJ[o + u];
        bv[d + u] = ubv[o + u];
        tv[d + u] = utv[o + u];
    }
}

// Expansion, ordering and summation of one coarse row in one warp, in shared memory: the
// lanes enumerate the row's (Q entry, B entry) pairs in order, each writing the products of
// its pair at their position in the definition order (a warp prefix sum over the pairs'
// product counts).  The products are then taken in chunks of 32 in that order: the lanes
// of a chunk that share a J are summed by the lowest one, in lane order, onto J's running
// sum (a slot in order of first appearance, found through a small open-addressing table),
// so every J sums its products in definition order; the slots are finally ranked by J.
// Rows are handled by a first kernel with room for
// GAL_CAP_S products per warp (most rows); longer rows go to a list that a second kernel
// accumulates in a hash table (below), and beyond its capacity through global memory
// with a quadratic scan.
constexpr int GAL_WARPS_S = 4;
constexpr int GAL_CAP_S = 256;  // a power of two: also the slots of the row's J table
constexpr int GAL_CAP_LOG = 8;
static_assert((1 << GAL_CAP_LOG) == GAL_CAP_S, "J table size");
constexpr int GAL_BLOCKS_L = 608;

template <typename T>
struct GalArgs {
    int nc;
    const int32_t *qrp, *qci;
    const T* qv;
    const int32_t *rp, *ci;
    const T *bv, *tv;
    const int32_t* pcol;
    const T* pval;
    const int32_t* pcnt;
    int c;
    const int32_t* poff;
    int32_t* pJ;  // global product space (rows beyond the shared capacity)
    T *pvb, *pvt;
    int32_t *ucnt, *uJ;
    T *ubv, *utv;
    uint8_t* head;
};

// One coarse row I in one warp.  local: sJ/svb/svt (products, then the row's slots), hkey
// and hval (the J table) in shared memory, GAL_CAP_S entries each (np <= GAL_CAP_S); else
// the products go to the global product space.
template <typename T>
__device__ void gal_row(const GalArgs<T>& a, int I, bool local, int* sJ, T* svb, T* svt, int* hkey,
                        unsigned char* hval) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int o = a.poff[I], np = a.poff[I + 1] - o;
    const int q0 = a.qrp[I], q1 = a.qrp[I + 1];
    int base = 0;
    for (int qc = q0; qc < q1; qc += 32) {  // the Q row's entries in chunks of 32
        // each lane one entry (fine row i, its B row's start and length), prefix of the lengths
        const int qq = qc + lane;
        const int ii = qq < q1 ? a.qci[qq] : 0;
        const int rb = qq < q1 ? a.rp[ii] : 0;
        const int rl = qq < q1 ? a.rp[ii + 1] - rb : 0;
        int rinc = rl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, rinc, d);
            if (lane >= d) rinc += v;
        }
        const int npairs = __shfl_sync(0xffffffffu, rinc, 31);
        for (int f0 = 0; f0 < npairs; f0 += 32) {
            const int f = f0 + lane;
            int k = 0;  // the chunk entry holding pair f: the first with rinc > f
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int ic = __shfl_sync(0xffffffffu, rinc, k + st - 1);
                if (ic <= f) k += st;
            }
            k = min(k, 31);
            const int i = __shfl_sync(0xffffffffu, ii, k);
            const int p = __shfl_sync(0xffffffffu, rb, k) + f - __shfl_sync(0xffffffffu, rinc - rl, k);
            const int q = qc + k;
            const int j = f < npairs ? a.ci[p] : 0;
            const int cnt = f < npairs ? a.pcnt[j] : 0;
            int incl = cnt;  // inclusive warp prefix sum of the product counts
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += v;
            }
            const int pos0 = base + incl - cnt;
            if (f < npairs) {
                const T qq_ = a.qv[q];
                const T qb = mul_rn(qq_, a.bv[p]);
                const T qt = a.tv ? mul_rn(qq_, a.tv[p]) : (j == i ? qq_ : T(0));
                for (int sl = 0; sl < cnt; ++sl) {
                    const T pv = a.pval[(int64_t)j * a.c + sl];
                    const int J = a.pcol[(int64_t)j * a.c + sl];
                    const int e = pos0 + sl;
                    if (local) {
                        sJ[e] = J;
                        svb[e] = mul_rn(qb, pv);
                        svt[e] = mul_rn(qt, pv);
                    } else {
                        a.pJ[o + e] = J;
                        a.pvb[o + e] = mul_rn(qb, pv);
                        a.pvt[o + e] = mul_rn(qt, pv);
                    }
                }
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncwarp();
    if (local) {
        for (int e = lane; e < GAL_CAP_S; e += 32) hkey[e] = 0;  // key J + 1; 0 = free
        __syncwarp();
        int U = 0;  // slots so far (U <= e0: each slot took at least one earlier product)
        for (int e0 = 0; e0 < np; e0 += 32) {
            const int e = e0 + lane;
            const int J = e < np ? sJ[e] : -1 - lane;
            const unsigned grp = __match_any_sync(0xffffffffu, J);
            const bool leader = e < np && (grp & lt) == 0u;
            bool claimed = false;
            unsigned h = 0;
            T sb = T(0), st = T(0);
            if (leader) {
                h = ((unsigned)J * 2654435761u) >> (32 - GAL_CAP_LOG);
                for (;;) {  // ends: the table has a free entry while U < GAL_CAP_S
                    const int k = hkey[h];
                    if (k == J + 1) break;
                    if (k == 0 && atomicCAS(&hkey[h], 0, J + 1) == 0) {
                        claimed = true;
                        break;
                    }
                    h = (h + 1) & (GAL_CAP_S - 1);
                }
                if (claimed) {
                    sb = svb[e];
                    st = svt[e];
                } else {  // J's slot from an earlier chunk (index < e0)
                    const int u = hval[h];
                    sb = add_rn(svb[u], svb[e]);
                    st = add_rn(svt[u], svt[e]);
                }
                for (unsigned m = grp & (grp - 1u); m; m &= m - 1u) {
                    const int pos = e0 + __ffs(m) - 1;
                    sb = add_rn(sb, svb[pos]);
                    st = add_rn(st, svt[pos]);
                }
            }
            const unsigned cb = __ballot_sync(0xffffffffu, claimed);
            __syncwarp();  // this chunk's products are read before slots overwrite them
            if (leader) {
                int u;
                if (claimed) {
                    u = U + __popc(cb & lt);  // < e0 + 32: a position already read
                    hval[h] = (unsigned char)u;
                    sJ[u] = J;
                } else {
                    u = hval[h];
                }
                svb[u] = sb;
                svt[u] = st;
            }
            U += __popc(cb);
            __syncwarp();
        }
        for (int u = lane; u < U; u += 32) {  // slot u goes to position rank(J) of the row
            const int Ju = sJ[u];
            int rank = 0;
            for (int v = 0; v < U; ++v) rank += sJ[v] < Ju;
            a.uJ[o + rank] = (int32_t)Ju;
            a.ubv[o + rank] = svb[u];
            a.utv[o + rank] = svt[u];
        }
        if (lane == 0) a.ucnt[I] = U;
        __syncwarp();
        return;
    }
    // products in global memory: quadratic scan
    for (int e = lane; e < np; e += 32) {
        const int Je = a.pJ[o + e];
        bool hd = true;
        for (int e2 = 0; e2 < e; ++e2)
            if (a.pJ[o + e2] == Je) {
                hd = false;
                break;
            }
        a.head[o + e] = hd ? 1 : 0;
    }
    __syncwarp();
    int cntu = 0;
    for (int e = lane; e < np; e += 32) {
        if (!a.head[o + e]) continue;
        ++cntu;
        const int Je = a.pJ[o + e];
        int rank = 0;
        for (int e2 = 0; e2 < np; ++e2) rank += (a.head[o + e2] && a.pJ[o + e2] < Je);
        T sb = a.pvb[o + e], st = a.pvt[o + e];
        for (int e2 = e + 1; e2 < np; ++e2)
            if (a.pJ[o + e2] == Je) {
                sb = add_rn(sb, a.pvb[o + e2]);
                st = add_rn(st, a.pvt[o + e2]);
            }
        a.uJ[o + rank] = Je;
        a.ubv[o + rank] = sb;
        a.utv[o + rank] = st;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cntu += __shfl_xor_sync(0xffffffffu, cntu, off);
    if (lane == 0) a.ucnt[I] = cntu;
    __syncwarp();
}

// rows with at most GAL_CAP_S products; the others are appended to `list`
template <typename T>
__global__ void __launch_bounds__(GAL_WARPS_S * 32)
    k_gal_small(const __grid_constant__ GalArgs<T> a, int32_t* __restrict__ list, int* __restrict__ nlist) {
    pdl_begin();
    __shared__ int sJ[GAL_WARPS_S][GAL_CAP_S], hkey[GAL_WARPS_S][GAL_CAP_S];
    __shared__ T svb[GAL_WARPS_S][GAL_CAP_S], svt[GAL_WARPS_S][GAL_CAP_S];
    __shared__ unsigned char hval[GAL_WARPS_S][GAL_CAP_S];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * GAL_WARPS_S + wid;
    if (I >= a.nc) return;
    const int np = a.poff[I + 1] - a.poff[I];
    if (np > GAL_CAP_S) {
        if (lane == 0) list[atomicAdd(nlist, 1)] = I;
        return;
    }
    gal_row<T>(a, I, true, sJ[wid], svb[wid], svt[wid], hkey[wid], hval[wid]);
}

// Long rows by accumulation instead of sorting: the products of each batch of 32 (Q, B)
// pairs are staged in definition order in shared memory; chunks of 32 staged products
// then find or claim their J in an open-addressing table (GAL_HSLOTS slots), the lanes
// that share a J in a chunk are summed by the lowest one in lane order, so every J
// accumulates its products in definition order.  The table's entries are finally sorted
// by J.  A row with more distinct J than half the table goes to the quadratic scan.
constexpr int GAL_HSLOTS = 2048;
constexpr int GAL_STAGE = 32 * 4;  // products of one batch of pairs (caliber <= 4)

template <typename T>
__device__ bool gal_row_hash(const GalArgs<T>& a, int I, int* hkey, T* hvb, T* hvt, int* sJ, T* sb_, T* st_,
                             unsigned long long* skeys) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int o = a.poff[I];
    for (int e = lane; e < GAL_HSLOTS; e += 32) {
        hkey[e] = -1;
        hvb[e] = T(0);
        hvt[e] = T(0);
    }
    __syncwarp();
    const int q0 = a.qrp[I], q1 = a.qrp[I + 1];
    int npairs = 0;
    for (int q = q0; q < q1; ++q) npairs += a.rp[a.qci[q] + 1] - a.rp[a.qci[q]];
    int used = 0;  // claimed slots
    for (int f0 = 0; f0 < npairs; f0 += 32) {
        const int f = f0 + lane;
        int q = q0, acc = 0, i = -1, p = -1;
        if (f < npairs) {
            for (; q < q1; ++q) {
                const int ii = a.qci[q], len = a.rp[ii + 1] - a.rp[ii];
                if (f < acc + len) {
                    i = ii;
                    p = a.rp[ii] + (f - acc);
                    break;
                }
                acc += len;
            }
        }
        const int j = f < npairs ? a.ci[p] : 0;
        const int cnt = f < npairs ? a.pcnt[j] : 0;
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        const int pos0 = incl - cnt, nb = __shfl_sync(0xffffffffu, incl, 31);
        if (f < npairs) {  // stage this batch's products in definition order
            const T qq = a.qv[q];
            const T qb = mul_rn(qq, a.bv[p]);
            const T qt = a.tv ? mul_rn(qq, a.tv[p]) : (j == i ? qq : T(0));
            for (int sl = 0; sl < cnt; ++sl) {
                const T pv = a.pval[(int64_t)j * a.c + sl];
                sJ[pos0 + sl] = a.pcol[(int64_t)j * a.c + sl];
                sb_[pos0 + sl] = mul_rn(qb, pv);
                st_[pos0 + sl] = mul_rn(qt, pv);
            }
        }
        __syncwarp();
        for (int e0 = 0; e0 < nb; e0 += 32) {
            const int e = e0 + lane;
            const int J = e < nb ? sJ[e] : -1 - lane;
            const unsigned grp = __match_any_sync(0xffffffffu, J);
            const bool leader = e < nb && (grp & lt) == 0u;
            bool claimed = false;
            if (leader) {
                // find or claim the slot of J (linear probing)
                unsigned h = ((unsigned)J * 2654435761u) & (GAL_HSLOTS - 1);
                int slot = -1;
                for (int probe = 0; probe < GAL_HSLOTS; ++probe) {
                    const int k = hkey[h];
                    if (k == J) {
                        slot = (int)h;
                        break;
                    }
                    if (k == -1) {
                        const int prev = atomicCAS(&hkey[h], -1, J);
                        if (prev == -1 || prev == J) {
                            slot = (int)h;
                            claimed = prev == -1;
                            break;
                        }
                    }
                    h = (h + 1) & (GAL_HSLOTS - 1);
                }
                if (slot >= 0) {
                    T vb = hvb[slot], vt = hvt[slot];
                    unsigned m = grp;
                    while (m) {  // the group's products in lane (= definition) order
                        const int l2 = __ffs(m) - 1;
                        m &= m - 1;
                        vb = add_rn(vb, sb_[e0 + l2]);
                        vt = add_rn(vt, st_[e0 + l2]);
                    }
                    hvb[slot] = vb;
                    hvt[slot] = vt;
                }
            }
            used += __popc(__ballot_sync(0xffffffffu, claimed));
            __syncwarp();
        }
        if (used > GAL_HSLOTS / 2) return false;  // too many distinct J: quadratic fallback
    }
    // compact the occupied slots, sort by J, write the row
    int u = 0;
    for (int e0 = 0; e0 < GAL_HSLOTS; e0 += 32) {
        const int e = e0 + lane;
        const bool occ = hkey[e] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, occ);
        if (occ) skeys[u + __popc(bal & lt)] = ((unsigned long long)(unsigned)hkey[e] << 32) | (unsigned)e;
        u += __popc(bal);
    }
    __syncwarp();
    int N = 32;
    while (N < u) N <<= 1;
    for (int e = u + lane; e < N; e += 32) skeys[e] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int e = lane; e < N; e += 32) {
                const int pe = e ^ jj;
                if (pe > e) {
                    const unsigned long long x = skeys[e], y = skeys[pe];
                    const bool up = (e & k) == 0;
                    if ((x > y) == up) {
                        skeys[e] = y;
                        skeys[pe] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int e = lane; e < u; e += 32) {
        const unsigned long long kk = skeys[e];
        const int slot = (int)(kk & 0xffffffffu);
        a.uJ[o + e] = (int32_t)(kk >> 32);
        a.ubv[o + e] = hvb[slot];
        a.utv[o + e] = hvt[slot];
    }
    if (lane == 0) a.ucnt[I] = u;
    __syncwarp();
    return true;
}

// the listed rows, one warp per block, persistent over the list
template <typename T>
__global__ void __launch_bounds__(32) k_gal_large(const __grid_constant__ GalArgs<T> a,
                                                  const int32_t* __restrict__ list, const int* __restrict__ nlist) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char gal_smem[];
    unsigned long long* skeys = reinterpret_cast<unsigned long long*>(gal_smem);  // GAL_HSLOTS
    T* hvb = reinterpret_cast<T*>(skeys + GAL_HSLOTS);
    T* hvt = hvb + GAL_HSLOTS;
    T* sb_ = hvt + GAL_HSLOTS;
    T* st_ = sb_ + GAL_STAGE;
    int* hkey = reinterpret_cast<int*>(st_ + GAL_STAGE);
    int* sJ = hkey + GAL_HSLOTS;
    const int cnt = *nlist;
    for (int k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int I = list[k];
        if (!gal_row_hash<T>(a, I, hkey, hvb, hvt, sJ, sb_, st_, skeys)) gal_row<T>(a, I, false, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
}

template <typename T>
void galerkin(const MatView<T>& B, const T* T_val, const int32_t* qrp, const int32_t* qci, const T* qv,
              const EllView<T>& P, int nc, GalerkinOut<T>& out, cudaStream_t s, bool defer) {
    TmpBuf<int32_t> np(nc, s), poff(nc + 1, s);
    BAMG_LAUNCH(k_gal_count, blocks_for(nc, GAL_COUNT_WARPS), GAL_COUNT_WARPS * 32, 0, s, nc, qrp, qci, B.rp, B.ci,
                P.pcnt, np.get());
    exclusive_scan(np.get(), poff.get(), nc, s);
    // bound on the product count: each entry b_ij meets at most c columns of Q and c rows of P
    const size_t bound = (size_t)B.nnz * P.c * P.c;
    BAMG_REQUIRE(bound < (size_t)INT32_MAX, BAMG_EINVAL, "galerkin: product count may overflow int32");
    const size_t tot = bound > 0 ? bound : 1;
    TmpBuf<int32_t> pJ(tot, s), uJ(tot, s), ucnt(nc, s);
    TmpBuf<T> pvb(tot, s), pvt(tot, s), ubv(tot, s), utv(tot, s);
    TmpBuf<uint8_t> head(tot, s);
    GalArgs<T> ga{nc,     qrp,    qci, qv,         B.rp,     B.ci,      B.v,       T_val,      P.pcol,   P.pval,
                  P.pcnt, P.c,    poff.get(), pJ.get(), pvb.get(), pvt.get(), ucnt.get(), uJ.get(), ubv.get(),
                  utv.get(), head.get()};
    TmpBuf<int32_t> list(nc, s);
    TmpBuf<int> nlist(1, s);
    BAMG_CK(cudaMemsetAsync(nlist.get(), 0, sizeof(int), s));
    BAMG_LAUNCH(k_gal_small<T>, blocks_for(nc, GAL_WARPS_S), GAL_WARPS_S * 32, 0, s, ga, list.get(), nlist.get());
    auto large_smem = [](size_t tb) {
        return (size_t)GAL_HSLOTS * (sizeof(unsigned long long) + 2 * tb + sizeof(int)) + GAL_STAGE * (2 * tb + sizeof(int));
    };
    const size_t smem_l = large_smem(sizeof(T));
    static std::atomic<bool> attr[256] = {};  // per device; idempotent across host threads
    int dev = 0;
    BAMG_CK(cudaGetDevice(&dev));
    BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
    if (!attr[dev]) {
        BAMG_CK(cudaFuncSetAttribute(k_gal_large<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)large_smem(sizeof(float))));
        BAMG_CK(cudaFuncSetAttribute(k_gal_large<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)large_smem(sizeof(double))));
        attr[dev] = true;
    }
    BAMG_LAUNCH(k_gal_large<T>, GAL_BLOCKS_L, 32, smem_l, s, ga, (const int32_t*)list.get(), (const int*)nlist.get());
    out.rp.alloc(nc + 1);
    size_t nz = tot;  // with defer: room for the bound, the count still on its way
    // (only while the bound's arrays stay small: large ones cost more to allocate than the wait)
    if (defer && tot * (sizeof(int32_t) + 2 * sizeof(T)) > ((size_t)64 << 20)) defer = false;
    if (defer) {
        exclusive_scan_total_begin(ucnt.get(), out.rp.get(), nc, s);
        out.nnz = -1;
    } else {
        out.nnz = exclusive_scan_total(ucnt.get(), out.rp.get(), nc, s);
        nz = out.nnz > 0 ? (size_t)out.nnz : 1;
    }
    out.ci.alloc(nz);
    out.bv.alloc(nz);
    out.tv.alloc(nz);
    BAMG_LAUNCH(k_gal_compact<T>, blocks_for(nc, GAL_COUNT_WARPS), GAL_COUNT_WARPS * 32, 0, s, nc, poff.get(),
                ucnt.get(), out.rp.get(), uJ.get(),
                ubv.get(), utv.get(), out.ci.get(), out.bv.get(), out.tv.get());
}

template <typename T>
void galerkin_nnz(GalerkinOut<T>& out, cudaStream_t s) {
    if (out.nnz < 0) out.nnz = scan_total_wait(s);
}

template <typename T>
__global__ void k_csr_to_dense(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const T* __restrict__ v, double* __restrict__ D) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) D[(int64_t)i * n + ci[p]] = (double)v[p];
}
template <typename T>
void csr_to_dense(int n, const int32_t* rp, const int32_t* ci, const T* v, double* D, cudaStream_t s) {
    BAMG_CK(cudaMemsetAsync(D, 0, sizeof(double) * n * n, s));
    if (n) BAMG_LAUNCH(k_csr_to_dense<T>, blocks_for(n, 64), 64, 0, s, n, rp, ci, v, D);
}

#define INST(T)                                                                                                     \
    template int interp_ls<T>(int, const int32_t*, const int32_t*, const T*, const uint8_t*, const int32_t*,       \
                              const T*, int, int, const double*, int, int, int, double, int32_t*, T*, int32_t*,     \
                              cudaStream_t, int*, const LsOut&);                                                    \
    template int interp_learned<T>(int, const int32_t*, const int32_t*, const T*, const uint8_t*, const int32_t*,  \
                                   const T*, int, int, const double*, int, int, int, double, const Model*, bool,    \
                                   int32_t*, T*, int32_t*, cudaStream_t, int*);                                     \
    template void build_restriction<T>(const EllView<T>&, int, DevBuf<int32_t>&, DevBuf<int32_t>&, DevBuf<T>&,      \
                                       cudaStream_t);                                                               \
    template void galerkin<T>(const MatView<T>&, const T*, const int32_t*, const int32_t*, const T*,                \
                              const EllView<T>&, int, GalerkinOut<T>&, cudaStream_t, bool);                         \
    template void galerkin_nnz<T>(GalerkinOut<T>&, cudaStream_t);                                                   \
    template void csr_to_dense<T>(int, const int32_t*, const int32_t*, const T*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace bamg
