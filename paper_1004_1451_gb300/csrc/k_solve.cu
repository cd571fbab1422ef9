// Solve phase: the V(nu1, nu2) cycle whose error propagator is Eq. (4.4),
// S^nu2 (I - P C_{l+1} Q B) S^nu1 with S = I - omega D^{-1} B and C_L = B_L^+, and the
// FP64 pieces of flexible GMRES on B x = 0 (Section 4.2): sparse products with B,
// classical Gram-Schmidt dots and updates, Givens rotations, the update x0 + Z y, and
// the true residual ||B x||_1 / ||x||_1.
#include <algorithm>
#include <atomic>
#include <utility>

#include "gmres_state.cuh"
#include "kernels.cuh"

namespace bamg {

// ---------------------------------------------------------------- V-cycle
// Per-row arithmetic shared by the grid kernels and the single-block coarse kernel, in
// the order of the plain definition: x1 = (w d^{-1}) b; x_new = x + (w d^{-1}) (b - B x);
// r = b - B x; b_c = Q r; x += P e_c.
// sum_p bv[p] * f(ci[p]) over p0 <= p < p1, accumulated in order; groups of four
// indices and gathers are issued before they are consumed so that each thread keeps
// several loads in flight.
template <typename T, typename F>
__device__ __forceinline__ T row_sum(int p0, int p1, const int32_t* __restrict__ ci, const T* __restrict__ bv, F f) {
    T s = T(0);
    int p = p0;
    for (; p + 4 <= p1; p += 4) {
        const int j0 = ci[p], j1 = ci[p + 1], j2 = ci[p + 2], j3 = ci[p + 3];
        const T b0 = bv[p], b1 = bv[p + 1], b2 = bv[p + 2], b3 = bv[p + 3];
        const T x0 = f(j0), x1 = f(j1), x2 = f(j2), x3 = f(j3);
        s += b0 * x0;
        s += b1 * x1;
        s += b2 * x2;
        s += b3 * x3;
    }
    for (; p < p1; ++p) s += bv[p] * f(ci[p]);
    return s;
}
template <typename T>
__device__ __forceinline__ T row_Bx(int i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const T* __restrict__ bv, const T* __restrict__ x) {
    return row_sum<T>(rp[i], rp[i + 1], ci, bv, [&](int j) { return x[j]; });
}
// B x1 with x1 = (w d^{-1}) b formed on the fly (the first sweep from a zero guess)
template <typename T>
__device__ __forceinline__ T row_Bx1(int i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const T* __restrict__ bv, const T* __restrict__ dinv, const T* __restrict__ b,
                                     T omega) {
    return row_sum<T>(rp[i], rp[i + 1], ci, bv, [&](int j) { return (omega * dinv[j]) * b[j]; });
}
template <typename T>
__device__ __forceinline__ T row_prolonged(int j, int c, const int32_t* __restrict__ pcol, const T* __restrict__ pval,
                                           const int32_t* __restrict__ pcnt, const T* __restrict__ ec,
                                           const T* __restrict__ x) {
    T s = T(0);
    for (int t = 0; t < pcnt[j]; ++t) s += pval[(int64_t)j * c + t] * ec[pcol[(int64_t)j * c + t]];
    return x[j] + s;
}

template <typename T>
__global__ void k_smooth0(int n, const T* __restrict__ dinv, const T* __restrict__ b, T* __restrict__ x, T omega) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (omega * dinv[i]) * b[i];
}
// two sweeps from a zero guess in one pass
template <typename T>
__global__ void k_presmooth2(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const T* __restrict__ bv, const T* __restrict__ dinv, const T* __restrict__ b,
                             T* __restrict__ y, T omega) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T x1 = (omega * dinv[i]) * b[i];
    y[i] = x1 + (omega * dinv[i]) * (b[i] - row_Bx1(i, rp, ci, bv, dinv, b, omega));
}
// one sweep; optionally also stores the result at Z + (*dj) n
template <typename T>
__global__ void k_smooth(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ bv, const T* __restrict__ dinv, const T* __restrict__ b,
                         const T* __restrict__ x, T* __restrict__ y, T omega, T* __restrict__ Z,
                         const int* __restrict__ dj) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = x[i] + (omega * dinv[i]) * (b[i] - row_Bx(i, rp, ci, bv, x));
    y[i] = v;
    if (Z) Z[(int64_t)(*dj) * n + i] = v;
}
template <typename T>
__global__ void k_resid(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const T* __restrict__ bv, const T* __restrict__ b, const T* __restrict__ x,
                        T* __restrict__ r) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - row_Bx(i, rp, ci, bv, x);
}
// The same three kernels with G lanes per row (G = 4 .. 32), for levels whose rows are
// long (the coarse levels of compatible-relaxation hierarchies): the lanes of a group take
// the entries p0 + lane, p0 + lane + G, ... and add their partial sums by a butterfly.
// Every lane of a warp takes part in the shuffles, also for rows past n.
template <int G, typename T, typename F>
__device__ __forceinline__ T row_sum_grp(int i, int n, int sub, const int32_t* __restrict__ rp,
                                         const int32_t* __restrict__ ci, const T* __restrict__ bv, F f) {
    T s = T(0);
    if (i < n)
        for (int p = rp[i] + sub; p < rp[i + 1]; p += G) s += bv[p] * f(ci[p]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}
template <typename T, int G>
__global__ void k_presmooth2_grp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const T* __restrict__ bv, const T* __restrict__ dinv, const T* __restrict__ b,
                                 T* __restrict__ y, T omega) {
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const T bx = row_sum_grp<G, T>(i, n, sub, rp, ci, bv, [&](int j) { return (omega * dinv[j]) * b[j]; });
    if (i < n && sub == 0) {
        const T x1 = (omega * dinv[i]) * b[i];
        y[i] = x1 + (omega * dinv[i]) * (b[i] - bx);
    }
}
template <typename T, int G>
__global__ void k_smooth_grp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const T* __restrict__ bv, const T* __restrict__ dinv, const T* __restrict__ b,
                             const T* __restrict__ x, T* __restrict__ y, T omega, T* __restrict__ Z,
                             const int* __restrict__ dj) {
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const T bx = row_sum_grp<G, T>(i, n, sub, rp, ci, bv, [&](int j) { return x[j]; });
    if (i < n && sub == 0) {
        const T v = x[i] + (omega * dinv[i]) * (b[i] - bx);
        y[i] = v;
        if (Z) Z[(int64_t)(*dj) * n + i] = v;
    }
}
template <typename T, int G>
__global__ void k_resid_grp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const T* __restrict__ bv, const T* __restrict__ b, const T* __restrict__ x,
                            T* __restrict__ r) {
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    const T bx = row_sum_grp<G, T>(i, n, sub, rp, ci, bv, [&](int j) { return x[j]; });
    if (i < n && sub == 0) r[i] = b[i] - bx;
}
#define BAMG_LAUNCH_GRP(G_, kern, n_, s_, ...)                                                          \
    do {                                                                                               \
        const unsigned gg_ = blocks_for((int64_t)(n_) * (G_), 256);                                    \
        switch (G_) {                                                                                  \
            case 4: BAMG_LAUNCH_PDL((kern<T, 4>), gg_, 256, 0, s_, __VA_ARGS__); break;                \
            case 8: BAMG_LAUNCH_PDL((kern<T, 8>), gg_, 256, 0, s_, __VA_ARGS__); break;                \
            case 16: BAMG_LAUNCH_PDL((kern<T, 16>), gg_, 256, 0, s_, __VA_ARGS__); break;              \
            default: BAMG_LAUNCH_PDL((kern<T, 32>), gg_, 256, 0, s_, __VA_ARGS__); break;             \
        }                                                                                              \
    } while (0)

template <typename T>
__global__ void k_restrict(int nc, const int32_t* __restrict__ qrp, const int32_t* __restrict__ qci,
                           const T* __restrict__ qv, const T* __restrict__ r, T* __restrict__ bc) {
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    bc[I] = row_sum<T>(qrp[I], qrp[I + 1], qci, qv, [&](int i) { return r[i]; });
}
template <typename T>
__global__ void k_prolong_add(int n, int c, const int32_t* __restrict__ pcol, const T* __restrict__ pval,
                              const int32_t* __restrict__ pcnt, const T* __restrict__ ec, T* __restrict__ x) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = row_prolonged(i, c, pcol, pval, pcnt, ec, x);
}
template <typename T>
__global__ void k_dense_mv(int n, const T* __restrict__ A, const T* __restrict__ b, T* __restrict__ x) {
    pdl_begin();
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    T s = T(0);
    for (int c = lane; c < n; c += 32) s += A[(int64_t)row * n + c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
}
template <typename T>
__global__ void k_copy(int n, const T* __restrict__ a, T* __restrict__ b, T* __restrict__ Z, const int* __restrict__ dj) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = a[i];
    if (Z) Z[(int64_t)(*dj) * n + i] = a[i];
}

// The coarse end of the cycle in one block: every level from the first one with at most
// TAIL_MAX_N rows and TAIL_MAX_NNZ entries down to the coarsest solve and back up, with
// block barriers between the phases instead of kernel boundaries (the levels are too
// small to fill the GPU, and each launch would cost more than its work).  Same per-row
// arithmetic and buffer sequence as the grid kernels, so the result is identical.
// The vectors of the tail levels live in shared memory, and so do the levels' matrices
// (B, D^{-1}, P, Q) and B_L^+ as far as they fit: they are copied in with cp.async at
// the start, before the wait on the preceding kernel (they do not change during a
// solve), so every later row walk reads shared memory instead of L2.
constexpr int TAIL_MAX_N = 1024;
constexpr int TAIL_MAX_NNZ = 16384;  // rows are walked serially per thread: dense levels stay on the grid
constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_MAX_LEVELS = 12;
constexpr int TAIL_SMEM = 227 * 1024;  // the opt-in maximum per block
template <typename T>
struct TailArgs {
    VLevel<T> lv[TAIL_MAX_LEVELS];
    int32_t soff[TAIL_MAX_LEVELS];  // byte offset of the level's staged matrices, -1: read from global
    int32_t pinv_off = -1;          // byte offset of the staged B_L^+, -1: read from global
    int32_t voff[TAIL_MAX_LEVELS];  // element offset of the level's vectors b, x, t in shared memory
    int nl = 0;  // levels in the tail; the last one is the coarsest
    const T* pinv = nullptr;
    int nu_pre = 0, nu_post = 0;
    T omega = T(0);
};

__host__ __device__ constexpr size_t al16(size_t b) { return (b + 15) & ~size_t(15); }
// Byte offsets of one non-coarsest level's arrays within its staged block; every array
// starts on a 16-byte boundary.
template <typename T>
struct TailLayout {
    size_t rp, ci, v, dinv, pcol, pval, pcnt, qrp, qci, qv, end;
    __host__ __device__ TailLayout(const VLevel<T>& L, int nc) {
        const size_t n = (size_t)L.B.n, nnz = (size_t)L.B.nnz, nP = n * (size_t)L.P.c, nq = (size_t)L.qnnz;
        rp = 0;
        ci = rp + al16(4 * (n + 1));
        v = ci + al16(4 * nnz);
        dinv = v + al16(sizeof(T) * nnz);
        pcol = dinv + al16(sizeof(T) * n);
        pval = pcol + al16(4 * nP);
        pcnt = pval + al16(sizeof(T) * nP);
        qrp = pcnt + al16(4 * n);
        qci = qrp + al16(4 * ((size_t)nc + 1));
        qv = qci + al16(4 * nq);
        end = qv + al16(sizeof(T) * nq);
    }
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
// Issue the copy of `bytes` (a multiple of 4) from global memory to 16-byte aligned
// shared memory: 16-byte pieces while the source is 16-byte aligned, 4-byte ones for the rest.
__device__ __forceinline__ void stage_async(unsigned char* dst, const void* src, size_t bytes) {
    const unsigned char* g = static_cast<const unsigned char*>(src);
    size_t done = 0;
    if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
        const size_t n16 = bytes >> 4;
        for (size_t k = threadIdx.x; k < n16; k += blockDim.x) cp_async16(dst + 16 * k, g + 16 * k);
        done = n16 << 4;
    }
    for (size_t k = (done >> 2) + threadIdx.x; k < (bytes >> 2); k += blockDim.x) cp_async4(dst + 4 * k, g + 4 * k);
}
// Level l of the tail with its matrix pointers moved to the staged copies.
template <typename T>
__device__ __forceinline__ VLevel<T> tail_level(const TailArgs<T>& a, int l, unsigned char* smem) {
    VLevel<T> v = a.lv[l];
    if (a.soff[l] < 0) return v;
    const TailLayout<T> o(v, a.lv[l + 1].B.n);
    unsigned char* base = smem + a.soff[l];
    v.B.rp = reinterpret_cast<const int32_t*>(base + o.rp);
    v.B.ci = reinterpret_cast<const int32_t*>(base + o.ci);
    v.B.v = reinterpret_cast<const T*>(base + o.v);
    v.dinv = reinterpret_cast<const T*>(base + o.dinv);
    v.P.pcol = reinterpret_cast<const int32_t*>(base + o.pcol);
    v.P.pval = reinterpret_cast<const T*>(base + o.pval);
    v.P.pcnt = reinterpret_cast<const int32_t*>(base + o.pcnt);
    v.qrp = reinterpret_cast<const int32_t*>(base + o.qrp);
    v.qci = reinterpret_cast<const int32_t*>(base + o.qci);
    v.qv = reinterpret_cast<const T*>(base + o.qv);
    return v;
}

// Issue the cp.async copies of the tail levels' matrices (and B_L^+) into shared memory.
template <typename T>
__device__ __forceinline__ void tail_stage(const TailArgs<T>& a, unsigned char* tail_smem) {
    for (int l = 0; l + 1 < a.nl; ++l) {
        if (a.soff[l] < 0) continue;
        const VLevel<T>& g = a.lv[l];
        const TailLayout<T> o(g, a.lv[l + 1].B.n);
        unsigned char* base = tail_smem + a.soff[l];
        const size_t n = (size_t)g.B.n, nP = n * (size_t)g.P.c;
        stage_async(base + o.rp, g.B.rp, 4 * (n + 1));
        stage_async(base + o.ci, g.B.ci, 4 * (size_t)g.B.nnz);
        stage_async(base + o.v, g.B.v, sizeof(T) * (size_t)g.B.nnz);
        stage_async(base + o.dinv, g.dinv, sizeof(T) * n);
        stage_async(base + o.pcol, g.P.pcol, 4 * nP);
        stage_async(base + o.pval, g.P.pval, sizeof(T) * nP);
        stage_async(base + o.pcnt, g.P.pcnt, 4 * n);
        stage_async(base + o.qrp, g.qrp, 4 * ((size_t)a.lv[l + 1].B.n + 1));
        stage_async(base + o.qci, g.qci, 4 * (size_t)g.qnnz);
        stage_async(base + o.qv, g.qv, sizeof(T) * (size_t)g.qnnz);
    }
    const int nL = a.lv[a.nl - 1].B.n;
    if (a.pinv_off >= 0) stage_async(tail_smem + a.pinv_off, a.pinv, sizeof(T) * (size_t)nL * nL);
}

// One pass of the V-cycle over the tail levels by one block (the staged copies complete at
// its start): reads the first tail level's b from global memory and writes that level's
// final x to the global buffer the grid kernels read it from.
template <typename T>
__device__ __forceinline__ void tail_cycle(const TailArgs<T>& a, unsigned char* tail_smem) {
    // the vectors of all tail levels: b, x and the work vector t of level l at
    // sbuf + voff[l] + {0, n, 2n}.  Which of x and t holds the iterate after the pre- (and the
    // post-) smoothing sweeps follows from the sweep counts, so the buffers are addressed from
    // the kernel parameters alone: a per-thread pointer table indexed by level would live in
    // local memory, which the large shared-memory carve-out leaves to L2.
    T* sbuf = reinterpret_cast<T*>(tail_smem);
    const int tid = threadIdx.x;
    const bool pre_sw = a.nu_pre >= 2 && ((a.nu_pre - 2) & 1);  // iterate in t after the down sweeps
    const bool post_sw = (a.nu_post & 1) != 0;                   // the up sweeps swap once more each
    for (int i = tid; i < a.lv[0].B.n; i += blockDim.x) sbuf[a.voff[0] + i] = a.lv[0].b[i];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    T* gx = a.lv[0].x;  // global buffer that receives the first tail level's result
    T* gt = a.lv[0].r;
    for (int l = 0; l + 1 < a.nl; ++l) {
        const VLevel<T> v = tail_level(a, l, tail_smem);
        const int n = v.B.n;
        T* b = sbuf + a.voff[l];
        T* x = b + n;
        T* t = b + 2 * n;
        if (a.nu_pre >= 2) {
            for (int i = tid; i < n; i += blockDim.x) {
                const T x1 = (a.omega * v.dinv[i]) * b[i];
                x[i] = x1 + (a.omega * v.dinv[i]) * (b[i] - row_Bx1(i, v.B.rp, v.B.ci, v.B.v, v.dinv, b, a.omega));
            }
            __syncthreads();
            for (int k = 2; k < a.nu_pre; ++k) {
                for (int i = tid; i < n; i += blockDim.x)
                    t[i] = x[i] + (a.omega * v.dinv[i]) * (b[i] - row_Bx(i, v.B.rp, v.B.ci, v.B.v, x));
                __syncthreads();
                T* q = x;
                x = t;
                t = q;
                if (l == 0) {
                    T* g = gx;
                    gx = gt;
                    gt = g;
                }
            }
        } else if (a.nu_pre == 1) {
            for (int i = tid; i < n; i += blockDim.x) x[i] = (a.omega * v.dinv[i]) * b[i];
            __syncthreads();
        } else {
            for (int i = tid; i < n; i += blockDim.x) x[i] = T(0);
            __syncthreads();
        }
        for (int i = tid; i < n; i += blockDim.x) t[i] = b[i] - row_Bx(i, v.B.rp, v.B.ci, v.B.v, x);
        __syncthreads();
        const int nc = a.lv[l + 1].B.n;
        T* bc = sbuf + a.voff[l + 1];
        for (int I = tid; I < nc; I += blockDim.x)
            bc[I] = row_sum<T>(v.qrp[I], v.qrp[I + 1], v.qci, v.qv, [&](int i) { return t[i]; });
        __syncthreads();
    }
    const int L = a.nl - 1;
    {  // coarsest: x = B_L^+ b, one warp per row as in the grid kernel
        const int n = a.lv[L].B.n;
        const int lane = tid & 31;
        const T* pinv = a.pinv_off >= 0 ? reinterpret_cast<const T*>(tail_smem + a.pinv_off) : a.pinv;
        const T* bL = sbuf + a.voff[L];
        T* xL = sbuf + a.voff[L] + n;
        for (int row = tid >> 5; row < n; row += blockDim.x >> 5) {
            T sum = T(0);
            for (int c = lane; c < n; c += 32) sum += pinv[(int64_t)row * n + c] * bL[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) xL[row] = sum;
        }
        __syncthreads();
    }
    for (int l = L - 1; l >= 0; --l) {
        const VLevel<T> v = tail_level(a, l, tail_smem);
        const int n = v.B.n;
        T* b = sbuf + a.voff[l];
        T* x = b + (pre_sw ? 2 : 1) * n;  // the down pass's iterate
        T* t = b + (pre_sw ? 1 : 2) * n;
        // the coarse correction: level l + 1's final iterate
        const int nc = a.lv[l + 1].B.n;
        const T* ec = sbuf + a.voff[l + 1] + (l + 1 == L ? 1 : ((pre_sw != post_sw) ? 2 : 1)) * nc;
        for (int i = tid; i < n; i += blockDim.x) x[i] = row_prolonged(i, v.P.c, v.P.pcol, v.P.pval, v.P.pcnt, ec, x);
        __syncthreads();
        for (int k = 0; k < a.nu_post; ++k) {
            for (int i = tid; i < n; i += blockDim.x)
                t[i] = x[i] + (a.omega * v.dinv[i]) * (b[i] - row_Bx(i, v.B.rp, v.B.ci, v.B.v, x));
            __syncthreads();
            T* q = x;
            x = t;
            t = q;
            if (l == 0) {
                T* g = gx;
                gx = gt;
                gt = g;
            }
        }
    }
    // the first tail level's x to the global buffer the grid kernels read it from
    const int n0 = a.lv[0].B.n;
    const T* xf = sbuf + a.voff[0] + ((a.nl > 1 && pre_sw != post_sw) ? 2 : 1) * n0;
    for (int i = tid; i < n0; i += blockDim.x) gx[i] = xf[i];
}

// Static shared memory of k_vcycle_tail: a copy of its arguments (the phases index them by
// level; from shared memory such reads are cheap).
constexpr int TAIL_STATIC = 4096;
static_assert(sizeof(TailArgs<double>) <= TAIL_STATIC && sizeof(TailArgs<double>) % 4 == 0, "tail arguments");
template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_tail(const __grid_constant__ TailArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ __align__(16) unsigned char sa_raw[sizeof(TailArgs<T>)];
    {
        const int* src = reinterpret_cast<const int*>(&a);
        int* dst = reinterpret_cast<int*>(sa_raw);
        for (int k = threadIdx.x; k < (int)(sizeof(TailArgs<T>) / 4); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const TailArgs<T>& sa = *reinterpret_cast<const TailArgs<T>*>(sa_raw);
    // the matrices first: they were written during the setup, long before this launch
    tail_stage(sa, tail_smem);
    pdl_begin();
    tail_cycle(sa, tail_smem);
}

// The buffer that holds a level's final x after the down and up passes (the sequence of
// swaps in vcycle and k_vcycle_tail).
template <typename T>
static T* final_x(const VLevel<T>& v, int nu_pre, int nu_post, bool coarsest) {
    if (coarsest) return v.x;
    T* x = v.x;
    T* t = v.r;
    for (int k = 2; k < nu_pre; ++k) std::swap(x, t);
    for (int k = 0; k < nu_post; ++k) std::swap(x, t);
    return x;
}

// One multicolour Gauss-Seidel colour: x_i <- x_i + (b_i - (B x)_i) / b_ii for the cnt states
// rows[0..cnt) of one colour, in place (no state of a colour reads another's value).
template <typename T>
__global__ void k_gs_colour(int cnt, const int32_t* __restrict__ rows, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const T* __restrict__ bv, const T* __restrict__ dinv,
                            const T* __restrict__ b, T* x) {
    pdl_begin();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    const int i = rows[k];
    const T bx = row_sum<T>(rp[i], rp[i + 1], ci, bv, [&](int j) { return x[j]; });
    x[i] = x[i] + dinv[i] * (b[i] - bx);
}

template <typename T>
static void gs_sweep(const VLevel<T>& v, bool reverse, cudaStream_t s) {
    for (int q = 0; q < v.gs_ncol; ++q) {
        const int c = reverse ? v.gs_ncol - 1 - q : q;
        const int a = v.gs_ptr[c], cnt = v.gs_ptr[c + 1] - a;
        if (cnt > 0)
            BAMG_LAUNCH_PDL(k_gs_colour<T>, blocks_for(cnt, 256), 256, 0, s, cnt, v.gs_rows + a, v.B.rp, v.B.ci,
                            v.B.v, v.dinv, (const T*)v.b, v.x);
    }
}

// The V-cycle with the multicolour Gauss-Seidel smoother: zero guess, nu_pre sweeps with
// the colours ascending, residual, restriction, recursion, B_L^+ on the coarsest level,
// prolongation, nu_post sweeps with the colours descending.  One launch per colour.
template <typename T>
static void vcycle_gs(const std::vector<VLevel<T>>& lv, const T* pinv, int nu_pre, int nu_post, cudaStream_t s, T* Z,
                      const int* dj) {
    const int L = (int)lv.size() - 1;
    for (int l = 0; l < L; ++l) {
        const VLevel<T>& v = lv[l];
        const int n = v.B.n;
        BAMG_CK(cudaMemsetAsync(v.x, 0, sizeof(T) * n, s));
        for (int k = 0; k < nu_pre; ++k) gs_sweep(v, false, s);
        BAMG_LAUNCH_PDL(k_resid<T>, blocks_for(n, 256), 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, (const T*)v.b,
                        (const T*)v.x, v.r);
        const int nc = lv[l + 1].B.n;
        BAMG_LAUNCH_PDL(k_restrict<T>, blocks_for(nc, 256), 256, 0, s, nc, v.qrp, v.qci, v.qv, (const T*)v.r,
                        lv[l + 1].b);
    }
    const int nL = lv[L].B.n;
    BAMG_LAUNCH_PDL(k_dense_mv<T>, blocks_for(nL, 4), 128, 0, s, nL, pinv, (const T*)lv[L].b, lv[L].x);
    for (int l = L - 1; l >= 0; --l) {
        const VLevel<T>& v = lv[l];
        const int n = v.B.n;
        BAMG_LAUNCH_PDL(k_prolong_add<T>, blocks_for(n, 256), 256, 0, s, n, v.P.c, v.P.pcol, v.P.pval, v.P.pcnt,
                        (const T*)lv[l + 1].x, v.x);
        for (int k = 0; k < nu_post; ++k) gs_sweep(v, true, s);
    }
    if (Z) {
        const int n = lv[0].B.n;
        BAMG_LAUNCH_PDL(k_copy<T>, blocks_for(n, 256), 256, 0, s, n, (const T*)lv[0].x, lv[0].x, Z, dj);
    }
}

// The tail levels l0..L of a hierarchy as kernel arguments: the vectors of every tail level
// in shared memory (3 n each), then the matrices of the finer tail levels (their rows are
// walked most) and B_L^+ staged while they fit in `budget` bytes; *smem = bytes used.
template <typename T>
static TailArgs<T> make_tail_args(const std::vector<VLevel<T>>& lv, int l0, const T* pinv, int nu_pre, int nu_post,
                                  T omega, size_t budget, size_t* smem_out) {
    const int L = (int)lv.size() - 1;
    TailArgs<T> a;
    a.nl = L - l0 + 1;
    for (int q = 0; q < a.nl; ++q) a.lv[q] = lv[l0 + q];
    a.pinv = pinv;
    a.nu_pre = nu_pre;
    a.nu_post = nu_post;
    a.omega = omega;
    size_t smem = 0;
    for (int q = 0; q < a.nl; ++q) {
        a.voff[q] = (int32_t)(smem / sizeof(T));
        smem += 3 * sizeof(T) * (size_t)a.lv[q].B.n;
    }
    BAMG_REQUIRE(smem <= 96 * 1024, BAMG_EINVAL, "vcycle tail: levels too large for shared memory");
    smem = al16(smem);
    for (int q = 0; q < a.nl; ++q) {
        a.soff[q] = -1;
        if (q + 1 == a.nl) continue;
        const size_t need = TailLayout<T>(a.lv[q], a.lv[q + 1].B.n).end;
        if (smem + need <= budget) {
            a.soff[q] = (int32_t)smem;
            smem += need;
        }
    }
    const size_t npinv = al16(sizeof(T) * (size_t)a.lv[a.nl - 1].B.n * a.lv[a.nl - 1].B.n);
    if (smem + npinv <= budget) {
        a.pinv_off = (int32_t)smem;
        smem += npinv;
    }
    *smem_out = smem;
    return a;
}

// ---------------------------------------------------------------- the coarse end on a cluster
// The tail levels spread over one cluster of CTAIL_CS blocks, one per SM.  Block q owns the
// rows [n q / CS, n (q + 1) / CS) of every tail level (for Q: the same split of the coarse
// rows).  Every block keeps a full copy of each tail level's vectors b, x and t.  A phase
// computes the block's own rows with the per-row arithmetic of the grid kernels (one thread
// per row, the same order of operations, so the result is identical) and stores each value
// into the copies of all blocks of the cluster (distributed shared memory).  A cluster
// barrier with release / acquire semantics then ends the phase, so every block reads the
// whole vector in the next one.  Each block stages only its own rows of B, P, Q and B_L^+,
// plus all of D^{-1}, which the first sweep reads at neighbouring rows.  The finest tail
// level may have CS times the rows of the single-block tail.
constexpr int CTAIL_CS = 8;  // blocks per cluster (the portable maximum)
constexpr int CTAIL_THREADS = 512;
constexpr int CTAIL_MAX_N = CTAIL_CS * CTAIL_THREADS;  // at most one row per thread on every level
constexpr size_t CTAIL_VEC_MAX = 96 * 1024;            // the replicated vectors of all tail levels
constexpr int CTAIL_STATIC = 12 * 1024;                // static shared memory (arguments, slices, copy list)
constexpr int CTAIL_JOBS = 16 * TAIL_MAX_LEVELS;       // copy jobs per block
constexpr int CTAIL_SUBJOB = 8192;                     // bytes per copy job at most (a multiple of 16)

template <typename T>
struct CTailArgs {
    VLevel<T> lv[TAIL_MAX_LEVELS];
    int32_t voff[TAIL_MAX_LEVELS];  // element offset of level l's b, x, t in the replicated region
    int32_t vec_bytes = 0;          // bytes of the replicated region (a multiple of 16)
    int32_t smem_bytes = 0;         // dynamic shared memory of each block
    int nl = 0;                     // levels in the tail; the last one is the coarsest
    const T* pinv = nullptr;
    int nu_pre = 0, nu_post = 0;
    T omega = T(0);
};

// One block's rows [lo, hi) of one tail level.  Every pointer addresses the element of the
// first own row (or entry), staged in shared memory or in global memory: rp[i - lo],
// ci[p - nz0], pcol[(i - lo) c + t], qrp[I - clo], qci[q - qz0], pinv[(i - lo) n + c];
// dinv covers all rows.
template <typename T>
struct CSlice {
    int lo, hi, nz0, qz0;
    const int32_t* rp;
    const int32_t* ci;
    const T* v;
    const T* dinv;
    const int32_t* pcol;
    const T* pval;
    const int32_t* pcnt;
    const int32_t* qrp;
    const int32_t* qci;
    const T* qv;
    const T* pinv;
};
struct CopyJob {
    const unsigned char* src;
    unsigned char* dst;
    int bytes;
};
static_assert(sizeof(CTailArgs<double>) + sizeof(CSlice<double>) * TAIL_MAX_LEVELS + sizeof(CopyJob) * CTAIL_JOBS +
                      sizeof(int) * (4 * TAIL_MAX_LEVELS + 1) + 64 <=
                  CTAIL_STATIC,
              "static shared memory of the cluster tail");

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every block of the cluster (the non-aligned form: the row loops before it
// may leave a warp's threads apart); stores before it are visible to all blocks after it
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// value v into element p of the same shared array in every block of the cluster
__device__ __forceinline__ void push_all(float* p, float v) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
#pragma unroll
    for (int r = 0; r < CTAIL_CS; ++r) {
        uint32_t ra;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
        asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
    }
}
__device__ __forceinline__ void push_all(double* p, double v) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
#pragma unroll
    for (int r = 0; r < CTAIL_CS; ++r) {
        uint32_t ra;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
        asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
    }
}

// Room for `bytes` copied from src into a 16-byte aligned region: the copy starts at the
// region's start plus (src mod 16), so source and destination agree modulo 16.
__host__ __device__ constexpr size_t stage_room(size_t bytes) { return al16(bytes + 16); }
// Copy job by the 32 lanes of one warp: [src, src + bytes) to dst, 16 bytes at a time where
// both are on a 16-byte boundary, 4 bytes at a time for the ragged ends.  (The block's warps
// take whole jobs, so issuing a job costs no block-wide pass; a staged array becomes jobs of
// at most CTAIL_SUBJOB bytes, so a long one still spreads over the warps.)
__device__ __forceinline__ void run_copy_warp(const CopyJob& j, int lane) {
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(j.src);
    const int head = (int)(((16 - (s0 & 15)) & 15) < (uintptr_t)j.bytes ? ((16 - (s0 & 15)) & 15) : j.bytes);
    const int n16 = (j.bytes - head) >> 4;
    const int tail0 = head + (n16 << 4);
    for (int k = lane; k < (head >> 2); k += 32) cp_async4(j.dst + 4 * k, j.src + 4 * k);
    for (int k = lane; k < n16; k += 32) cp_async16(j.dst + head + 16 * k, j.src + head + 16 * k);
    for (int k = lane; k < ((j.bytes - tail0) >> 2); k += 32) cp_async4(j.dst + tail0 + 4 * k, j.src + tail0 + 4 * k);
}

template <typename T>
__global__ void __cluster_dims__(CTAIL_CS, 1, 1) __launch_bounds__(CTAIL_THREADS)
    k_vcycle_tail_cluster(const __grid_constant__ CTailArgs<T> ga) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(16) unsigned char sa_raw[sizeof(CTailArgs<T>)];
    __shared__ CSlice<T> sl[TAIL_MAX_LEVELS];
    __shared__ CopyJob jobs[CTAIL_JOBS];
    __shared__ int plan[TAIL_MAX_LEVELS][4];  // per level: bytes to stage, arrays, offset (-1: not staged), job
    __shared__ int njobs;
    const int tid = threadIdx.x;
    {
        const int* src = reinterpret_cast<const int*>(&ga);
        int* dst = reinterpret_cast<int*>(sa_raw);
        for (int k = tid; k < (int)(sizeof(CTailArgs<T>) / 4); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const CTailArgs<T>& a = *reinterpret_cast<const CTailArgs<T>*>(sa_raw);
    const int q = (int)cluster_rank(), L = a.nl - 1;
    auto row_lo = [&](int l, int r) { return (int)(((int64_t)a.lv[l].B.n * r) / CTAIL_CS); };
    // ---- the staging plan, one thread per level (the matrices were written during the setup,
    // long before this launch, so they are read before the wait on the preceding kernel): the
    // level's own rows, their entry ranges and the arrays to stage; then thread 0 places the
    // levels in order while the budget lasts (global memory beyond); then each level's thread
    // fills in its copy jobs and shared-memory pointers.
    CSlice<T> c;
    const unsigned char* src[10];
    size_t bytes[10];
    int na = 0;
    if (tid < a.nl) {
        const int l = tid;
        const VLevel<T>& g = a.lv[l];
        const int lo = row_lo(l, q), hi = row_lo(l, q + 1), rows = hi - lo, n = g.B.n;
        c.lo = lo;
        c.hi = hi;
        c.nz0 = c.qz0 = 0;
        c.rp = c.ci = c.pcol = c.pcnt = c.qrp = c.qci = nullptr;
        c.v = c.dinv = c.pval = c.qv = c.pinv = nullptr;
        if (l < L) {
            const int clo = row_lo(l + 1, q), chi = row_lo(l + 1, q + 1), pc = g.P.c;
            const int nz0 = g.B.rp[lo], nz1 = g.B.rp[hi], qz0 = g.qrp[clo], qz1 = g.qrp[chi];
            c.nz0 = nz0;
            c.qz0 = qz0;
            c.rp = g.B.rp + lo;
            c.ci = g.B.ci + nz0;
            c.v = g.B.v + nz0;
            c.dinv = g.dinv;
            c.pcol = g.P.pcol + (int64_t)lo * pc;
            c.pval = g.P.pval + (int64_t)lo * pc;
            c.pcnt = g.P.pcnt + lo;
            c.qrp = g.qrp + clo;
            c.qci = g.qci + qz0;
            c.qv = g.qv + qz0;
            const unsigned char* s_[10] = {(const unsigned char*)c.rp,   (const unsigned char*)c.ci,
                                           (const unsigned char*)c.v,    (const unsigned char*)c.dinv,
                                           (const unsigned char*)c.pcol, (const unsigned char*)c.pval,
                                           (const unsigned char*)c.pcnt, (const unsigned char*)c.qrp,
                                           (const unsigned char*)c.qci,  (const unsigned char*)c.qv};
            const size_t b_[10] = {4 * (size_t)(rows + 1),        4 * (size_t)(nz1 - nz0),
                                   sizeof(T) * (size_t)(nz1 - nz0), sizeof(T) * (size_t)n,
                                   4 * (size_t)rows * pc,          sizeof(T) * (size_t)rows * pc,
                                   4 * (size_t)rows,               4 * (size_t)(chi - clo + 1),
                                   4 * (size_t)(qz1 - qz0),        sizeof(T) * (size_t)(qz1 - qz0)};
            for (int k = 0; k < 10; ++k) {
                src[k] = s_[k];
                bytes[k] = b_[k];
            }
            na = 10;
        } else if (a.pinv) {
            c.pinv = a.pinv + (int64_t)lo * n;
            src[0] = (const unsigned char*)c.pinv;
            bytes[0] = sizeof(T) * (size_t)rows * n;
            na = 1;
        }
        size_t need = 0;
        int nz = 0;
        for (int k = 0; k < na; ++k) {
            need += stage_room(bytes[k]);
            nz += (int)((bytes[k] + CTAIL_SUBJOB - 1) / CTAIL_SUBJOB);
        }
        plan[l][0] = na > 0 ? (int)need : -1;
        plan[l][1] = nz;
    }
    __syncthreads();
    if (tid == 0) {
        size_t off = (size_t)a.vec_bytes;
        const size_t budget = (size_t)a.smem_bytes;
        int nj = 0;
        for (int l = 0; l <= L; ++l) {
            const int need = plan[l][0], nz = plan[l][1];
            if (need >= 0 && off + (size_t)need <= budget && nj + nz <= CTAIL_JOBS) {
                plan[l][2] = (int)off;
                plan[l][3] = nj;
                off += (size_t)need;
                nj += nz;
            } else {
                plan[l][2] = -1;
            }
        }
        njobs = nj;
    }
    __syncthreads();
    if (tid < a.nl) {
        const int l = tid;
        if (plan[l][2] >= 0) {
            size_t off = (size_t)plan[l][2];
            int nj = plan[l][3];
            unsigned char* d[10];
            for (int k = 0; k < na; ++k) {
                d[k] = sm + off + (reinterpret_cast<uintptr_t>(src[k]) & 15);
                off += stage_room(bytes[k]);
                for (size_t o = 0; o < bytes[k]; o += CTAIL_SUBJOB)  // o keeps src and dst congruent mod 16
                    jobs[nj++] = CopyJob{src[k] + o, d[k] + o, (int)min((size_t)CTAIL_SUBJOB, bytes[k] - o)};
            }
            if (l < L) {
                c.rp = reinterpret_cast<const int32_t*>(d[0]);
                c.ci = reinterpret_cast<const int32_t*>(d[1]);
                c.v = reinterpret_cast<const T*>(d[2]);
                c.dinv = reinterpret_cast<const T*>(d[3]);
                c.pcol = reinterpret_cast<const int32_t*>(d[4]);
                c.pval = reinterpret_cast<const T*>(d[5]);
                c.pcnt = reinterpret_cast<const int32_t*>(d[6]);
                c.qrp = reinterpret_cast<const int32_t*>(d[7]);
                c.qci = reinterpret_cast<const int32_t*>(d[8]);
                c.qv = reinterpret_cast<const T*>(d[9]);
            } else {
                c.pinv = reinterpret_cast<const T*>(d[0]);
            }
        }
        sl[l] = c;
    }
    __syncthreads();
    {
        const int wid = tid >> 5, nw = blockDim.x >> 5, lane = tid & 31;
        for (int k = wid; k < njobs; k += nw) run_copy_warp(jobs[k], lane);
    }
    pdl_begin();
    // ---- the first tail level's right-hand side (written by the preceding kernel)
    T* sbuf = reinterpret_cast<T*>(sm);
    for (int i = tid; i < a.lv[0].B.n; i += blockDim.x) sbuf[a.voff[0] + i] = a.lv[0].b[i];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    cluster_barrier();  // every block of the cluster runs before the first remote store
    const bool pre_sw = a.nu_pre >= 2 && ((a.nu_pre - 2) & 1);
    const bool post_sw = (a.nu_post & 1) != 0;
    const T omega = a.omega;
    T* gx = a.lv[0].x;  // global buffer that receives the first tail level's result
    T* gt = a.lv[0].r;
    for (int l = 0; l < L; ++l) {
        const CSlice<T>& c = sl[l];
        const int n = a.lv[l].B.n;
        T* b = sbuf + a.voff[l];
        T* x = b + n;
        T* t = b + 2 * n;
        auto Bx = [&](int i, const T* y) {
            return row_sum<T>(c.rp[i - c.lo] - c.nz0, c.rp[i - c.lo + 1] - c.nz0, c.ci, c.v,
                              [&](int j) { return y[j]; });
        };
        if (a.nu_pre >= 2) {
            for (int i = c.lo + tid; i < c.hi; i += blockDim.x) {
                const T x1 = (omega * c.dinv[i]) * b[i];
                const T bx1 = row_sum<T>(c.rp[i - c.lo] - c.nz0, c.rp[i - c.lo + 1] - c.nz0, c.ci, c.v,
                                         [&](int j) { return (omega * c.dinv[j]) * b[j]; });
                push_all(x + i, x1 + (omega * c.dinv[i]) * (b[i] - bx1));
            }
            cluster_barrier();
            for (int k = 2; k < a.nu_pre; ++k) {
                for (int i = c.lo + tid; i < c.hi; i += blockDim.x)
                    push_all(t + i, x[i] + (omega * c.dinv[i]) * (b[i] - Bx(i, x)));
                cluster_barrier();
                T* sw = x;
                x = t;
                t = sw;
                if (l == 0) {
                    T* g = gx;
                    gx = gt;
                    gt = g;
                }
            }
        } else if (a.nu_pre == 1) {
            for (int i = c.lo + tid; i < c.hi; i += blockDim.x) push_all(x + i, (omega * c.dinv[i]) * b[i]);
            cluster_barrier();
        } else {
            for (int i = tid; i < n; i += blockDim.x) x[i] = T(0);  // every block clears its own copy
            __syncthreads();
        }
        for (int i = c.lo + tid; i < c.hi; i += blockDim.x) push_all(t + i, b[i] - Bx(i, x));
        cluster_barrier();
        const CSlice<T>& cc = sl[l + 1];
        T* bc = sbuf + a.voff[l + 1];
        for (int I = cc.lo + tid; I < cc.hi; I += blockDim.x)
            push_all(bc + I, row_sum<T>(c.qrp[I - cc.lo] - c.qz0, c.qrp[I - cc.lo + 1] - c.qz0, c.qci, c.qv,
                                        [&](int i) { return t[i]; }));
        cluster_barrier();
    }
    {  // coarsest: x = B_L^+ b, one warp per row as in the grid kernel
        const CSlice<T>& c = sl[L];
        const int n = a.lv[L].B.n, lane = tid & 31;
        const T* bL = sbuf + a.voff[L];
        T* xL = sbuf + a.voff[L] + n;
        for (int row = c.lo + (tid >> 5); row < c.hi; row += blockDim.x >> 5) {
            T sum = T(0);
            for (int col = lane; col < n; col += 32) sum += c.pinv[(int64_t)(row - c.lo) * n + col] * bL[col];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) {
                if (L == 0)
                    gx[row] = sum;
                else
                    push_all(xL + row, sum);
            }
        }
        if (L == 0) return;
        cluster_barrier();
    }
    for (int l = L - 1; l >= 0; --l) {
        const CSlice<T>& c = sl[l];
        const int n = a.lv[l].B.n, nc = a.lv[l + 1].B.n, pc = a.lv[l].P.c;
        T* b = sbuf + a.voff[l];
        T* x = b + (pre_sw ? 2 : 1) * n;  // the down pass's iterate
        T* t = b + (pre_sw ? 1 : 2) * n;
        const T* ec = sbuf + a.voff[l + 1] + (l + 1 == L ? 1 : ((pre_sw != post_sw) ? 2 : 1)) * nc;
        const bool last = (l == 0 && a.nu_post == 0);
        for (int i = c.lo + tid; i < c.hi; i += blockDim.x) {
            const int r = i - c.lo;
            T s = T(0);
            for (int k = 0; k < c.pcnt[r]; ++k) s += c.pval[(int64_t)r * pc + k] * ec[c.pcol[(int64_t)r * pc + k]];
            if (last)
                gx[i] = x[i] + s;
            else
                push_all(x + i, x[i] + s);
        }
        if (last) return;
        cluster_barrier();
        for (int k = 0; k < a.nu_post; ++k) {
            const bool fin = (l == 0 && k + 1 == a.nu_post);
            for (int i = c.lo + tid; i < c.hi; i += blockDim.x) {
                const T y = x[i] + (omega * c.dinv[i]) * (b[i] - row_sum<T>(c.rp[i - c.lo] - c.nz0,
                                                                            c.rp[i - c.lo + 1] - c.nz0, c.ci, c.v,
                                                                            [&](int j) { return x[j]; }));
                if (fin)
                    gt[i] = y;  // the buffer the swap below makes gx
                else
                    push_all(t + i, y);
            }
            if (fin) return;
            cluster_barrier();
            T* sw = x;
            x = t;
            t = sw;
            if (l == 0) {
                T* g = gx;
                gx = gt;
                gt = g;
            }
        }
    }
}

// The tail levels l0..L as arguments of the cluster kernel (the replicated vectors first;
// each block plans its own staging in the rest of `smem_bytes`).
template <typename T>
static CTailArgs<T> make_ctail_args(const std::vector<VLevel<T>>& lv, int l0, const T* pinv, int nu_pre, int nu_post,
                                    T omega, size_t smem_bytes) {
    const int L = (int)lv.size() - 1;
    CTailArgs<T> a;
    a.nl = L - l0 + 1;
    for (int q = 0; q < a.nl; ++q) a.lv[q] = lv[l0 + q];
    a.pinv = pinv;
    a.nu_pre = nu_pre;
    a.nu_post = nu_post;
    a.omega = omega;
    size_t vec = 0;
    for (int q = 0; q < a.nl; ++q) {
        a.voff[q] = (int32_t)(vec / sizeof(T));
        vec += 3 * sizeof(T) * (size_t)a.lv[q].B.n;
    }
    a.vec_bytes = (int32_t)al16(vec);
    a.smem_bytes = (int32_t)smem_bytes;
    BAMG_REQUIRE((size_t)a.vec_bytes <= smem_bytes, BAMG_EINVAL, "vcycle tail: vectors exceed shared memory");
    return a;
}

// First level of the cluster tail (L + 1: none): the finest level from which on every level
// has at most CTAIL_MAX_N rows and the replicated vectors fit.
template <typename T>
static int ctail_start(const std::vector<VLevel<T>>& lv) {
    const int L = (int)lv.size() - 1;
    for (int l = 1; l <= L; ++l) {
        if (L - l + 1 > TAIL_MAX_LEVELS || lv[l].B.n > CTAIL_MAX_N) continue;
        size_t vec = 0;
        for (int q = l; q <= L; ++q) vec += 3 * sizeof(T) * (size_t)lv[q].B.n;
        if (vec <= CTAIL_VEC_MAX) return l;
    }
    return L + 1;
}

// Whether this device runs the cluster kernel at its shared-memory size (checked once per
// device; the attribute is per device and idempotent).
template <typename T>
static bool ctail_available() {
    static std::atomic<int> state[256] = {};  // 0 unknown, 1 yes, 2 no
    int dev = 0;
    BAMG_CK(cudaGetDevice(&dev));
    BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
    int st = state[dev].load();
    if (st == 0) {
        int cl = 0;
        BAMG_CK(cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, dev));
        bool ok = cl != 0;
        if (ok)
            ok = cudaFuncSetAttribute(k_vcycle_tail_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TAIL_SMEM - CTAIL_STATIC) == cudaSuccess;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CTAIL_CS);
            cfg.blockDim = dim3(CTAIL_THREADS);
            cfg.dynamicSmemBytes = TAIL_SMEM - CTAIL_STATIC;
            int nclusters = 0;
            ok = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail_cluster<T>, &cfg) == cudaSuccess &&
                 nclusters >= 1;
        }
        cudaGetLastError();  // a refusal above is an answer, not an error of later calls
        st = ok ? 1 : 2;
        state[dev].store(st);
    }
    return st == 1;
}

// First level handled by the single-block tail (L + 1: none).
template <typename T>
static int tail_start(const std::vector<VLevel<T>>& lv) {
    const int L = (int)lv.size() - 1;
    for (int l = 1; l <= L; ++l)
        if (lv[l].B.n <= TAIL_MAX_N && lv[l].B.nnz <= TAIL_MAX_NNZ && L - l + 1 <= TAIL_MAX_LEVELS) return l;
    return L + 1;
}

template <typename T>
void vcycle(const std::vector<VLevel<T>>& lv, const T* pinv, double omega_d, int nu_pre, int nu_post, cudaStream_t s,
            T* Z, const int* dj) {
    if (lv.size() > 1 && lv[0].gs_ncol > 0) {
        vcycle_gs<T>(lv, pinv, nu_pre, nu_post, s, Z, dj);
        return;
    }
    const int L = (int)lv.size() - 1;
    const T omega = (T)omega_d;
    // the levels from l0 on run in one launch: every level from the first one with at most
    // CTAIL_MAX_N rows on a thread-block cluster (k_vcycle_tail_cluster) where the device has
    // clusters, else those from the first one with at most TAIL_MAX_N rows in one block
    // (k_vcycle_tail)
    const bool on_cluster = lv[0].tail_form == 0 && L >= 1 && ctail_available<T>();
    const int l0 = on_cluster ? ctail_start(lv) : tail_start(lv);
    std::vector<T*> xcur(L + 1), xtmp(L + 1);
    for (int l = 0; l < std::min(L, l0); ++l) {
        const VLevel<T>& v = lv[l];
        const int n = v.B.n;
        const unsigned g = blocks_for(n, 256);
        const int G = lanes_per_row(n, v.B.nnz);
        T* x = v.x;
        T* t = v.r;
        if (nu_pre >= 2) {
            if (G == 1)
                BAMG_LAUNCH_PDL(k_presmooth2<T>, g, 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, x, omega);
            else
                BAMG_LAUNCH_GRP(G, k_presmooth2_grp, n, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, x, omega);
            for (int k = 2; k < nu_pre; ++k) {
                if (G == 1)
                    BAMG_LAUNCH_PDL(k_smooth<T>, g, 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, x, t, omega,
                                    (T*)nullptr, (const int*)nullptr);
                else
                    BAMG_LAUNCH_GRP(G, k_smooth_grp, n, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, (const T*)x, t,
                                    omega, (T*)nullptr, (const int*)nullptr);
                T* q = x;
                x = t;
                t = q;
            }
        } else if (nu_pre == 1) {
            BAMG_LAUNCH_PDL(k_smooth0<T>, g, 256, 0, s, n, v.dinv, v.b, x, omega);
        } else {
            BAMG_CK(cudaMemsetAsync(x, 0, sizeof(T) * n, s));
        }
        if (G == 1)
            BAMG_LAUNCH_PDL(k_resid<T>, g, 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, v.b, x, t);
        else
            BAMG_LAUNCH_GRP(G, k_resid_grp, n, s, n, v.B.rp, v.B.ci, v.B.v, v.b, (const T*)x, t);
        const int nc = lv[l + 1].B.n;
        BAMG_LAUNCH_PDL(k_restrict<T>, blocks_for(nc, 256), 256, 0, s, nc, v.qrp, v.qci, v.qv, t, lv[l + 1].b);
        xcur[l] = x;
        xtmp[l] = t;
    }
    if (l0 <= L && on_cluster) {
        const CTailArgs<T> a = make_ctail_args(lv, l0, pinv, nu_pre, nu_post, omega, (size_t)(TAIL_SMEM - CTAIL_STATIC));
        BAMG_LAUNCH_PDL(k_vcycle_tail_cluster<T>, CTAIL_CS, CTAIL_THREADS, TAIL_SMEM - CTAIL_STATIC, s, a);
        xcur[l0] = final_x(lv[l0], nu_pre, nu_post, l0 == L);
    } else if (l0 <= L) {
        size_t smem = 0;
        const TailArgs<T> a =
            make_tail_args(lv, l0, pinv, nu_pre, nu_post, omega, (size_t)(TAIL_SMEM - TAIL_STATIC), &smem);
        // the attribute is per device: set once on each device (idempotent; several host
        // threads may get here)
        static std::atomic<bool> attr[256] = {};
        int dev = 0;
        BAMG_CK(cudaGetDevice(&dev));
        BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
        if (!attr[dev]) {
            BAMG_CK(cudaFuncSetAttribute(k_vcycle_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TAIL_SMEM - TAIL_STATIC));
            attr[dev] = true;
        }
        BAMG_LAUNCH_PDL(k_vcycle_tail<T>, 1, TAIL_THREADS, smem, s, a);
        xcur[l0] = final_x(lv[l0], nu_pre, nu_post, l0 == L);
    } else {
        const int n = lv[L].B.n;
        BAMG_LAUNCH_PDL(k_dense_mv<T>, blocks_for(n, 4), 128, 0, s, n, pinv, lv[L].b, lv[L].x);
        xcur[L] = lv[L].x;
        if (L == 0 && Z) BAMG_LAUNCH_PDL(k_copy<T>, blocks_for(n, 256), 256, 0, s, n, lv[0].x, lv[0].x, Z, dj);
    }
    for (int l = std::min(L, l0) - 1; l >= 0; --l) {
        const VLevel<T>& v = lv[l];
        const int n = v.B.n;
        const unsigned g = blocks_for(n, 256);
        T* x = xcur[l];
        T* t = xtmp[l];
        T* zl = (l == 0) ? Z : nullptr;
        const int G = lanes_per_row(n, v.B.nnz);
        BAMG_LAUNCH_PDL(k_prolong_add<T>, g, 256, 0, s, n, v.P.c, v.P.pcol, v.P.pval, v.P.pcnt, xcur[l + 1], x);
        for (int k = 0; k < nu_post; ++k) {
            if (G == 1)
                BAMG_LAUNCH_PDL(k_smooth<T>, g, 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, x, t, omega,
                                k == nu_post - 1 ? zl : (T*)nullptr, dj);
            else
                BAMG_LAUNCH_GRP(G, k_smooth_grp, n, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, v.b, (const T*)x, t, omega,
                                k == nu_post - 1 ? zl : (T*)nullptr, dj);
            T* q = x;
            x = t;
            t = q;
        }
        if (nu_post == 0 && zl) BAMG_LAUNCH_PDL(k_copy<T>, g, 256, 0, s, n, x, x, zl, dj);
        xcur[l] = x;
    }
    if (L > 0 && xcur[0] != lv[0].x)
        BAMG_LAUNCH_PDL(k_copy<T>, blocks_for(lv[0].B.n, 256), 256, 0, s, lv[0].B.n, xcur[0], lv[0].x, (T*)nullptr,
                    (const int*)nullptr);
}

// ---------------------------------------------------------------- FP64 Krylov pieces
template <typename TX>
__global__ void k_spmv64(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ bv, const TX* __restrict__ x, double* __restrict__ y, double alpha) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) s += bv[p] * (double)x[ci[p]];
    y[i] = alpha * s;
}
void spmv_f64(const MatView<double>& B, const double* x, double* y, double alpha, cudaStream_t s) {
    BAMG_LAUNCH(k_spmv64<double>, blocks_for(B.n, 256), 256, 0, s, B.n, B.rp, B.ci, B.v, x, y, alpha);
}
void spmv_f64_from_f32(const MatView<double>& B, const float* x, double* y, cudaStream_t s) {
    BAMG_LAUNCH(k_spmv64<float>, blocks_for(B.n, 256), 256, 0, s, B.n, B.rp, B.ci, B.v, x, y, 1.0);
}

constexpr int DOT_ROWS = 128;
int dots_partial_blocks(int n) { return (int)blocks_for(n, DOT_ROWS); }

__global__ void __launch_bounds__(256) k_dots_partial(int n, const double* __restrict__ V, int64_t ldv, int nv,
                                                      const double* __restrict__ w, double* __restrict__ partial) {
    pdl_begin();
    __shared__ double sw[DOT_ROWS];
    const int r0 = blockIdx.x * DOT_ROWS;
    const int cnt = min(DOT_ROWS, n - r0);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sw[e] = w[r0 + e];
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = wid; q < nv; q += nw) {
        const double* vq = V + (int64_t)q * ldv + r0;
        double acc = 0.0;
#pragma unroll 4
        for (int e = lane; e < cnt; e += 32) acc += vq[e] * sw[e];
        acc = warp_sum(acc);
        if (lane == 0) partial[(int64_t)blockIdx.x * nv + q] = acc;
    }
}

// One warp per column: lanes take the block partials in a fixed stride, then a fixed
// butterfly; the order depends only on nb, so the result is deterministic.
__global__ void k_reduce_cols(int nb, int nv, const double* __restrict__ partial, double* __restrict__ h) {
    pdl_begin();
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= nv) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += partial[(int64_t)b * nv + q];
    s = warp_sum(s);
    if (lane == 0) h[q] = s;
}

void dots(int n, const double* V, int64_t ldv, int nv, const double* w, double* d_h, double* d_partial,
          cudaStream_t s) {
    const int nb = dots_partial_blocks(n);
    BAMG_LAUNCH(k_dots_partial, nb, 256, 0, s, n, V, ldv, nv, w, d_partial);
    BAMG_LAUNCH(k_reduce_cols, blocks_for(nv, 4), 128, 0, s, nb, nv, d_partial, d_h);
}

__global__ void k_update_minus(int n, const double* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ h,
                               double* __restrict__ w) {
    pdl_begin();
    __shared__ double sh[GMRES_MMAX + 1];
    for (int q = threadIdx.x; q < nv; q += blockDim.x) sh[q] = h[q];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int q = 0; q < nv; ++q) s -= V[(int64_t)q * ldv + i] * sh[q];
    w[i] = s;
}
void update_minus(int n, const double* V, int64_t ldv, int nv, const double* d_h, double* w, cudaStream_t s) {
    BAMG_LAUNCH(k_update_minus, blocks_for(n, 256), 256, 0, s, n, V, ldv, nv, d_h, w);
}

template <typename TZ>
__global__ void k_form_x(int n, const double* __restrict__ x0, const TZ* __restrict__ Z, int64_t ldz, int nz,
                         const double* __restrict__ y, double* __restrict__ x, const int* __restrict__ dnz) {
    pdl_begin();
    if (dnz) nz = *dnz;  // the column count from device memory
    __shared__ double sy[GMRES_MMAX];
    for (int q = threadIdx.x; q < nz; q += blockDim.x) sy[q] = y[q];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int q = 0; q < nz; ++q) s += (double)Z[(int64_t)q * ldz + i] * sy[q];
    x[i] = x0[i] + s;
}
template <typename TZ>
void form_x(int n, const double* x0, const TZ* Z, int64_t ldz, int nz, const double* d_y, double* x, cudaStream_t s,
            const int* dnz) {
    BAMG_LAUNCH(k_form_x<TZ>, blocks_for(n, 256), 256, 0, s, n, x0, Z, ldz, nz, d_y, x, dnz);
}

// sums of |Bx|, (Bx)^2, |x|, x and x^2 over rows: per-block partials then a fixed-order sum.
__global__ void __launch_bounds__(256) k_resnorm_partial(int n, const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ ci, const double* __restrict__ bv,
                                                         const double* __restrict__ x, double* __restrict__ partial) {
    pdl_begin();
    __shared__ double sh[RESNORM_SUMS][8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[RESNORM_SUMS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p) s += bv[p] * x[ci[p]];
        v[0] = fabs(s);
        v[1] = s * s;
        v[2] = fabs(x[i]);
        v[3] = x[i];
        v[4] = x[i] * x[i];
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < RESNORM_SUMS; ++q) {
        const double t = warp_sum(v[q]);
        if (lane == 0) sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < RESNORM_SUMS) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * RESNORM_SUMS + threadIdx.x] = t;
    }
}
void residual_norms(const MatView<double>& B, const double* x, double* d_out, double* d_partial, cudaStream_t s) {
    const int nb = (int)blocks_for(B.n, 256);
    BAMG_LAUNCH(k_resnorm_partial, nb, 256, 0, s, B.n, B.rp, B.ci, B.v, x, d_partial);
    BAMG_LAUNCH(k_reduce_cols, blocks_for(RESNORM_SUMS, 4), 128, 0, s, nb, RESNORM_SUMS, d_partial, d_out);  // a warp per sum
}

// y = x * num or x / num with num = d_num[num_idx] (a device scalar); the quotients are
// correctly rounded from one reciprocal per block.
__global__ void k_scale_vec(int n, const double* __restrict__ x, const double* __restrict__ d_num, int num_idx,
                            int reciprocal, double* __restrict__ y) {
    pdl_begin();
    __shared__ double s_r;
    const double a = d_num[num_idx];
    if (reciprocal && threadIdx.x == 0) s_r = a != 0.0 ? 1.0 / a : 0.0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = reciprocal ? (a != 0.0 ? div_by_recip(x[i], a, s_r) : 0.0) : x[i] * a;
}
void scale_vec(int n, double* x, const double* d_num, int num_idx, bool reciprocal, double* y, cudaStream_t s) {
    BAMG_LAUNCH(k_scale_vec, blocks_for(n, 256), 256, 0, s, n, x, d_num, num_idx, reciprocal ? 1 : 0, y);
}

// Start of a cycle: beta = ||r0||_2 from nrm2, g = beta e_1; hn = beta scales v_1.
__global__ void k_gmres_init(double* __restrict__ st, int m) {
    pdl_begin();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GmresLayout L(m);
    const double beta = sqrt(st[L.nrm2]);
    for (int i = 0; i <= m; ++i) st[L.g + i] = 0.0;
    st[L.g] = beta;
    st[L.hn] = beta;
    st[L.rhn] = beta != 0.0 ? 1.0 / beta : 0.0;
    st[L.est] = beta;
}
void gmres_init(double* d_state, int m, cudaStream_t s) { BAMG_LAUNCH(k_gmres_init, 1, 32, 0, s, d_state, m); }

// y = R^{-1} g for the leading (j+1) x (j+1) block: column-oriented back substitution by
// one warp, R read from the state in global memory (column-major, consecutive lanes read
// consecutive rows of a column), y in shared memory.
__global__ void k_solve_y(double* __restrict__ st, int j, int m, const int* __restrict__ dj) {
    pdl_begin();
    if (dj) j = *dj - 1;  // the last column from device memory
    __shared__ double y[GMRES_MMAX];
    GmresLayout L(m);
    const int lane = threadIdx.x;
    const double* R = st + L.R;
    for (int r = lane; r <= j; r += 32) y[r] = st[L.g + r];
    __syncwarp();
    for (int q = j; q >= 0; --q) {
        const double* col = R + (int64_t)q * m;
        if (lane == 0) y[q] /= col[q];
        __syncwarp();
        const double yq = y[q];
        for (int r = lane; r < q; r += 32) y[r] -= col[r] * yq;
        __syncwarp();
    }
    for (int r = lane; r <= j; r += 32) st[L.y + r] = y[r];
}
void gmres_solve_y(double* d_state, int j, int m, cudaStream_t s, const int* dj) {
    BAMG_LAUNCH(k_solve_y, 1, 32, 0, s, d_state, j, m, dj);
}


// ---------------------------------------------------------------- graph-replayable Arnoldi step
// The kernels below read the Arnoldi index j from device memory (*dj), so one captured
// graph serves every iteration of a cycle: v_j = w_{j-1} / ||w_{j-1}|| -> V-cycle input,
// z_j <- V-cycle output, w = V[j+1] = B z_j, two classical Gram-Schmidt passes, ||w||, the
// Givens update and j <- j + 1 (w stays in V[j+1] unscaled until the next step scales it,
// so the step's last kernel is one block).
template <typename T>
__global__ void k_v_to_in(int n, double* __restrict__ V, const int* __restrict__ dj, const double* __restrict__ hr,
                          T* __restrict__ vin) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = *dj;
    if (i >= n) return;
    double* v = V + (int64_t)j * n;
    double vi = v[i];
    if (j > 0) {  // v_0 arrives scaled from the start of the cycle; hr = (||w||, 1 / ||w||)
        const double h = hr[0];
        vi = h != 0.0 ? div_by_recip(vi, h, hr[1]) : 0.0;  // the correctly rounded quotient
        v[i] = vi;
    }
    vin[i] = (T)vi;
}
__global__ void k_inc_j(int* dj) {
    pdl_begin();
    if (threadIdx.x == 0 && blockIdx.x == 0) *dj += 1;
}
// Fused Arnoldi kernels over row tiles (one block each).  The column sums of the per-tile
// dot products are formed again by every block that needs them (warp per column, lanes
// strided over the tiles, the same order in every block), so the reductions need no kernel
// of their own; the tile grows with n so that there are at most ARN_MAX_TILES of them.  (One
// tile per SM, which cuts the partials every block sums by 40%, measured 60 us per bench step
// slower than 256 tiles: the update's latency wants the blocks.)
constexpr int ARN_MIN_TILE = 256;
constexpr int ARN_MAX_TILES = 256;
int arn_tile_rows(int n) {
    const int64_t t = ((int64_t)n + ARN_MAX_TILES - 1) / ARN_MAX_TILES;
    return (int)std::max<int64_t>(ARN_MIN_TILE, (t + ARN_MIN_TILE - 1) / ARN_MIN_TILE * ARN_MIN_TILE);
}
int arn_tiles(int n) { return (int)blocks_for(n, arn_tile_rows(n)); }

__device__ __forceinline__ double arn_colsum(const double* __restrict__ P, int nb, int stride, int q, int lane) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += P[(int64_t)b * stride + q];
    return warp_sum(s);
}
// The column sums of the per-tile partials (nb rows of `stride`), q < ncol, formed once by the
// block of the grid that finishes last, in arn_colsum's order (so the totals are those every
// block formed for itself before): every block counts itself on *cnt after its partials are
// written and fenced; the last one sums and resets the count for the next kernel.  Every
// thread of the block calls it.
__device__ __forceinline__ void arn_last_block_sums(const double* P, int nb, int stride, int ncol,
                                                    unsigned* __restrict__ cnt, double* __restrict__ tot) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1u) == (unsigned)gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = wid; q < ncol; q += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(P + (int64_t)b * stride + q);
        s = warp_sum(s);
        if (lane == 0) tot[q] = s;
    }
    if (threadIdx.x == 0) *cnt = 0u;
}
// per-tile dots of the tile's rows of w with V[0..j] (self = 0) or with itself; the block
// has just written w, so these reads hit the caches.  Each writing lane fences after its last
// partial (arn_last_block_sums reads them from another block).
__device__ __forceinline__ void arn_tile_dots(const double* __restrict__ V, int n, int j, int r0, int cnt,
                                              const double* w, int self, double* __restrict__ Pout, int stride) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nv = self ? 1 : j + 1;
    const double* wt = w + r0;
    for (int q = wid; q < nv; q += nw) {
        const double* vq = self ? wt : V + (int64_t)q * n + r0;
        double acc = 0.0;
#pragma unroll 4
        for (int e = lane; e < cnt; e += 32) acc += vq[e] * wt[e];
        acc = warp_sum(acc);
        if (lane == 0) Pout[(int64_t)blockIdx.x * stride + q] = acc;
    }
    if (lane == 0 && wid < nv) __threadfence();  // once, after the warp's last partial
}

// w = V[j+1] = B z_j (FP64) and its per-tile dots with V[0..j]
template <typename TX>
__global__ void __launch_bounds__(256) k_arn_spmv_dots(int n, int tile, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ bv,
                                                       const TX* __restrict__ z, const int* __restrict__ dj,
                                                       double* __restrict__ V, double* __restrict__ Pout, int stride,
                                                       unsigned* __restrict__ ticket, double* __restrict__ tot) {
    pdl_begin();
    const int j = *dj;
    const int r0 = blockIdx.x * tile, cnt = min(tile, n - r0);
    double* w = V + (int64_t)(j + 1) * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = r0 + e;
        w[i] = row_sum<double>(rp[i], rp[i + 1], ci, bv, [&](int c) { return (double)z[c]; });
    }
    __syncthreads();
    arn_tile_dots(V, n, j, r0, cnt, w, 0, Pout, stride);
    if (ticket) arn_last_block_sums(Pout, gridDim.x, stride, j + 1, ticket, tot);
}

// h = column sums of Pin (block 0 stores them at hout), or with ticket the totals at hout that
// the preceding kernel's last block formed; w -= V[0..j] h; then the per-tile dots of the new
// w with V[0..j] (next_self = 0) or with itself (next_self = 1), with ticket summed by this
// kernel's last block into tot
__global__ void __launch_bounds__(256) k_arn_update_dots(int n, int tile, const int* __restrict__ dj,
                                                         double* __restrict__ V, const double* __restrict__ Pin,
                                                         int nb, double* __restrict__ hout, double* __restrict__ Pout,
                                                         int stride, int next_self, unsigned* __restrict__ ticket,
                                                         double* __restrict__ tot) {
    pdl_begin();
    __shared__ double sh[GMRES_MMAX + 1];
    const int j = *dj;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (ticket) {
        for (int q = threadIdx.x; q <= j; q += blockDim.x) sh[q] = hout[q];
    } else {
        for (int q = wid; q <= j; q += nw) {
            const double hq = arn_colsum(Pin, nb, stride, q, lane);
            if (lane == 0) {
                sh[q] = hq;
                if (blockIdx.x == 0) hout[q] = hq;
            }
        }
    }
    __syncthreads();
    const int r0 = blockIdx.x * tile, cnt = min(tile, n - r0);
    double* w = V + (int64_t)(j + 1) * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = r0 + e;
        double sacc = w[i];
#pragma unroll 8
        for (int q = 0; q <= j; ++q) sacc -= V[(int64_t)q * n + i] * sh[q];
        w[i] = sacc;
    }
    __syncthreads();
    arn_tile_dots(V, n, j, r0, cnt, w, next_self, Pout, stride);
    if (ticket) arn_last_block_sums(Pout, gridDim.x, stride, next_self ? 1 : j + 1, ticket, tot);
}

// Givens update (one thread) fused with v_{j+1} = w / ||w||: every block forms ||w|| from the
// partial sums itself (once, not per thread), so the scaling does not wait for the rotation.
__global__ void k_givens_scale_j(int n, double* __restrict__ V, const int* __restrict__ dj, double* __restrict__ st,
                                 int m, const double* __restrict__ Pn, int nb, int stride) {
    pdl_begin();
    __shared__ double col[GMRES_MMAX + 1], cs[GMRES_MMAX], sn[GMRES_MMAX], s_nrm2, s_hn, s_rhn;
    GmresLayout L(m);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = *dj;
    if (threadIdx.x < 32) {  // ||w||^2 from the per-tile partial sums
        const double nn = arn_colsum(Pn, nb, stride, 0, threadIdx.x);
        if (threadIdx.x == 0) {
            s_nrm2 = nn;
            s_hn = sqrt(nn);
            s_rhn = s_hn != 0.0 ? 1.0 / s_hn : 0.0;
            if (blockIdx.x == 0) st[L.nrm2] = nn;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        // operands staged in shared memory by the block, then the serial rotations
        for (int q = threadIdx.x; q <= j; q += blockDim.x) {
            col[q] = st[L.h1 + q] + st[L.h2 + q];
            if (q < j) {
                cs[q] = st[L.cs + q];
                sn[q] = st[L.sn + q];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double hn = sqrt(s_nrm2);
            col[j + 1] = hn;
            for (int q = 0; q < j; ++q) {
                const double c = cs[q], s = sn[q];
                const double a = col[q], b = col[q + 1];
                col[q] = c * a + s * b;
                col[q + 1] = -s * a + c * b;
            }
            const double a = col[j], b = col[j + 1];
            const double den = hypot(a, b);
            const double c = den == 0.0 ? 1.0 : a / den, s = den == 0.0 ? 0.0 : b / den;
            st[L.cs + j] = c;
            st[L.sn + j] = s;
            col[j] = c * a + s * b;
            const double gj = st[L.g + j];
            st[L.g + j + 1] = -s * gj;
            st[L.g + j] = c * gj;
            st[L.est] = fabs(st[L.g + j + 1]);
            st[L.hn] = hn;
        }
        __syncthreads();
        for (int q = threadIdx.x; q <= j; q += blockDim.x) st[L.R + q + (int64_t)j * m] = col[q];
    }
    if (i < n) {  // w / ||w|| with the block's one square root and reciprocal (correctly rounded quotients)
        double* w = V + (int64_t)(j + 1) * n;
        w[i] = s_hn != 0.0 ? div_by_recip(w[i], s_hn, s_rhn) : 0.0;
    }
}

// Givens update of Hessenberg column j (one block) with ||w||^2 at st[nrm2] (summed by the
// preceding kernel), then j += 1; with a conditional handle also the device-side loop's
// condition: go on while j < ctl[2], h_{j+1,j} != 0 and estimate * kappa > tol ||x||_1 (the
// host's test for a true residual check, with the same operands).
__global__ void k_givens_end(int* __restrict__ dj, double* __restrict__ st, int m, const double* __restrict__ ctl,
                             cudaGraphConditionalHandle cond) {
    pdl_begin();
    __shared__ double col[GMRES_MMAX + 1], cs[GMRES_MMAX], sn[GMRES_MMAX];
    GmresLayout L(m);
    const int j = *dj;
    for (int q = threadIdx.x; q <= j; q += blockDim.x) {
        col[q] = st[L.h1 + q] + st[L.h2 + q];
        if (q < j) {
            cs[q] = st[L.cs + q];
            sn[q] = st[L.sn + q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nn = st[L.nrm2], hn = sqrt(nn);
        col[j + 1] = hn;
        for (int q = 0; q < j; ++q) {
            const double c = cs[q], s = sn[q];
            const double a = col[q], b = col[q + 1];
            col[q] = c * a + s * b;
            col[q + 1] = -s * a + c * b;
        }
        const double a = col[j], b = col[j + 1];
        const double den = hypot(a, b);
        const double c = den == 0.0 ? 1.0 : a / den, s = den == 0.0 ? 0.0 : b / den;
        st[L.cs + j] = c;
        st[L.sn + j] = s;
        col[j] = c * a + s * b;
        const double gj = st[L.g + j];
        st[L.g + j + 1] = -s * gj;
        st[L.g + j] = c * gj;
        const double est = fabs(st[L.g + j + 1]);
        st[L.est] = est;
        st[L.hn] = hn;
        st[L.rhn] = hn != 0.0 ? 1.0 / hn : 0.0;
        *dj = j + 1;
        if (cond) {
            const bool stop = j + 1 >= (int)ctl[2] || hn == 0.0 || est * ctl[0] <= ctl[1];
            cudaGraphSetConditional(cond, stop ? 0u : 1u);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q <= j; q += blockDim.x) st[L.R + q + (int64_t)j * m] = col[q];
}

template <typename T>
void arnoldi_step_graphable(int n, const MatView<double>& B, double* V, T* Z, T* vin, T* zout, int* dj,
                            double* st, int m, double* partial, const std::vector<VLevel<T>>& lv,
                            const T* pinv, double omega, int nu_pre, int nu_post, double* h_est, const double* ctl,
                            cudaGraphConditionalHandle cond, cudaStream_t s) {
    GmresLayout L(m);
    const unsigned g = blocks_for(n, 256);
    const int stride = m + 1;
    BAMG_LAUNCH_PDL(k_v_to_in<T>, g, 256, 0, s, n, V, (const int*)dj, (const double*)(st + L.hn), vin);
    vcycle<T>(lv, pinv, omega, nu_pre, nu_post, s, Z, dj);
    const int tile = arn_tile_rows(n), nt = arn_tiles(n);
    double* Pa = partial;
    double* Pb = partial + (size_t)nt * stride;
    // each kernel's last block sums the per-tile partials for the next (ticket = dj + 1)
    unsigned* ticket = reinterpret_cast<unsigned*>(dj + 1);
    BAMG_LAUNCH_PDL(k_arn_spmv_dots<T>, nt, 256, 0, s, n, tile, B.rp, B.ci, B.v, (const T*)zout, (const int*)dj, V,
                    Pa, stride, ticket, st + L.h1);
    BAMG_LAUNCH_PDL(k_arn_update_dots, nt, 256, 0, s, n, tile, (const int*)dj, V, (const double*)Pa, nt, st + L.h1,
                    Pb, stride, 0, ticket, st + L.h2);
    BAMG_LAUNCH_PDL(k_arn_update_dots, nt, 256, 0, s, n, tile, (const int*)dj, V, (const double*)Pb, nt, st + L.h2,
                    Pa, stride, 1, ticket, st + L.nrm2);
    BAMG_LAUNCH_PDL(k_givens_end, 1, 64, 0, s, dj, st, m, ctl, cond);
    if (!cond) BAMG_CK(cudaMemcpyAsync(h_est, st + L.est, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

template void arnoldi_step_graphable<float>(int, const MatView<double>&, double*, float*, float*, float*, int*,
                                            double*, int, double*, const std::vector<VLevel<float>>&, const float*,
                                            double, int, int, double*, const double*, cudaGraphConditionalHandle,
                                            cudaStream_t);
template void arnoldi_step_graphable<double>(int, const MatView<double>&, double*, double*, double*, double*, int*,
                                             double*, int, double*, const std::vector<VLevel<double>>&,
                                             const double*, double, int, int, double*, const double*,
                                             cudaGraphConditionalHandle, cudaStream_t);

// ---------------------------------------------------------------- preconditioned Arnoldi
// Section 4.3: Arnoldi on the left-preconditioned matrix C B.  One step: vin = B v_j in
// FP64 rounded to the V-cycle's arithmetic, z = C vin (one V-cycle), w = V[j+1] = z in
// FP64 with its per-tile dots against V[0..j]; the two Gram-Schmidt passes and the
// scaling are the FGMRES kernels'; the raw Hessenberg column is kept in H.
template <typename T>
__global__ void k_parn_bv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ bv, const double* __restrict__ V, const int* __restrict__ dj,
                          T* __restrict__ vin) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* v = V + (int64_t)(*dj) * n;
    vin[i] = (T)row_sum<double>(rp[i], rp[i + 1], ci, bv, [&](int c) { return v[c]; });
}

template <typename TX>
__global__ void __launch_bounds__(256) k_parn_store_dots(int n, int tile, const TX* __restrict__ z,
                                                         const int* __restrict__ dj, double* __restrict__ V,
                                                         double* __restrict__ Pout, int stride) {
    pdl_begin();
    const int j = *dj;
    const int r0 = blockIdx.x * tile, cnt = min(tile, n - r0);
    double* w = V + (int64_t)(j + 1) * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) w[r0 + e] = (double)z[r0 + e];
    __syncthreads();
    arn_tile_dots(V, n, j, r0, cnt, w, 0, Pout, stride);
}

// H[0..j, j] = h1 + h2 (the two Gram-Schmidt passes), H[j+1, j] = ||w||; column-major, ld ldh
__global__ void k_parn_hess(const double* __restrict__ st, int m, const int* __restrict__ dj, double* __restrict__ H,
                            int ldh) {
    pdl_begin();
    const GmresLayout L(m);
    const int j = *dj;
    for (int r = threadIdx.x; r <= j; r += blockDim.x) H[r + (int64_t)j * ldh] = st[L.h1 + r] + st[L.h2 + r];
    if (threadIdx.x == 0) H[j + 1 + (int64_t)j * ldh] = sqrt(st[L.nrm2]);
}

// Eigenvector of the k x k upper Hessenberg H_k for its eigenvalue closest to 0 (Section 4.3),
// by inverse iteration with shift 0: H_k = L U by Gaussian elimination with partial
// pivoting between neighbouring rows (a Hessenberg column has one sub-diagonal entry),
// then up to PARN_INV_ITERS solves from the all-ones vector, each normalised to unit
// 2-norm with its largest-modulus entry positive, until two iterates agree to 1e-15.  A
// zero pivot is replaced by 2^-52 times the largest entry of H_k (the matrix is singular
// to working precision exactly when the Ritz value is 0).  One block, k <= PARN_MMAX.
constexpr int PARN_INV_ITERS = 50;
__global__ void __launch_bounds__(128) k_ritz_hess(const double* __restrict__ H, int ldh, int k,
                                                   double* __restrict__ eta) {
    pdl_begin();
    __shared__ double A[PARN_MMAX][PARN_MMAX + 1];
    __shared__ double mult[PARN_MMAX], y[PARN_MMAX], prev[PARN_MMAX];
    __shared__ int swp[PARN_MMAX];
    __shared__ double s_scale, s_norm;
    __shared__ int s_done;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < k * k; e += blockDim.x) {
        const int r = e % k, c = e / k;
        A[r][c] = H[r + (int64_t)c * ldh];
    }
    __syncthreads();
    if (wid == 0) {
        double mx = 0.0;
        for (int e = lane; e < k * k; e += 32) mx = fmax(mx, fabs(A[e % k][e / k]));
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_scale = mx > 0.0 ? mx * 0x1p-52 : 0x1p-1022;
    }
    __syncthreads();
    for (int c = 0; c + 1 < k; ++c) {
        if (tid == 0) swp[c] = fabs(A[c + 1][c]) > fabs(A[c][c]) ? 1 : 0;
        __syncthreads();
        if (swp[c])
            for (int q = c + tid; q < k; q += blockDim.x) {
                const double t = A[c][q];
                A[c][q] = A[c + 1][q];
                A[c + 1][q] = t;
            }
        __syncthreads();
        if (tid == 0) {
            if (A[c][c] == 0.0) A[c][c] = s_scale;
            mult[c] = A[c + 1][c] / A[c][c];
        }
        __syncthreads();
        for (int q = c + 1 + tid; q < k; q += blockDim.x) A[c + 1][q] -= mult[c] * A[c][q];
        __syncthreads();
    }
    if (tid == 0 && A[k - 1][k - 1] == 0.0) A[k - 1][k - 1] = s_scale;
    for (int r = tid; r < k; r += blockDim.x) {
        y[r] = 1.0 / sqrt((double)k);
        prev[r] = y[r];
    }
    if (tid == 0) s_done = 0;
    __syncthreads();
    for (int t = 0; t < PARN_INV_ITERS && !s_done; ++t) {
        if (wid == 0) {
            if (lane == 0)  // the row operations of the factorisation on the right-hand side
                for (int c = 0; c + 1 < k; ++c) {
                    if (swp[c]) {
                        const double q = y[c];
                        y[c] = y[c + 1];
                        y[c + 1] = q;
                    }
                    y[c + 1] -= mult[c] * y[c];
                }
            __syncwarp();
            for (int q = k - 1; q >= 0; --q) {  // U y = y, column by column
                if (lane == 0) y[q] /= A[q][q];
                __syncwarp();
                const double yq = y[q];
                for (int r = lane; r < q; r += 32) y[r] -= A[r][q] * yq;
                __syncwarp();
            }
            double ss = 0.0, big = 0.0;
            int at = 0;
            for (int r = lane; r < k; r += 32) {
                ss += y[r] * y[r];
                if (fabs(y[r]) > big) big = fabs(y[r]), at = r;
            }
            for (int o = 16; o; o >>= 1) {
                ss += __shfl_xor_sync(0xffffffffu, ss, o);
                const double ob = __shfl_xor_sync(0xffffffffu, big, o);
                const int oa = __shfl_xor_sync(0xffffffffu, at, o);
                if (ob > big || (ob == big && oa < at)) big = ob, at = oa;
            }
            const double sc = (y[at] < 0.0 ? -1.0 : 1.0) / sqrt(ss);
            double dif = 0.0;
            for (int r = lane; r < k; r += 32) {
                y[r] *= sc;
                dif = fmax(dif, fabs(y[r] - prev[r]));
                prev[r] = y[r];
            }
            for (int o = 16; o; o >>= 1) dif = fmax(dif, __shfl_xor_sync(0xffffffffu, dif, o));
            if (lane == 0) {
                s_norm = ss;
                s_done = (t > 0 && dif <= 1e-15) ? 1 : 0;
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < k; r += blockDim.x) eta[r] = y[r];
}

template <typename T>
void parnoldi_step(int n, const MatView<double>& B, double* V, T* vin, T* zout, int* dj, double* st, int m,
                   double* H, int ldh, double* partial, const std::vector<VLevel<T>>& lv, const T* pinv, double omega,
                   int nu_pre, int nu_post, cudaStream_t s) {
    GmresLayout L(m);
    const unsigned g = blocks_for(n, 256);
    const int stride = m + 1;
    BAMG_LAUNCH_PDL(k_parn_bv<T>, g, 256, 0, s, n, B.rp, B.ci, B.v, (const double*)V, (const int*)dj, vin);
    vcycle<T>(lv, pinv, omega, nu_pre, nu_post, s, (T*)nullptr, (const int*)nullptr);
    const int tile = arn_tile_rows(n), nt = arn_tiles(n);
    double* Pa = partial;
    double* Pb = partial + (size_t)nt * stride;
    BAMG_LAUNCH_PDL(k_parn_store_dots<T>, nt, 256, 0, s, n, tile, (const T*)zout, (const int*)dj, V, Pa, stride);
    BAMG_LAUNCH_PDL(k_arn_update_dots, nt, 256, 0, s, n, tile, (const int*)dj, V, (const double*)Pa, nt, st + L.h1,
                    Pb, stride, 0, (unsigned*)nullptr, (double*)nullptr);
    BAMG_LAUNCH_PDL(k_arn_update_dots, nt, 256, 0, s, n, tile, (const int*)dj, V, (const double*)Pb, nt, st + L.h2,
                    Pa, stride, 1, (unsigned*)nullptr, (double*)nullptr);
    BAMG_LAUNCH_PDL(k_givens_scale_j, g, 256, 0, s, n, V, (const int*)dj, st, m, (const double*)Pa, nt, stride);
    BAMG_LAUNCH_PDL(k_parn_hess, 1, 64, 0, s, (const double*)st, m, (const int*)dj, H, ldh);
    BAMG_LAUNCH_PDL(k_inc_j, 1, 32, 0, s, dj);
}
template void parnoldi_step<float>(int, const MatView<double>&, double*, float*, float*, int*, double*, int, double*,
                                   int, double*, const std::vector<VLevel<float>>&, const float*, double, int, int,
                                   cudaStream_t);
template void parnoldi_step<double>(int, const MatView<double>&, double*, double*, double*, int*, double*, int,
                                    double*, int, double*, const std::vector<VLevel<double>>&, const double*, double,
                                    int, int, cudaStream_t);

void ritz_closest_to_zero(const double* H, int ldh, int k, double* eta, cudaStream_t s) {
    BAMG_REQUIRE(k >= 1 && k <= PARN_MMAX, BAMG_EINVAL, "pArnoldi: Hessenberg order out of range");
    BAMG_LAUNCH(k_ritz_hess, 1, 128, 0, s, H, ldh, k, eta);
}

// ---------------------------------------------------------------- persistent Arnoldi cycle
// FGMRES Arnoldi steps of one restart cycle in a single cooperative launch: the same phases
// as the captured step (v_j to the V-cycle's precision, the V-cycle's grid levels, the
// single-block tail on block 0, the FP64 SpMV with the first Gram-Schmidt dots, two update
// passes, the Givens update with the scaling of v_{j+1}, the stop test of k_givens_end), with
// a grid-wide barrier between phases instead of a kernel boundary.  The per-row arithmetic,
// the row tiles of the Arnoldi kernels and every reduction order are those of the separate
// kernels, so the iterates are bit-identical.  Vectors written inside the kernel are read
// through plain pointers (never the read-only path); the matrices are read-only.
constexpr int PERSIST_THREADS = TAIL_THREADS;
constexpr int PERSIST_MAX_LEVELS = 24;
constexpr unsigned long long GRID_BAR_SPIN_LIMIT = 1ull << 24;  // then the barrier gives up

template <typename T>
struct CycleArgs {
    VLevel<T> lv[PERSIST_MAX_LEVELS];
    int L = 0, l0 = 0;
    const T* pinv = nullptr;
    TailArgs<T> tail;
    T omega = T(0);
    int nu_pre = 0, nu_post = 0;
    MatView<double> B;
    double* V = nullptr;
    T* Z = nullptr;
    T* vin = nullptr;
    double* st = nullptr;
    double* partial = nullptr;
    int m = 0, tile = 0, nt = 0;
    int* dj = nullptr;
    const double* ctl = nullptr;  // kappa, tol ||x||_1, last j + 1
    unsigned* bar = nullptr;      // arrivals, generation
    int* err = nullptr;           // 1 when a barrier wait gave up
};

// Grid-wide barrier of a cooperative launch: arrival counter and generation in global
// memory.  The block barrier orders every thread's writes before thread 0's fence and
// arrival (release), and thread 0's fence after it sees the new generation before the
// block's later reads (acquire).  The wait polls tightly, then backs off, and gives up
// after GRID_BAR_SPIN_LIMIT polls (or when another block gave up): it sets *err and
// returns false.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long polls = 0;
            while (*gen == g0) {
                if (*(volatile int*)err) break;
                if (++polls > GRID_BAR_SPIN_LIMIT) {
                    atomicExch(err, 1);
                    break;
                }
                if (polls > 512) __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)err == 0;
}

template <typename T>
__device__ __forceinline__ T prow_Bx(int i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const T* __restrict__ bv, const T* x) {
    return row_sum<T>(rp[i], rp[i + 1], ci, bv, [&](int j) { return x[j]; });
}

template <typename T>
__global__ void __launch_bounds__(PERSIST_THREADS, 1) k_arnoldi_cycle(const __grid_constant__ CycleArgs<T> a) {
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ double sh[GMRES_MMAX + 1];
    __shared__ double gcol[GMRES_MMAX + 1], gcs[GMRES_MMAX], gsn[GMRES_MMAX], s_nrm2;
    const bool has_tail = a.l0 <= a.L;
    if (has_tail && blockIdx.x == 0) tail_stage(a.tail, psm);
    pdl_begin();
    const int n = a.lv[0].B.n;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const GmresLayout GL(a.m);
    const int stride = a.m + 1;
    const T omega = a.omega;
    const int Lg = a.L < a.l0 ? a.L : a.l0;  // grid levels 0 .. Lg-1
    int j = *a.dj;
    for (;;) {
        // ---- v_j in the V-cycle's precision
        for (int i = gtid; i < n; i += gsz) a.vin[i] = (T)a.V[(int64_t)j * n + i];
        if (!grid_sync(a.bar, a.err)) return;
        // ---- V-cycle, down (the buffer sequence of vcycle())
        T* xcur[PERSIST_MAX_LEVELS];
        T* xtmp[PERSIST_MAX_LEVELS];
        for (int l = 0; l < Lg; ++l) {
            const VLevel<T>& v = a.lv[l];
            const int nl = v.B.n;
            T* b = l == 0 ? a.vin : v.b;
            T* x = v.x;
            T* t = v.r;
            if (a.nu_pre >= 2) {
                for (int i = gtid; i < nl; i += gsz) {
                    const T x1 = (omega * v.dinv[i]) * b[i];
                    x[i] = x1 + (omega * v.dinv[i]) *
                                    (b[i] - row_sum<T>(v.B.rp[i], v.B.rp[i + 1], v.B.ci, v.B.v,
                                                       [&](int c) { return (omega * v.dinv[c]) * b[c]; }));
                }
                if (!grid_sync(a.bar, a.err)) return;
                for (int k = 2; k < a.nu_pre; ++k) {
                    for (int i = gtid; i < nl; i += gsz)
                        t[i] = x[i] + (omega * v.dinv[i]) * (b[i] - prow_Bx(i, v.B.rp, v.B.ci, v.B.v, x));
                    if (!grid_sync(a.bar, a.err)) return;
                    T* q = x;
                    x = t;
                    t = q;
                }
            } else if (a.nu_pre == 1) {
                for (int i = gtid; i < nl; i += gsz) x[i] = (omega * v.dinv[i]) * b[i];
                if (!grid_sync(a.bar, a.err)) return;
            } else {
                for (int i = gtid; i < nl; i += gsz) x[i] = T(0);
                if (!grid_sync(a.bar, a.err)) return;
            }
            for (int i = gtid; i < nl; i += gsz) t[i] = b[i] - prow_Bx(i, v.B.rp, v.B.ci, v.B.v, x);
            if (!grid_sync(a.bar, a.err)) return;
            const int nc = a.lv[l + 1].B.n;
            T* bc = a.lv[l + 1].b;
            for (int I = gtid; I < nc; I += gsz)
                bc[I] = row_sum<T>(v.qrp[I], v.qrp[I + 1], v.qci, v.qv, [&](int i) { return t[i]; });
            if (!grid_sync(a.bar, a.err)) return;
            xcur[l] = x;
            xtmp[l] = t;
        }
        // ---- the coarse end: the single-block tail, or B_L^+ by the grid
        if (has_tail) {
            if (blockIdx.x == 0) tail_cycle(a.tail, psm);
            if (!grid_sync(a.bar, a.err)) return;
            xcur[a.l0] = a.tail.lv[0].x;  // set below from the tail's buffer bookkeeping
        } else {
            const int nL = a.lv[a.L].B.n;
            T* bL = a.L == 0 ? a.vin : a.lv[a.L].b;
            for (int row = gtid >> 5; row < nL; row += gsz >> 5) {
                T sum = T(0);
                for (int c = lane; c < nL; c += 32) sum += a.pinv[(int64_t)row * nL + c] * bL[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0) a.lv[a.L].x[row] = sum;
            }
            if (!grid_sync(a.bar, a.err)) return;
            xcur[a.L] = a.lv[a.L].x;
        }
        if (has_tail) {  // the buffer the tail left the first tail level's x in (final_x)
            const VLevel<T>& v = a.lv[a.l0];
            if (a.l0 == a.L) {
                xcur[a.l0] = v.x;
            } else {
                T* x = v.x;
                T* t = v.r;
                for (int k = 2; k < a.nu_pre; ++k) {
                    T* q = x;
                    x = t;
                    t = q;
                }
                for (int k = 0; k < a.nu_post; ++k) {
                    T* q = x;
                    x = t;
                    t = q;
                }
                xcur[a.l0] = x;
            }
        }
        // ---- V-cycle, up
        for (int l = Lg - 1; l >= 0; --l) {
            const VLevel<T>& v = a.lv[l];
            const int nl = v.B.n;
            T* b = l == 0 ? a.vin : v.b;
            T* x = xcur[l];
            T* t = xtmp[l];
            T* zl = l == 0 ? a.Z : nullptr;
            const T* ec = xcur[l + 1];
            for (int i = gtid; i < nl; i += gsz) {
                T s = T(0);
                for (int q = 0; q < v.P.pcnt[i]; ++q)
                    s += v.P.pval[(int64_t)i * v.P.c + q] * ec[v.P.pcol[(int64_t)i * v.P.c + q]];
                x[i] = x[i] + s;
            }
            if (!grid_sync(a.bar, a.err)) return;
            for (int k = 0; k < a.nu_post; ++k) {
                T* zk = k == a.nu_post - 1 ? zl : nullptr;
                for (int i = gtid; i < nl; i += gsz) {
                    const T val = x[i] + (omega * v.dinv[i]) * (b[i] - prow_Bx(i, v.B.rp, v.B.ci, v.B.v, x));
                    t[i] = val;
                    if (zk) zk[(int64_t)j * nl + i] = val;
                }
                if (!grid_sync(a.bar, a.err)) return;
                T* q = x;
                x = t;
                t = q;
            }
            if (a.nu_post == 0 && zl) {
                for (int i = gtid; i < nl; i += gsz) zl[(int64_t)j * nl + i] = x[i];
                if (!grid_sync(a.bar, a.err)) return;
            }
            xcur[l] = x;
        }
        const T* z = a.L == 0 ? a.lv[0].x : xcur[0];
        if (a.L == 0 && a.Z) {
            for (int i = gtid; i < n; i += gsz) a.Z[(int64_t)j * n + i] = z[i];
            if (!grid_sync(a.bar, a.err)) return;
        }
        // ---- w = V[j+1] = B z (FP64) and its per-tile dots with V[0..j]
        double* w = a.V + (int64_t)(j + 1) * n;
        double* Pa = a.partial;
        double* Pb = a.partial + (size_t)a.nt * stride;
        for (int tl = blockIdx.x; tl < a.nt; tl += gridDim.x) {
            const int r0 = tl * a.tile, cnt = min(a.tile, n - r0);
            for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
                const int i = r0 + e;
                w[i] = row_sum<double>(a.B.rp[i], a.B.rp[i + 1], a.B.ci, a.B.v, [&](int c) { return (double)z[c]; });
            }
            __syncthreads();
            for (int q = wid; q <= j; q += nw) {
                const double* vq = a.V + (int64_t)q * n + r0;
                double acc = 0.0;
                for (int e = lane; e < cnt; e += 32) acc += vq[e] * w[r0 + e];
                acc = warp_sum(acc);
                if (lane == 0) Pa[(int64_t)tl * stride + q] = acc;
            }
            __syncthreads();
        }
        if (!grid_sync(a.bar, a.err)) return;
        // ---- two classical Gram-Schmidt passes: h = column sums of Pin; w -= V[0..j] h; dots
        for (int pass = 0; pass < 2; ++pass) {
            const double* Pin = pass == 0 ? Pa : Pb;
            double* Pout = pass == 0 ? Pb : Pa;
            double* hout = a.st + (pass == 0 ? GL.h1 : GL.h2);
            for (int q = wid; q <= j; q += nw) {
                double sacc = 0.0;
                for (int bb = lane; bb < a.nt; bb += 32) sacc += Pin[(int64_t)bb * stride + q];
                sacc = warp_sum(sacc);
                if (lane == 0) {
                    sh[q] = sacc;
                    if (blockIdx.x == 0) hout[q] = sacc;
                }
            }
            __syncthreads();
            for (int tl = blockIdx.x; tl < a.nt; tl += gridDim.x) {
                const int r0 = tl * a.tile, cnt = min(a.tile, n - r0);
                for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
                    const int i = r0 + e;
                    double sacc = w[i];
                    for (int q = 0; q <= j; ++q) sacc -= a.V[(int64_t)q * n + i] * sh[q];
                    w[i] = sacc;
                }
                __syncthreads();
                const int nv = pass == 1 ? 1 : j + 1;
                for (int q = wid; q < nv; q += nw) {
                    const double* vq = pass == 1 ? w + r0 : a.V + (int64_t)q * n + r0;
                    double acc = 0.0;
                    for (int e = lane; e < cnt; e += 32) acc += vq[e] * w[r0 + e];
                    acc = warp_sum(acc);
                    if (lane == 0) Pout[(int64_t)tl * stride + q] = acc;
                }
                __syncthreads();
            }
            if (!grid_sync(a.bar, a.err)) return;
        }
        // ---- ||w||, the Givens update (block 0) and v_{j+1} = w / ||w|| (every block)
        if (wid == 0) {
            double nn = 0.0;
            for (int bb = lane; bb < a.nt; bb += 32) nn += Pa[(int64_t)bb * stride];
            nn = warp_sum(nn);
            if (lane == 0) s_nrm2 = nn;
        }
        __syncthreads();
        if (blockIdx.x == 0) {
            double* st = a.st;
            if (threadIdx.x == 0) st[GL.nrm2] = s_nrm2;
            for (int q = threadIdx.x; q <= j; q += blockDim.x) {
                gcol[q] = st[GL.h1 + q] + st[GL.h2 + q];
                if (q < j) {
                    gcs[q] = st[GL.cs + q];
                    gsn[q] = st[GL.sn + q];
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                const double hn = sqrt(s_nrm2);
                gcol[j + 1] = hn;
                for (int q = 0; q < j; ++q) {
                    const double c = gcs[q], sn = gsn[q];
                    const double x0 = gcol[q], x1 = gcol[q + 1];
                    gcol[q] = c * x0 + sn * x1;
                    gcol[q + 1] = -sn * x0 + c * x1;
                }
                const double x0 = gcol[j], x1 = gcol[j + 1];
                const double den = hypot(x0, x1);
                const double c = den == 0.0 ? 1.0 : x0 / den, sn = den == 0.0 ? 0.0 : x1 / den;
                st[GL.cs + j] = c;
                st[GL.sn + j] = sn;
                gcol[j] = c * x0 + sn * x1;
                const double gj = st[GL.g + j];
                st[GL.g + j + 1] = -sn * gj;
                st[GL.g + j] = c * gj;
                st[GL.est] = fabs(st[GL.g + j + 1]);
                st[GL.hn] = hn;
                st[GL.rhn] = hn != 0.0 ? 1.0 / hn : 0.0;
            }
            __syncthreads();
            for (int q = threadIdx.x; q <= j; q += blockDim.x) st[GL.R + q + (int64_t)j * a.m] = gcol[q];
        }
        {  // w / ||w||, the square root and the reciprocal formed once per thread (both are long
           // instruction sequences at GB300's FP64 rate); the quotients correctly rounded, as
           // the plain algorithm's w / h_{j+1,j}
            const double hn = sqrt(s_nrm2), rhn = hn != 0.0 ? 1.0 / hn : 0.0;
            for (int i = gtid; i < n; i += gsz) w[i] = hn != 0.0 ? div_by_recip(w[i], hn, rhn) : 0.0;
        }
        if (!grid_sync(a.bar, a.err)) return;
        // ---- the stop test of k_givens_end, taken by every block on the same values
        const int jn = j + 1;
        const double est = *(volatile double*)(a.st + GL.est), hn = *(volatile double*)(a.st + GL.hn);
        const bool stop = jn >= (int)a.ctl[2] || hn == 0.0 || est * a.ctl[0] <= a.ctl[1];
        j = jn;
        if (stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *a.dj = jn;
            return;
        }
    }
}

// Launches k_arnoldi_cycle for the steps *dj .. until its stop test (ctl) on stream s.
// Returns false, launching nothing, when the hierarchy or the device does not qualify:
// a grid level with long rows (the lane-group kernels), more than PERSIST_MAX_LEVELS
// levels, a tail that does not fit beside the kernel's own shared memory, or no
// cooperative launch of one 1024-thread block per SM.
template <typename T>
bool arnoldi_cycle_persistent(int n, const MatView<double>& B, double* V, T* Z, T* vin, int* dj, double* st, int m,
                              double* partial, const std::vector<VLevel<T>>& lv, const T* pinv, double omega,
                              int nu_pre, int nu_post, const double* ctl, unsigned* bar, int* err, cudaStream_t s) {
    const int L = (int)lv.size() - 1;
    if (L + 1 > PERSIST_MAX_LEVELS) return false;
    const int l0 = tail_start(lv);
    if (lv[0].gs_ncol > 0) return false;  // the multicolour Gauss-Seidel smoother runs in the graph form
    for (int l = 0; l < std::min(L, l0); ++l)
        if (lanes_per_row(lv[l].B.n, lv[l].B.nnz) != 1) return false;
    int dev = 0, sms = 0, coop = 0;
    BAMG_CK(cudaGetDevice(&dev));
    BAMG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BAMG_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop || sms <= 0) return false;
    cudaFuncAttributes fa{};
    BAMG_CK(cudaFuncGetAttributes(&fa, k_arnoldi_cycle<T>));
    const size_t budget = (size_t)TAIL_SMEM - fa.sharedSizeBytes - 1024;
    CycleArgs<T> a;
    a.L = L;
    a.l0 = l0;
    for (int l = 0; l <= L; ++l) a.lv[l] = lv[l];
    a.pinv = pinv;
    size_t smem = 0;
    if (l0 <= L) {
        size_t need = 0;
        for (int q = l0; q <= L; ++q) need += 3 * sizeof(T) * (size_t)lv[q].B.n;
        if (al16(need) > budget) return false;
        a.tail = make_tail_args(lv, l0, pinv, nu_pre, nu_post, (T)omega, budget, &smem);
    }
    a.omega = (T)omega;
    a.nu_pre = nu_pre;
    a.nu_post = nu_post;
    a.B = B;
    a.V = V;
    a.Z = Z;
    a.vin = vin;
    a.st = st;
    a.partial = partial;
    a.m = m;
    a.tile = arn_tile_rows(n);
    a.nt = arn_tiles(n);
    a.dj = dj;
    a.ctl = ctl;
    a.bar = bar;
    a.err = err;
    static std::atomic<bool> attr[256] = {};
    BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
    if (!attr[dev]) {
        BAMG_CK(cudaFuncSetAttribute(k_arnoldi_cycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)TAIL_SMEM - fa.sharedSizeBytes)));
        attr[dev] = true;
    }
    int per_sm = 0;
    BAMG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_cycle<T>, PERSIST_THREADS, smem));
    if (per_sm < 1) return false;
    BAMG_CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    BAMG_CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(PERSIST_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BAMG_CK(cudaLaunchKernelEx(&cfg, k_arnoldi_cycle<T>, a));
    count_launch();
    BAMG_CK(cudaGetLastError());
    return true;
}
template bool arnoldi_cycle_persistent<float>(int, const MatView<double>&, double*, float*, float*, int*, double*, int,
                                              double*, const std::vector<VLevel<float>>&, const float*, double, int,
                                              int, const double*, unsigned*, int*, cudaStream_t);
template bool arnoldi_cycle_persistent<double>(int, const MatView<double>&, double*, double*, double*, int*, double*,
                                               int, double*, const std::vector<VLevel<double>>&, const double*,
                                               double, int, int, const double*, unsigned*, int*, cudaStream_t);

// `sweeps` sweeps of the smoother S of Eq. (4.4) on one level, ping-ponging between x and
// y; the result ends in x (one copy when sweeps is odd).
template <typename T>
void smooth_sweeps(const VLevel<T>& v, const T* b, T* x, T* y, double omega_d, int sweeps, cudaStream_t s) {
    const int n = v.B.n;
    const unsigned g = blocks_for(n, 256);
    const T omega = (T)omega_d;
    T* cur = x;
    T* nxt = y;
    for (int k = 0; k < sweeps; ++k) {
        BAMG_LAUNCH(k_smooth<T>, g, 256, 0, s, n, v.B.rp, v.B.ci, v.B.v, v.dinv, b, cur, nxt, omega, (T*)nullptr,
                    (const int*)nullptr);
        T* q = cur;
        cur = nxt;
        nxt = q;
    }
    if (cur != x) BAMG_CK(cudaMemcpyAsync(x, cur, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
}
template void smooth_sweeps<float>(const VLevel<float>&, const float*, float*, float*, double, int, cudaStream_t);
template void smooth_sweeps<double>(const VLevel<double>&, const double*, double*, double*, double, int, cudaStream_t);

template void vcycle<float>(const std::vector<VLevel<float>>&, const float*, double, int, int, cudaStream_t, float*,
                            const int*);
template void vcycle<double>(const std::vector<VLevel<double>>&, const double*, double, int, int, cudaStream_t,
                             double*, const int*);
template void form_x<float>(int, const double*, const float*, int64_t, int, const double*, double*, cudaStream_t,
                             const int*);
template void form_x<double>(int, const double*, const double*, int64_t, int, const double*, double*, cudaStream_t,
                              const int*);

}  // namespace bamg
