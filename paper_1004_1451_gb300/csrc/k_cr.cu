// Compatible-relaxation coarsening, Algorithm 1 (Section 3.1): an independent set of
// the graph of B to start, then rounds of nu F-relaxation sweeps (Eq. (3.2)) from random
// starts in [1, 2); while the convergence estimate of Eq. (3.3) exceeds theta, an
// independent set of the slow points joins C.  Independent sets use Luby's rule with
// fixed SplitMix64 priorities: an undecided candidate enters when its key (priority,
// index) beats every undecided neighbour's, after which its undecided neighbours leave.
#include "kernels.cuh"

namespace bamg {

__global__ void k_tcount(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         int32_t* __restrict__ cnt) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] != i) atomicAdd(cnt + ci[p], 1);
}
__global__ void k_tfill(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const int32_t* __restrict__ rpT, int32_t* __restrict__ cursor, int32_t* __restrict__ ciT) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = ci[p];
        if (j != i) ciT[rpT[j] + atomicAdd(cursor + j, 1)] = i;
    }
}

__device__ __forceinline__ bool beats(uint64_t pi, int i, uint64_t pj, int j) { return pi > pj || (pi == pj && i > j); }

__global__ void k_mis_step(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const int32_t* __restrict__ rpT, const int32_t* __restrict__ ciT,
                           const uint8_t* __restrict__ und, uint8_t* __restrict__ win, uint64_t seed, uint64_t stream,
                           int* __restrict__ left) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *left = 0;  // counted by this round's k_mis_remove
    if (i >= n) return;
    if (!und[i]) {
        win[i] = 0;
        return;
    }
    const uint64_t pi = counter_u64(seed, stream, (uint64_t)i);
    bool ok = true;
    for (int p = rp[i]; p < rp[i + 1] && ok; ++p) {
        const int j = ci[p];
        if (j != i && und[j] && !beats(pi, i, counter_u64(seed, stream, (uint64_t)j), j)) ok = false;
    }
    for (int p = rpT[i]; p < rpT[i + 1] && ok; ++p) {
        const int j = ciT[p];
        if (und[j] && !beats(pi, i, counter_u64(seed, stream, (uint64_t)j), j)) ok = false;
    }
    win[i] = ok ? 1 : 0;
}

__global__ void k_mis_remove(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ rpT, const int32_t* __restrict__ ciT,
                             uint8_t* __restrict__ und, const uint8_t* __restrict__ win, uint8_t* __restrict__ chosen,
                             int* __restrict__ left) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !und[i]) return;
    if (win[i]) {
        chosen[i] = 1;
        und[i] = 0;
        return;
    }
    for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] != i && win[ci[p]]) {
            und[i] = 0;
            return;
        }
    for (int p = rpT[i]; p < rpT[i + 1]; ++p)
        if (win[ciT[p]]) {
            und[i] = 0;
            return;
        }
    atomicAdd(left, 1);
}

// chosen |= independent set of the candidates (und on entry; consumed).  The host reads
// the count of undecided candidates every MIS_CHECK rounds: rounds after the last
// decision change nothing (no candidate is left), so the result is that of a check
// after every round.
constexpr int MIS_CHECK = 4;
static void independent_set(int n, const int32_t* rp, const int32_t* ci, const int32_t* rpT, const int32_t* ciT,
                            uint8_t* und, uint8_t* chosen, uint64_t seed, uint64_t stream, cudaStream_t s) {
    TmpBuf<uint8_t> win(n, s);
    TmpBuf<int> left(1, s);
    const unsigned g = blocks_for(n, 256);
    for (int round = 0; round <= n; round += MIS_CHECK) {
        for (int k = 0; k < MIS_CHECK; ++k) {
            BAMG_LAUNCH(k_mis_step, g, 256, 0, s, n, rp, ci, rpT, ciT, und, win.get(), seed, stream, left.get());
            BAMG_LAUNCH(k_mis_remove, g, 256, 0, s, n, rp, ci, rpT, ciT, und, win.get(), chosen, left.get());
        }
        int h = 0;
        BAMG_CK(cudaMemcpyAsync(&h, left.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
        if (h == 0) return;
    }
    throw Error(BAMG_ETIMEOUT, "independent set did not terminate");
}

__global__ void k_cr_start(int n, const uint8_t* __restrict__ cf, double* __restrict__ u, uint64_t seed,
                           uint64_t stream) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] = cf[i] ? 0.0 : 1.0 + counter_uniform(seed, stream, (uint64_t)i);
}

template <typename T>
__global__ void k_frelax(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const T* __restrict__ bv, const uint8_t* __restrict__ cf, const double* __restrict__ u,
                         double* __restrict__ un, double omega) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i]) {
        un[i] = 0.0;
        return;
    }
    double s = 0.0, d = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const int j = ci[p];
        if (j == i) d = (double)bv[p];
        if (!cf[j]) s += (double)bv[p] * u[j];
    }
    un[i] = u[i] - (omega * (1.0 / d)) * s;
}

// k_frelax with G lanes per row (long rows of coarse levels): strided partial sums added
// by a butterfly; the lane holding the diagonal contributes d, the others 0.
template <typename T, int G>
__global__ void k_frelax_grp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const T* __restrict__ bv, const uint8_t* __restrict__ cf, const double* __restrict__ u,
                             double* __restrict__ un, double omega) {
    pdl_begin();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G), sub = (int)(t % G);
    double s = 0.0, d = 0.0;
    const bool live = i < n && !cf[i];
    if (live)
        for (int p = rp[i] + sub; p < rp[i + 1]; p += G) {
            const int j = ci[p];
            if (j == i) d = (double)bv[p];
            if (!cf[j]) s += (double)bv[p] * u[j];
        }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if (i < n && sub == 0) un[i] = live ? u[i] - (omega * (1.0 / d)) * s : 0.0;
}

__global__ void k_cr_norms(int n, const double* __restrict__ u0, const double* __restrict__ u,
                           double* __restrict__ partial) {
    pdl_begin();
    __shared__ double sh[2][8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < n) {
        a = u0[i] * u0[i];
        b = u[i] * u[i];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * 2 + threadIdx.x] = t;
    }
}
__global__ void k_sum2(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    pdl_begin();
    const int q = threadIdx.x;
    if (q >= 2) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * 2 + q];
    out[q] = s;
}

__global__ void k_cr_slow(int n, const uint8_t* __restrict__ cf, const double* __restrict__ up,
                          const double* __restrict__ u, double theta, uint8_t* __restrict__ cand) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cand[i] = (!cf[i] && fabs(u[i]) / fabs(up[i]) > theta) ? 1 : 0;
}

__global__ void k_u8_to_i32(int n, const uint8_t* __restrict__ a, int32_t* __restrict__ b) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}
__global__ void k_cidx_from_scan(int n, const uint8_t* __restrict__ cf, const int32_t* __restrict__ sc,
                                 int32_t* __restrict__ cidx) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cidx[i] = cf[i] ? sc[i] : -1;
}

template <typename T>
int coarsen_cr(const MatView<T>& B, int level, uint64_t seed, double theta, int nu, double omega, int max_rounds,
               uint8_t* cf, int32_t* cidx, int* nc_out, cudaStream_t s) {
    const int n = B.n;
    const unsigned g = blocks_for(n, 256);
    const int G = lanes_per_row(n, B.nnz);
    // transpose pattern for the undirected neighbourhoods
    TmpBuf<int32_t> cnt(n, s), rpT(n + 1, s), cursor(n, s);
    BAMG_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * n, s));
    BAMG_CK(cudaMemsetAsync(cursor.get(), 0, sizeof(int32_t) * n, s));
    BAMG_LAUNCH(k_tcount, g, 256, 0, s, n, B.rp, B.ci, cnt.get());
    exclusive_scan(cnt.get(), rpT.get(), n, s);
    TmpBuf<int32_t> ciT(B.nnz > 0 ? B.nnz : 1, s);  // bound: the off-diagonal entries of B
    BAMG_LAUNCH(k_tfill, g, 256, 0, s, n, B.rp, B.ci, rpT.get(), cursor.get(), ciT.get());
    TmpBuf<uint8_t> und(n, s), cand(n, s);
    BAMG_CK(cudaMemsetAsync(cf, 0, n, s));
    BAMG_CK(cudaMemsetAsync(und.get(), 1, n, s));
    independent_set(n, B.rp, B.ci, rpT.get(), ciT.get(), und.get(), cf, seed, STREAM_MIS + ((uint64_t)level << 8), s);
    TmpBuf<double> u0(n, s), ua(n, s), ub(n, s), norms(2, s), part((size_t)g * 2, s);
    int rounds = 0;
    double h[2];
    for (;;) {
        BAMG_LAUNCH(k_cr_start, g, 256, 0, s, n, cf, u0.get(), seed, STREAM_CR + ((uint64_t)level << 8) + rounds);
        const double* cur = u0.get();
        double* prev = nullptr;
        double* bufs[2] = {ua.get(), ub.get()};
        for (int k = 0; k < nu; ++k) {
            double* nxt = bufs[k & 1];
            const unsigned gg = blocks_for((int64_t)n * G, 256);
            switch (G) {
                case 1: BAMG_LAUNCH(k_frelax<T>, g, 256, 0, s, n, B.rp, B.ci, B.v, cf, cur, nxt, omega); break;
                case 4: BAMG_LAUNCH((k_frelax_grp<T, 4>), gg, 256, 0, s, n, B.rp, B.ci, B.v, cf, cur, nxt, omega); break;
                case 8: BAMG_LAUNCH((k_frelax_grp<T, 8>), gg, 256, 0, s, n, B.rp, B.ci, B.v, cf, cur, nxt, omega); break;
                case 16:
                    BAMG_LAUNCH((k_frelax_grp<T, 16>), gg, 256, 0, s, n, B.rp, B.ci, B.v, cf, cur, nxt, omega);
                    break;
                default:
                    BAMG_LAUNCH((k_frelax_grp<T, 32>), gg, 256, 0, s, n, B.rp, B.ci, B.v, cf, cur, nxt, omega);
            }
            prev = const_cast<double*>(cur);
            cur = nxt;
        }
        BAMG_LAUNCH(k_cr_norms, g, 256, 0, s, n, u0.get(), cur, part.get());
        BAMG_LAUNCH(k_sum2, 1, 32, 0, s, (int)g, part.get(), norms.get());
        BAMG_CK(cudaMemcpyAsync(h, norms.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
        const double rho = std::pow(std::sqrt(h[1]) / std::sqrt(h[0]), 1.0 / nu);
        if (!(rho > theta) || rounds >= max_rounds || h[0] == 0.0) break;
        BAMG_LAUNCH(k_cr_slow, g, 256, 0, s, n, cf, prev, cur, theta, cand.get());
        ++rounds;
        independent_set(n, B.rp, B.ci, rpT.get(), ciT.get(), cand.get(), cf, seed,
                        STREAM_MIS + ((uint64_t)level << 8) + rounds, s);
    }
    TmpBuf<int32_t> ci32(n, s), sc(n + 1, s);
    BAMG_LAUNCH(k_u8_to_i32, g, 256, 0, s, n, cf, ci32.get());
    exclusive_scan(ci32.get(), sc.get(), n, s);
    BAMG_LAUNCH(k_cidx_from_scan, g, 256, 0, s, n, cf, sc.get(), cidx);
    *nc_out = read_int(sc.get() + n, s);
    return rounds;
}

// ---------------------------------------------------------------- colouring of the smoother
// Colour c = an independent set (the rule above, priority stream STREAM_COLOUR + (level <<
// 8) + c) of the states the earlier colours left, in the symmetrised graph of B, until
// every state has a colour.  The classes go out as one row list sorted by (colour, state)
// with host offsets ptr[0..ncol].
__global__ void k_colour_take(int n, const uint8_t* __restrict__ chosen, int c, int32_t* __restrict__ colour,
                              uint8_t* __restrict__ left, int* __restrict__ remaining) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (chosen[i]) {
        colour[i] = c;
        left[i] = 0;
    } else if (left[i]) {
        atomicAdd(remaining, 1);
    }
}

constexpr int MAX_COLOURS = 255;  // the stream encoding leaves 8 bits for the colour

void colour_classes(int n, int nnz, const int32_t* rp, const int32_t* ci, int level, uint64_t seed,
                    std::vector<int>& ptr, DevBuf<int32_t>& rows, cudaStream_t s) {
    const unsigned g = blocks_for(n, 256);
    TmpBuf<int32_t> cnt(n, s), rpT(n + 1, s), cursor(n, s);
    BAMG_CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * n, s));
    BAMG_CK(cudaMemsetAsync(cursor.get(), 0, sizeof(int32_t) * n, s));
    BAMG_LAUNCH(k_tcount, g, 256, 0, s, n, rp, ci, cnt.get());
    exclusive_scan(cnt.get(), rpT.get(), n, s);
    TmpBuf<int32_t> ciT(nnz > 0 ? nnz : 1, s);
    BAMG_LAUNCH(k_tfill, g, 256, 0, s, n, rp, ci, rpT.get(), cursor.get(), ciT.get());
    TmpBuf<uint8_t> left(n, s), und(n, s), chosen(n, s);
    TmpBuf<int32_t> colour(n, s);
    TmpBuf<int> rem(1, s);
    BAMG_CK(cudaMemsetAsync(left.get(), 1, n, s));
    int ncol = 0;
    for (int c = 0; c < MAX_COLOURS; ++c) {
        BAMG_CK(cudaMemcpyAsync(und.get(), left.get(), n, cudaMemcpyDeviceToDevice, s));
        BAMG_CK(cudaMemsetAsync(chosen.get(), 0, n, s));
        independent_set(n, rp, ci, rpT.get(), ciT.get(), und.get(), chosen.get(), seed,
                        STREAM_COLOUR + ((uint64_t)level << 8) + (uint64_t)c, s);
        BAMG_CK(cudaMemsetAsync(rem.get(), 0, sizeof(int), s));
        BAMG_LAUNCH(k_colour_take, g, 256, 0, s, n, (const uint8_t*)chosen.get(), c, colour.get(), left.get(),
                    rem.get());
        if (read_int(rem.get(), s) == 0) {
            ncol = c + 1;
            break;
        }
    }
    BAMG_REQUIRE(ncol > 0, BAMG_ETIMEOUT, "colouring: more than 255 colours");
    std::vector<int32_t> hc(n), hr(n);
    BAMG_CK(cudaMemcpyAsync(hc.data(), colour.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    ptr.assign(ncol + 1, 0);
    for (int i = 0; i < n; ++i) ptr[hc[i] + 1]++;
    for (int c = 0; c < ncol; ++c) ptr[c + 1] += ptr[c];
    std::vector<int> at(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n; ++i) hr[at[hc[i]]++] = i;  // ascending states within a colour
    rows.alloc(n);
    BAMG_CK(cudaMemcpyAsync(rows.get(), hr.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    BAMG_CK(cudaStreamSynchronize(s));
}

template int coarsen_cr<float>(const MatView<float>&, int, uint64_t, double, int, double, int, uint8_t*, int32_t*,
                               int*, cudaStream_t);
template int coarsen_cr<double>(const MatView<double>&, int, uint64_t, double, int, double, int, uint8_t*, int32_t*,
                                int*, cudaStream_t);

}  // namespace bamg
