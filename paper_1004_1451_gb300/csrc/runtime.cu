// Host runtime of the library: the hierarchy, the bootstrap setup (Section 1 steps 1-4,
// Algorithm 3 with mu = 1, then the rebuild from the enriched test sets), flexible GMRES
// preconditioned by the V-cycle (Section 4.2), import/export, and the C ABI of bamg.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <type_traits>

#include "gmres_state.cuh"
#include "kernels.cuh"

namespace bamg {

static std::atomic<uint64_t> g_launches{0};
static thread_local uint64_t t_launches = 0;  // this thread's share, for graph-capture bookkeeping
void count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
void count_launches(int64_t k) {
    g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed);
    t_launches += (uint64_t)k;
}
static thread_local std::string g_err;
bool& pdl_enabled() {
    static const bool env_on = [] {
        const char* e = std::getenv("BAMG_PDL");
        return !(e && std::strcmp(e, "0") == 0);
    }();
    static thread_local bool on = env_on;
    return on;
}
void set_last_error(const std::string& m) { g_err = m; }
cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t st = nullptr;
    return st;
}
StackArena*& tmp_arena() {
    static thread_local StackArena* a = nullptr;
    return a;
}
// Sets the allocation stream for the lifetime of the object.
static inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// V-cycle factor helpers: x0 = 1 + u (SplitMix64 seed 7, stream 0), sums of r and r^2,
// r <- (r - mean) * scale, r <- r - t.
__global__ void k_vf_start(int n, double* __restrict__ x) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0 + counter_uniform(7, 0, (uint64_t)i);
}
__global__ void k_vf_moments(int n, const double* __restrict__ r, double* __restrict__ mom) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < n) {
        a = r[i];
        b = a * a;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(mom, a);
        atomicAdd(mom + 1, b);
    }
}
__global__ void k_vf_affine(int n, double* __restrict__ r, double mean, double scale) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = (r[i] - mean) * scale;
}
__global__ void k_vf_axpy(int n, double* __restrict__ r, const double* __restrict__ t) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] -= t[i];
}

// X[i * ld + col] = x_i / sqrt(nrm2[0]) (the MLE restart's state-vector column)
template <typename T>
__global__ void k_state_col(int n, const double* __restrict__ x, const double* __restrict__ nrm2, T* __restrict__ X,
                            int ld, int col) {
    pdl_begin();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
    if (i < n) X[(int64_t)i * ld + col] = (T)(x[i] * s);
}

// active[k] = 1 for the random vectors, sel[q] for eigenvector column ldU + q, else 0.
__global__ void k_active_mask(int r, int ldU, int nvec, int ld, const uint8_t* __restrict__ sel,
                              uint8_t* __restrict__ active) {
    pdl_begin();
    const int k = threadIdx.x;
    if (k >= ld) return;
    uint8_t a = 0;
    if (k < r) a = 1;
    else if (k >= ldU && k - ldU < nvec) a = sel[k - ldU];
    active[k] = a;
}

template <typename T>
struct LevelT {
    int n = 0, nnz = 0;
    DevBuf<int32_t> rp, ci;
    DevBuf<T> bv, tv;  // B_l and T_l (T on B's pattern)
    DevBuf<T> dB, dT, dinv;
    int nx = 0, ny = 0;
    DevBuf<uint8_t> cf;
    DevBuf<int32_t> cidx, c2f;
    int nc = 0;
    DevBuf<int32_t> pcol, pcnt;
    DevBuf<T> pval;
    DevBuf<int32_t> qrp, qci;
    DevBuf<T> qv;
    DevBuf<T> X;
    DevBuf<double> w, lam;
    DevBuf<uint8_t> sel;
    DevBuf<T> vb, vx, vr;
    DevBuf<int32_t> gs_rows;  // multicolour Gauss-Seidel classes (rows by colour)
    std::vector<int> gs_ptr;
    MatView<T> B() const { return MatView<T>{n, nnz, rp.get(), ci.get(), bv.get()}; }
    EllView<T> P(int c) const { return EllView<T>{n, c, pcol.get(), pval.get(), pcnt.get()}; }
    void diagonals(cudaStream_t s) {
        dB.alloc(n);
        dT.alloc(n);
        dinv.alloc(n);
        launch_diagonals<T>(n, rp.get(), ci.get(), bv.get(), tv.get(), dB.get(), dT.get(), dinv.get(), s);
    }
};

// BAMG_TRACE set (and not "0"): the setup synchronises at each phase boundary and prints
// the wall time of every phase to stderr.  Diagnostic only; off by default.
struct PhaseTrace {
    bool on = false;
    cudaStream_t s = nullptr;
    std::chrono::steady_clock::time_point t;
    std::string out;
    explicit PhaseTrace(cudaStream_t s_) : s(s_) {
        const char* e = std::getenv("BAMG_TRACE");
        on = e && std::strcmp(e, "0") != 0;
        if (on) {
            cudaStreamSynchronize(s);
            t = std::chrono::steady_clock::now();
        }
    }
    void mark(const char* what, int l = -1) {
        if (!on) return;
        const auto issued = std::chrono::steady_clock::now();
        cudaStreamSynchronize(s);
        const auto now = std::chrono::steady_clock::now();
        const double ms = std::chrono::duration<double, std::milli>(now - t).count();
        const double ims = std::chrono::duration<double, std::milli>(issued - t).count();
        char buf[96];  // phase: host time to issue its work / wall time to its completion
        if (l >= 0)
            std::snprintf(buf, sizeof buf, " %s@%d %.3f/%.3f", what, l, ims, ms);
        else
            std::snprintf(buf, sizeof buf, " %s %.3f/%.3f", what, ims, ms);
        out += buf;
        t = now;
    }
    ~PhaseTrace() {
        if (on) std::fprintf(stderr, "bamg setup phases (ms):%s\n", out.c_str());
    }
};

// The solve's private stream and its two fence events.  Held by the base class so that it
// is destroyed after every device buffer of the derived solver: buffers (re)allocated
// during a solve (the MLE restart's rebuilt levels) are released on this stream.
struct PrivateStream {
    cudaStream_t ps = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ~PrivateStream() {
        if (ps) cudaStreamSynchronize(ps);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (ps) cudaStreamDestroy(ps);
    }
};

struct SolverBase {
    PrivateStream priv;  // first member: destroyed last
    bamg_opts o{};
    cudaStream_t s = nullptr;
    double setup_ms = 0.0;
    virtual ~SolverBase() {}
    virtual int nlevels() const = 0;
    virtual void level_size(int l, int64_t* n, int64_t* nnz) const = 0;
    virtual void solve(double* x, int flags, double tol, bamg_stats* st) = 0;
    virtual void parnoldi(double* x, int flags, double tol, bamg_stats* st) = 0;
    virtual void mle_setup(const bamg_csr* A, int r, int levels, double tol, int max_cycles, bool l2, double* x,
                           bool x_host, bamg_stats* st) = 0;
    virtual void vcycle_apply(const double* v, double* z) = 0;
    virtual void smooth_apply(int level, int sweeps, const void* b, void* x, void* work) = 0;
    virtual int precision() const = 0;
    virtual double vcycle_factor(int iters) = 0;
    virtual void export_obj(int level, int what, void* h_dst, int64_t cap, int64_t* bytes) = 0;
    // training-data recording (bamg_interp_dataset): features and LS rows of every fit
    bool record = false;
    float* rec_feat = nullptr;
    float* rec_target = nullptr;
    int64_t rec_cap = 0, rec_rows = 0;
    int interp_used = BAMG_INTERP_LS;
    double rho_measured = 0.0;
    virtual void layout(int level, int* ld, int* r, int* v0, int* nvec) const = 0;
};

template <typename T>
struct Solver : SolverBase {
    std::vector<std::unique_ptr<LevelT<T>>> lv;
    int r = 0, ldU = 0, ldV = 0, ld = 0, nvec = 0, nL = 0;
    DevBuf<double> b64_own;  // FP64 values of B_0 when T = float
    const double* b64 = nullptr;
    DevBuf<double> pinv64;
    DevBuf<T> pinvT;
    DevBuf<double> x_init;
    // Krylov workspace
    int m = 0;
    DevBuf<double> V, state, partial, x0, xw, rn;
    DevBuf<T> Z, vin, zout;
    DevBuf<int> dj;
    double* h_pin = nullptr;
    // one Arnoldi step captured as a CUDA graph, replayed on the private stream
    cudaStream_t& ps = priv.ps;
    cudaEvent_t& ev_in = priv.ev_in;
    cudaEvent_t& ev_out = priv.ev_out;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_kernels = 0;  // kernels of one step
    int64_t graph_post = 0;     // kernels of the check after the device-side loop (one per launch)
    bool graph_loop = false;    // one launch runs steps until the device-side test stops it
    DevBuf<double> ctl;         // the loop's kappa, tol ||x||_1 and last j + 1
    DevBuf<unsigned> pbar;      // grid barrier of the persistent Arnoldi cycle
    DevBuf<int> perr;           // set when one of its barrier waits gave up

    ~Solver() override {
        cudaStreamSynchronize(s);
        if (ps) cudaStreamSynchronize(ps);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (h_pin) cudaFreeHost(h_pin);
        // the private stream itself is destroyed by SolverBase::priv after the buffers
    }
    int nlevels() const override { return (int)lv.size(); }
    void level_size(int l, int64_t* n, int64_t* nnz) const override {
        *n = lv[l]->n;
        *nnz = lv[l]->nnz;
    }
    void layout(int l, int* ld_, int* r_, int* v0, int* nv) const override {
        (void)l;
        if (ld_) *ld_ = ld;
        if (r_) *r_ = r;
        if (v0) *v0 = ldU;
        if (nv) *nv = nvec;
    }
    MatView<double> B64() const { return MatView<double>{lv[0]->n, lv[0]->nnz, lv[0]->rp.get(), lv[0]->ci.get(), b64}; }
    double ridge() const { return std::is_same<T, float>::value ? o.ridge32 : o.ridge; }

    std::vector<VLevel<T>> vlevels(const T* b0, T* x0v) {
        std::vector<VLevel<T>> v(lv.size());
        for (size_t l = 0; l < lv.size(); ++l) {
            LevelT<T>& L = *lv[l];
            v[l].B = L.B();
            v[l].dinv = L.dinv.get();
            if (l + 1 < lv.size()) {
                v[l].P = L.P(o.caliber);
                v[l].qrp = L.qrp.get();
                v[l].qci = L.qci.get();
                v[l].qv = L.qv.get();
                v[l].qnnz = (int)L.qci.n;
            }
            v[l].b = L.vb.get();
            v[l].x = L.vx.get();
            v[l].r = L.vr.get();
            if (o.smoother == BAMG_SMOOTH_MCGS && l + 1 < lv.size() && !L.gs_ptr.empty()) {
                v[l].gs_rows = L.gs_rows.get();
                v[l].gs_ptr = L.gs_ptr.data();
                v[l].gs_ncol = (int)L.gs_ptr.size() - 1;
            }
        }
        v[0].b = const_cast<T*>(b0);
        v[0].x = x0v;
        v[0].tail_form = o.coarse_tail;
        return v;
    }

    DevBuf<int> ls_err;  // bit 1: a neighbourhood search overflowed; bit 2: B_L^+ failed (read once per setup)
    std::unique_ptr<StackArena> arena;  // the setup's temporaries
    PhaseTrace* trace = nullptr;  // set during a traced setup

    void alloc_vcycle_work() {
        for (auto& L : lv) {
            L->vb.alloc(L->n);
            L->vx.alloc(L->n);
            L->vr.alloc(L->n);
        }
    }

    // --------------------------------------------------------------- interpolation step
    // P_l by Algorithm 2 from the active columns of X_l, Q_l, and the Galerkin products
    // into level l+1 (replacing its operators).
    void build_level_operators(int l, const uint8_t* d_active, int ncols_w) {
        LevelT<T>& c = *lv[l];
        LevelT<T>& nx = *lv[l + 1];
        c.w.alloc(ld);
        BAMG_CK(cudaMemsetAsync(c.w.get(), 0, sizeof(double) * ld, s));
        tv_weights<T>(c.B(), ncols_w, ld, 0, d_active, o.weight_floor, c.X.get(), c.w.get(), s);
        if (trace) trace->mark(" w", l);
        c.pcol.alloc((size_t)c.n * o.caliber);
        c.pval.alloc((size_t)c.n * o.caliber);
        c.pcnt.alloc(c.n);
        if (o.interp == BAMG_INTERP_LEARNED) {
            interp_learned<T>(c.n, c.rp.get(), c.ci.get(), c.bv.get(), c.cf.get(), c.cidx.get(), c.X.get(), ld, ld,
                              c.w.get(), o.z, o.mmax, o.caliber, ridge(), o.model->impl, o.learned_refit != 0,
                              c.pcol.get(), c.pval.get(), c.pcnt.get(), s, ls_err.get());
        } else {
            LsOut ex;
            if (record) {
                if (rec_feat && rec_target && rec_rows + c.n <= rec_cap) {
                    ex.feat = rec_feat + rec_rows * MLP_F;
                    ex.target = rec_target + rec_rows * MLP_S;
                }
                rec_rows += c.n;
            }
            interp_ls<T>(c.n, c.rp.get(), c.ci.get(), c.bv.get(), c.cf.get(), c.cidx.get(), c.X.get(), ld, ld,
                         c.w.get(), o.z, o.mmax, o.caliber, ridge(), c.pcol.get(), c.pval.get(), c.pcnt.get(), s,
                         ls_err.get(), ex);
        }
        if (trace) trace->mark(" interp", l);
        build_restriction<T>(c.P(o.caliber), c.nc, c.qrp, c.qci, c.qv, s);
        if (trace) trace->mark(" q", l);
        GalerkinOut<T> go;
        // the entry count reaches the host while the compaction and the diagonals run (the
        // coarse arrays have room for the product count's bound)
        galerkin<T>(c.B(), c.tv.get(), c.qrp.get(), c.qci.get(), c.qv.get(), c.P(o.caliber), c.nc, go, s, true);
        nx.n = c.nc;
        nx.rp = std::move(go.rp);
        nx.ci = std::move(go.ci);
        nx.bv = std::move(go.bv);
        nx.tv = std::move(go.tv);
        nx.diagonals(s);
        galerkin_nnz<T>(go, s);
        nx.nnz = go.nnz;
        if (trace) trace->mark(" gal", l);
    }

    void split(int l) {
        LevelT<T>& c = *lv[l];
        c.cf.alloc(c.n);
        c.cidx.alloc(c.n);
        if (o.coarsen == BAMG_COARSEN_GRID) {
            coarsen_grid(c.nx, c.ny, c.cf.get(), c.cidx.get(), s);
            c.nc = ((c.nx + 1) / 2) * ((c.ny + 1) / 2);
        } else {
            int nc = 0;
            coarsen_cr<T>(c.B(), l, o.seed, o.cr_theta, o.cr_nu, o.cr_omega, o.cr_max_rounds, c.cf.get(), c.cidx.get(),
                          &nc, s);
            c.nc = nc;
        }
        BAMG_REQUIRE(c.nc > 0 && c.nc < c.n, BAMG_ENUMERIC, "coarsening produced no coarse level");
        c.c2f.alloc(c.nc);
        coarse_to_fine(c.n, c.cf.get(), c.cidx.get(), c.c2f.get(), s);
    }

    // --------------------------------------------------------------- setup
    // Algorithm 3 as a recursion over the levels (the same steps in the same order as the
    // CPU restatement): first visit (relax U_l, split), interpolation step (P_l, Q_l,
    // B_{l+1}, T_{l+1}; U_{l+1} = R U_l on the first descent), recursive call, upward step
    // (V_l = P_l V_{l+1}, shifted sweeps, lambda update, selection).
    int levels_max = 0;
    int L_idx = -1;  // index of the coarsest level once the first descent reached it

    bool first_visit(int l) {
        LevelT<T>& c = *lv[l];
        if (l == levels_max || c.n <= o.coarse_max) {
            L_idx = l;
            return true;
        }
        {
            TmpBuf<T> work((size_t)c.n * ld, s);
            relax<T>(c.B(), nullptr, c.dB.get(), c.dinv.get(), nullptr, nullptr, r, ld, 0, (T)o.omega, o.nu_tv,
                     c.X.get(), work.get(), s);
        }
        if (trace) trace->mark("relax", l);
        split(l);
        if (trace) trace->mark("split", l);
        return false;
    }

    void interp_step(int l, bool with_v) {
        const bool create = (int)lv.size() == l + 1;
        if (create) {
            auto nl = std::make_unique<LevelT<T>>();
            nl->nx = (lv[l]->nx + 1) / 2;
            nl->ny = (lv[l]->ny + 1) / 2;
            lv.push_back(std::move(nl));
        }
        if (with_v) {
            TmpBuf<uint8_t> active(32, s);
            BAMG_LAUNCH(k_active_mask, 1, 32, 0, s, r, ldU, nvec, ld, lv[l]->sel.get(), active.get());
            build_level_operators(l, active.get(), ld);
        } else {
            build_level_operators(l, nullptr, r);
        }
        if (create) {
            LevelT<T>& cc = *lv[l];
            LevelT<T>& nn = *lv[l + 1];
            nn.X.alloc((size_t)nn.n * ld);
            BAMG_CK(cudaMemsetAsync(nn.X.get(), 0, sizeof(T) * nn.n * ld, s));
            inject_cols<T>(nn.n, cc.c2f.get(), cc.X.get(), nn.X.get(), ld, 0, r, s);
        }
        if (trace) trace->mark(with_v ? "rebuild" : "operators", l);
    }

    void coarsest_eigs(int l) {
        LevelT<T>& Lc = *lv[l];
        nL = Lc.n;
        BAMG_REQUIRE(nL <= 64, BAMG_EINVAL, "coarsest level has more than 64 states: raise `levels` or lower coarse_max");
        TmpBuf<double> Bd((size_t)nL * nL, s), Td((size_t)nL * nL, s), Vd((size_t)nL * (o.k_ev + 1), s);
        TmpBuf<int32_t> kinds(o.k_ev + 1, s);
        csr_to_dense<T>(nL, Lc.rp.get(), Lc.ci.get(), Lc.bv.get(), Bd.get(), s);
        csr_to_dense<T>(nL, Lc.rp.get(), Lc.ci.get(), Lc.tv.get(), Td.get(), s);
        Lc.lam.ensure(ldV);
        BAMG_CK(cudaMemsetAsync(Lc.lam.get(), 0, sizeof(double) * ldV, s));
        const int nv = coarse_eig(nL, Bd.get(), Td.get(), o.k_ev, Lc.lam.get(), Vd.get(), kinds.get(),
                                  std::is_same<T, float>::value, s);
        BAMG_REQUIRE(nv > 0, BAMG_ENUMERIC, "coarsest eigensolve did not converge");
        nvec = nv;
        launch_vecs_to_strided<double, T>(nL, nvec, Vd.get(), Lc.X.get(), ld, ldU, s);
        ++coarse_solves;
        if (trace) trace->mark("coarse_eig");
    }

    void up_step(int l) {
        LevelT<T>& c = *lv[l];
        LevelT<T>& ch = *lv[l + 1];
        prolong_cols<T>(c.P(o.caliber), ch.X.get(), c.X.get(), ld, ldU, nvec, s);
        c.lam.ensure(ldV);
        BAMG_CK(cudaMemcpyAsync(c.lam.get(), ch.lam.get(), sizeof(double) * ldV, cudaMemcpyDeviceToDevice, s));
        relax_v(l);
        c.sel.ensure(ldV);
        rayleigh_update<T>(c.B(), c.tv.get(), c.X.get(), nvec, ld, ldU, o.ev_change_tol, c.lam.get(), c.sel.get(), s);
        if (trace) trace->mark("up", l);
    }

    // nu_ev sweeps on (B_l - lambda_i T_l) x^(i) = 0 over the eigenvector columns
    void relax_v(int l) {
        LevelT<T>& c = *lv[l];
        TmpBuf<T> work((size_t)c.n * ld, s);
        relax<T>(c.B(), c.tv.get(), c.dB.get(), c.dinv.get(), c.dT.get(), c.lam.get(), nvec, ld, ldU, (T)o.omega,
                 o.nu_ev, c.X.get(), work.get(), s);
    }

    // bootamg_mle (Algorithm 3) with loop count o.mu.  V_l = {} only on the first visit of
    // level l; later visits relax V_l on the way down and fit P_l to U_l and V_l (the
    // reading of the CPU restatement); U_l is relaxed on the first visit only.
    void mle(int l, bool first) {
        if (first) {
            if (first_visit(l)) {
                coarsest_eigs(l);
                return;
            }
        } else if (l == L_idx) {
            coarsest_eigs(l);
            return;
        } else {
            relax_v(l);
        }
        for (int it = 0; it < o.mu; ++it) {
            const bool fresh = first && it == 0;
            interp_step(l, !fresh);
            mle(l + 1, fresh);
            up_step(l);
        }
    }

    // Section 1: all P_l, B_l, T_l recalculated top-down from U_l and the selected V_l
    void rebuild() {
        for (int l = 0; l < L_idx; ++l) interp_step(l, true);
    }

    // minimal-norm inverse of the coarsest B_L (Section 4.2)
    void coarse_pinv_now() {
        LevelT<T>& Lc = *lv[L_idx];
        TmpBuf<double> Bd((size_t)nL * nL, s);
        csr_to_dense<T>(nL, Lc.rp.get(), Lc.ci.get(), Lc.bv.get(), Bd.get(), s);
        pinv64.ensure((size_t)nL * nL);
        coarse_pinv(nL, Bd.get(), pinv64.get(), std::is_same<T, float>::value, s, ls_err.get());
        pinvT.ensure((size_t)nL * nL);
        if constexpr (std::is_same<T, double>::value)
            BAMG_CK(cudaMemcpyAsync(pinvT.get(), pinv64.get(), sizeof(double) * nL * nL, cudaMemcpyDeviceToDevice, s));
        else
            launch_convert<double, float>((int64_t)nL * nL, pinv64.get(), pinvT.get(), s);
        if (trace) trace->mark("pinv");
    }

    // colour classes of every level but the coarsest for the multicolour Gauss-Seidel
    // smoother, on the final B_l
    void build_colours() {
        if (o.smoother != BAMG_SMOOTH_MCGS) return;
        for (size_t l = 0; l + 1 < lv.size(); ++l) {
            LevelT<T>& c = *lv[l];
            colour_classes(c.n, c.nnz, c.rp.get(), c.ci.get(), (int)l, o.seed, c.gs_ptr, c.gs_rows, s);
        }
        if (trace) trace->mark("colours");
    }

    // the state-vector approximation V_0[:, 0] in FP64 into y, scaled to 1^T y = 1; the
    // l1 ratio ||B y||_1 / ||y||_1 and the 2-norm ratio into h_ratio[0..1] when given
    void state_vector(double* y, double* h_ratio) {
        const int n = lv[0]->n;
        launch_strided_to_vec<T, double>(n, lv[0]->X.get(), ld, ldU, y, s);
        TmpBuf<double> sums(8, s), part((size_t)blocks_for(n, 256) * RESNORM_SUMS, s);
        residual_norms(B64(), y, sums.get(), part.get(), s);
        scale_vec(n, y, sums.get(), 3, true, y, s);
        if (h_ratio) {  // the ratios are scale invariant: read them off the same sums
            double h[RESNORM_SUMS];
            BAMG_CK(cudaMemcpyAsync(h, sums.get(), sizeof h, cudaMemcpyDeviceToHost, s));
            BAMG_CK(cudaStreamSynchronize(s));
            h_ratio[0] = h[2] > 0.0 ? h[0] / h[2] : INFINITY;
            h_ratio[1] = h[4] > 0.0 ? std::sqrt(h[1] / h[4]) : INFINITY;
        }
    }

    int coarse_solves = 0;

    void read_input(const bamg_csr* A, int r_) {
        const int n = A->n;
        r = r_;
        const int32_t *rpA = A->row_ptr, *ciA = A->col;
        const double* vA = A->val;
        DevBuf<int32_t> hrp, hci;
        DevBuf<double> hv;
        if (A->on_host) {
            hrp.alloc(n + 1);
            hci.alloc(std::max(A->nnz, 1));
            hv.alloc(std::max(A->nnz, 1));
            BAMG_CK(cudaMemcpyAsync(hrp.get(), A->row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
            BAMG_CK(cudaMemcpyAsync(hci.get(), A->col, sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice, s));
            BAMG_CK(cudaMemcpyAsync(hv.get(), A->val, sizeof(double) * A->nnz, cudaMemcpyHostToDevice, s));
            rpA = hrp.get();
            ciA = hci.get();
            vA = hv.get();
        }
        DevBuf<int32_t> rpB, ciB;
        DevBuf<double> vB;
        const int flags = build_system_matrix(n, A->nnz, rpA, ciA, vA, rpB, ciB, vB, s);
        BAMG_REQUIRE(!(flags & 8), BAMG_EINVAL, "A: column indices must be sorted, unique and within [0, n)");
        BAMG_REQUIRE(!(flags & 1), BAMG_ENOTSTOCH, "A has a negative entry");
        BAMG_REQUIRE(!(flags & 4), BAMG_ENOTSTOCH, "A has a_ii = 1 (absorbing state)");
        BAMG_REQUIRE(!(flags & 2), BAMG_ENOTSTOCH, "A is not column stochastic (|colsum - 1| > 1e-12)");
        auto L0 = std::make_unique<LevelT<T>>();
        L0->n = n;
        L0->nnz = read_int(rpB.get() + n, s);
        L0->rp = std::move(rpB);
        L0->ci = std::move(ciB);
        if constexpr (std::is_same<T, double>::value) {
            L0->bv = std::move(vB);
            b64 = L0->bv.get();
        } else {
            L0->bv.alloc(L0->nnz);
            launch_convert<double, float>(L0->nnz, vB.get(), L0->bv.get(), s);
            b64_own = std::move(vB);
            b64 = b64_own.get();
        }
        L0->tv.alloc(L0->nnz);
        launch_identity_on_pattern<T>(n, L0->rp.get(), L0->ci.get(), L0->tv.get(), s);
        L0->diagonals(s);
        L0->nx = o.grid_nx;
        L0->ny = o.grid_ny;
        constexpr int W = V16<T>::W;
        ldU = round_up(r, W);
        ldV = round_up(o.k_ev + 1, W);
        ld = ldU + ldV;
        BAMG_REQUIRE(ld <= 32, BAMG_EINVAL, "r + k_ev too large: padded test-vector block must be <= 32 columns");
        ls_err.alloc(1);
        BAMG_CK(cudaMemsetAsync(ls_err.get(), 0, sizeof(int), s));
        L0->X.alloc((size_t)n * ld);
        BAMG_CK(cudaMemsetAsync(L0->X.get(), 0, sizeof(T) * n * ld, s));
        launch_tv_init<T>(n, r, ld, 0, o.seed, o.tv_lo, o.tv_hi, L0->X.get(), s);
        lv.clear();
        lv.push_back(std::move(L0));
        nvec = 0;
        coarse_solves = 0;
        L_idx = -1;
    }

    // The setup's device-side error flags (ls_err) reach the host without the setup waiting for
    // the device: the copy is queued into the pinned block (double slot 30) and read by the
    // next call that uses the hierarchy, which waits for the device in any case (bamg_solve
    // after its first residual read, at no cost).
    bool setup_flags_pending = false;
    void queue_setup_flags() {
        ensure_private_stream();
        int* hf = reinterpret_cast<int*>(h_pin + 30);
        *hf = 0;
        BAMG_CK(cudaMemcpyAsync(hf, ls_err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        setup_flags_pending = true;
    }
    // synced: the queued copy is known to have completed (a later wait covered it)
    void check_setup_flags(bool synced) {
        if (!setup_flags_pending) return;
        if (!synced) BAMG_CK(cudaStreamSynchronize(s));
        setup_flags_pending = false;
        const int h_err = *reinterpret_cast<const int*>(h_pin + 30);
        BAMG_REQUIRE(!(h_err & 2), BAMG_ENUMERIC, "singular coarsest factor");
        BAMG_REQUIRE(!(h_err & 1), BAMG_EOVERFLOW, "neighbourhood search: a fine point needs more than 2048 recorded states");
    }
    void check_search_overflow() {
        const int h_err = read_int(ls_err.get(), s);
        BAMG_REQUIRE(!(h_err & 2), BAMG_ENUMERIC, "singular coarsest factor");
        BAMG_REQUIRE(!(h_err & 1), BAMG_EOVERFLOW, "neighbourhood search: a fine point needs more than 2048 recorded states");
    }

    // Bootstrap setup: o.setup_cycles MLE cycles, then the rebuild, B_L^+ and the initial
    // guess.  With `mle_tol` > 0 (the stand-alone MLE of Section 4.1) the cycles go on
    // until the state vector approximation meets the tolerance (2-norm ratio when
    // mle_l2, else the l1 ratio) or `max_cycles` cycles ran; *h_cycles / h_ratio report.
    void setup(const bamg_csr* A, int r_, int levels, double mle_tol = 0.0, int max_cycles = 0, bool mle_l2 = false,
               int* h_cycles = nullptr, double* h_ratio = nullptr) {
        auto t0 = std::chrono::steady_clock::now();
        AllocStream as_(s);
        if (!arena || arena->s != s) arena = std::make_unique<StackArena>(s);
        ArenaScope ar_(*arena);
        PhaseTrace tr(s);
        trace = tr.on ? &tr : nullptr;
        struct Untrace {
            PhaseTrace*& p;
            ~Untrace() { p = nullptr; }
        } untrace_{trace};
        levels_max = levels;
        read_input(A, r_);
        const int n = A->n;
        tr.mark("input");
        x_init.alloc(n);
        if (mle_tol > 0.0) {
            int cycles = 0;
            double rat[2] = {INFINITY, INFINITY};
            while (true) {
                mle(0, cycles == 0);
                ++cycles;
                state_vector(x_init.get(), rat);
                if (rat[mle_l2 ? 1 : 0] <= mle_tol || cycles >= max_cycles) break;
            }
            if (h_cycles) *h_cycles = cycles;
            if (h_ratio) h_ratio[0] = rat[0], h_ratio[1] = rat[1];
        } else {
            mle(0, true);
            for (int c = 1; c < o.setup_cycles; ++c) mle(0, false);
        }
        BAMG_REQUIRE(L_idx >= 0, BAMG_ECUDA, "setup did not reach a coarsest level");
        rebuild();
        coarse_pinv_now();
        build_colours();
        if (mle_tol <= 0.0) state_vector(x_init.get(), nullptr);
        alloc_vcycle_work();
        setup_flags_pending = false;
        if (mle_tol > 0.0)
            check_search_overflow();
        else
            queue_setup_flags();
        tr.mark("guess");
        setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }

    // MLE restart (the reading of Section 5.1's "restarting the MLE iterations"): the
    // iterate x becomes the state-vector test vector of every level (x / ||x||_2 on level 0,
    // injected on the coarser ones), all P_l, B_l, T_l are rebuilt and B_L^+ recomputed.
    // Runs on the solve's stream after a host synchronisation (the old operators are no
    // longer in use); the captured Arnoldi step is dropped, its pointers being stale.
    void mle_restart(const double* x) {
        BAMG_CK(cudaStreamSynchronize(s));
        AllocStream as_(s);
        const int n = lv[0]->n;
        {
            TmpBuf<double> nrm(2, s), part((size_t)dots_partial_blocks(n) + 64, s);
            dots(n, x, n, 1, x, nrm.get(), part.get(), s);
            BAMG_LAUNCH(k_state_col<T>, blocks_for(n, 256), 256, 0, s, n, x, (const double*)nrm.get(), lv[0]->X.get(), ld,
                        ldU);
        }
        for (int l = 0; l < L_idx; ++l) {
            BAMG_CK(cudaMemsetAsync(lv[l]->sel.get(), 1, 1, s));
            interp_step(l, true);
            inject_cols<T>(lv[l + 1]->n, lv[l]->c2f.get(), lv[l]->X.get(), lv[l + 1]->X.get(), ld, ldU, 1, s);
        }
        coarse_pinv_now();
        build_colours();
        check_search_overflow();
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        ++mle_restarts;
    }
    int mle_restarts = 0;

    // --------------------------------------------------------------- import
    void import(int nlev, const bamg_level_in* in, const double* h_pinv, const double* h_x_init) {
        AllocStream as_(s);
        lv.clear();
        for (int l = 0; l < nlev; ++l) {
            auto L = std::make_unique<LevelT<T>>();
            L->n = in[l].n;
            L->nnz = in[l].nnz;
            L->rp.alloc(L->n + 1);
            L->ci.alloc(std::max(L->nnz, 1));
            L->bv.alloc(std::max(L->nnz, 1));
            BAMG_CK(cudaMemcpyAsync(L->rp.get(), in[l].h_row_ptr, sizeof(int32_t) * (L->n + 1), cudaMemcpyHostToDevice, s));
            BAMG_CK(cudaMemcpyAsync(L->ci.get(), in[l].h_col, sizeof(int32_t) * L->nnz, cudaMemcpyHostToDevice, s));
            DevBuf<double> v64(std::max(L->nnz, 1));
            BAMG_CK(cudaMemcpyAsync(v64.get(), in[l].h_val, sizeof(double) * L->nnz, cudaMemcpyHostToDevice, s));
            if constexpr (std::is_same<T, double>::value) {
                L->bv = std::move(v64);
            } else {
                launch_convert<double, float>(L->nnz, v64.get(), L->bv.get(), s);
                if (l == 0) b64_own = std::move(v64);
                BAMG_CK(cudaStreamSynchronize(s));
            }
            L->diagonals(s);
            if (l + 1 < nlev) {
                const int c = o.caliber;
                std::vector<int32_t> pcol((size_t)L->n * c, -1), pcnt(L->n, 0);
                std::vector<T> pval((size_t)L->n * c, T(0));
                for (int i = 0; i < L->n; ++i) {
                    const int a = in[l].h_p_row_ptr[i], b = in[l].h_p_row_ptr[i + 1];
                    BAMG_REQUIRE(b - a <= c, BAMG_EINVAL, "import: a row of P has more than `caliber` entries");
                    pcnt[i] = b - a;
                    for (int q = a; q < b; ++q) {
                        pcol[(size_t)i * c + (q - a)] = in[l].h_p_col[q];
                        pval[(size_t)i * c + (q - a)] = (T)in[l].h_p_val[q];
                    }
                }
                L->pcol.alloc(pcol.size());
                L->pval.alloc(pval.size());
                L->pcnt.alloc(pcnt.size());
                BAMG_CK(cudaMemcpyAsync(L->pcol.get(), pcol.data(), sizeof(int32_t) * pcol.size(), cudaMemcpyHostToDevice, s));
                BAMG_CK(cudaMemcpyAsync(L->pval.get(), pval.data(), sizeof(T) * pval.size(), cudaMemcpyHostToDevice, s));
                BAMG_CK(cudaMemcpyAsync(L->pcnt.get(), pcnt.data(), sizeof(int32_t) * pcnt.size(), cudaMemcpyHostToDevice, s));
                L->nc = in[l + 1].n;
                build_restriction<T>(L->P(c), L->nc, L->qrp, L->qci, L->qv, s);
                BAMG_CK(cudaStreamSynchronize(s));
            }
            lv.push_back(std::move(L));
        }
        b64 = std::is_same<T, double>::value ? reinterpret_cast<const double*>(lv[0]->bv.get()) : b64_own.get();
        nL = lv.back()->n;
        pinv64.alloc((size_t)nL * nL);
        BAMG_CK(cudaMemcpyAsync(pinv64.get(), h_pinv, sizeof(double) * nL * nL, cudaMemcpyHostToDevice, s));
        pinvT.alloc((size_t)nL * nL);
        launch_convert<double, T>((int64_t)nL * nL, pinv64.get(), pinvT.get(), s);
        x_init.alloc(lv[0]->n);
        BAMG_CK(cudaMemcpyAsync(x_init.get(), h_x_init, sizeof(double) * lv[0]->n, cudaMemcpyHostToDevice, s));
        build_colours();
        alloc_vcycle_work();
        BAMG_CK(cudaStreamSynchronize(s));
    }

    // --------------------------------------------------------------- V-cycle
    int precision() const override { return std::is_same<T, float>::value ? BAMG_F32 : BAMG_F64; }

    void smooth_apply(int level, int sweeps, const void* b, void* x, void* work) override {
        check_setup_flags(false);
        BAMG_REQUIRE(level >= 0 && level < (int)lv.size(), BAMG_EINVAL, "smooth_apply: no such level");
        BAMG_REQUIRE(sweeps >= 0, BAMG_EINVAL, "smooth_apply: sweeps < 0");
        VLevel<T> v;
        v.B = lv[level]->B();
        v.dinv = lv[level]->dinv.get();
        smooth_sweeps<T>(v, (const T*)b, (T*)x, (T*)work, o.omega, sweeps, s);
    }

    // power iteration on the residual propagator I - B C (see bamg_vcycle_factor)
    double vcycle_factor(int iters) override {
        check_setup_flags(false);
        AllocStream as_(s);
        const int n = lv[0]->n;
        const MatView<double> B = B64();
        TmpBuf<double> x(n, s), r(n, s), z(n, s), t(n, s), mom(2, s);
        if (!h_pin) BAMG_CK(cudaMallocHost(&h_pin, 32 * sizeof(double)));
        BAMG_LAUNCH(k_vf_start, blocks_for(n, 256), 256, 0, s, n, x.get());
        spmv_f64(B, x.get(), r.get(), 1.0, s);
        auto normalise = [&]() {  // r <- (r - mean) / ||r - mean||; returns the norm
            BAMG_CK(cudaMemsetAsync(mom.get(), 0, 2 * sizeof(double), s));
            BAMG_LAUNCH(k_vf_moments, blocks_for(n, 256), 256, 0, s, n, (const double*)r.get(), mom.get());
            BAMG_CK(cudaMemcpyAsync(h_pin, mom.get(), 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            BAMG_CK(cudaStreamSynchronize(s));
            const double mean = h_pin[0] / n;
            const double nrm = std::sqrt(std::max(h_pin[1] - n * mean * mean, 0.0));
            BAMG_LAUNCH(k_vf_affine, blocks_for(n, 256), 256, 0, s, n, r.get(), mean, nrm > 0.0 ? 1.0 / nrm : 0.0);
            return nrm;
        };
        normalise();
        std::vector<double> logs;
        for (int k = 0; k < iters; ++k) {
            vcycle_apply(r.get(), z.get());
            spmv_f64(B, z.get(), t.get(), 1.0, s);
            BAMG_LAUNCH(k_vf_axpy, blocks_for(n, 256), 256, 0, s, n, r.get(), (const double*)t.get());
            const double nr = normalise();
            if (!(nr > 0.0)) break;
            logs.push_back(std::log(nr));
        }
        if (logs.empty()) return 0.0;
        double acc = 0.0;
        const size_t h = logs.size() / 2;
        for (size_t k = h; k < logs.size(); ++k) acc += logs[k];
        return std::exp(acc / (double)(logs.size() - h));
    }

    void vcycle_apply(const double* v, double* z) override {
        check_setup_flags(false);
        AllocStream as_(s);
        const int n = lv[0]->n;
        if constexpr (std::is_same<T, double>::value) {
            auto vl = vlevels(v, z);
            vcycle<T>(vl, pinvT.get(), o.omega, o.nu_pre, o.nu_post, s);
        } else {
            vin.ensure(n);
            TmpBuf<float> zo(n, s);
            launch_convert<double, float>(n, v, vin.get(), s);
            auto vl = vlevels(vin.get(), zo.get());
            vcycle<T>(vl, pinvT.get(), o.omega, o.nu_pre, o.nu_post, s);
            launch_convert<float, double>(n, zo.get(), z, s);
        }
    }

    // --------------------------------------------------------------- FGMRES
    double read_d(const double* d) {
        BAMG_CK(cudaMemcpyAsync(h_pin, d, sizeof(double), cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
        return h_pin[0];
    }
    void read_n(const double* d, int k) {
        BAMG_CK(cudaMemcpyAsync(h_pin, d, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
    }

    // One Arnoldi step captured as a CUDA graph.  Preferred form: the step is the body of
    // a WHILE conditional node, so one launch runs steps until the step's last kernel
    // stops the loop (the host's own test for a true residual check) and the host waits
    // once per check instead of once per step.  Where the driver refuses the conditional
    // node the graph is one step per launch.
    void capture_step(int n) {
        if (!ctl.get()) ctl.alloc(3);
        if (!(o.device_loop && capture_step_graph(n, true))) capture_step_graph(n, false);
    }
    bool capture_step_graph(int n, bool loop) {
        std::vector<VLevel<T>> vl = vlevels(vin.get(), zout.get());
        const uint64_t c0 = t_launches;  // other threads may launch meanwhile
        cudaGraph_t g = nullptr;
        cudaGraphConditionalHandle cond = 0;
        cudaGraphNode_t cnode = nullptr;
        if (loop) {
            BAMG_CK(cudaGraphCreate(&g, 0));
            bool ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
            cudaGraphNodeParams p = {};
            if (ok) {
                p.type = cudaGraphNodeTypeConditional;
                p.conditional.handle = cond;
                p.conditional.type = cudaGraphCondTypeWhile;
                p.conditional.size = 1;
                ok = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &p) == cudaSuccess;
            }
            if (ok)
                ok = cudaStreamBeginCaptureToGraph(s, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                cudaGraphDestroy(g);
                return false;
            }
        } else {
            BAMG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        }
        try {
            PdlScope pdl_;  // programmatic edges between the step's kernels
            arnoldi_step_graphable<T>(n, B64(), V.get(), Z.get(), vin.get(), zout.get(), dj.get(), state.get(), m,
                                      partial.get(), vl, pinvT.get(), o.omega, o.nu_pre, o.nu_post, h_pin, ctl.get(),
                                      cond, s);
        } catch (...) {
            cudaGraph_t c = nullptr;
            cudaStreamEndCapture(s, &c);
            if (loop) {
                if (g) cudaGraphDestroy(g);
            } else if (c) {
                cudaGraphDestroy(c);
            }
            throw;
        }
        cudaGraph_t c = nullptr;
        BAMG_CK(cudaStreamEndCapture(s, &c));
        if (!loop) g = c;
        const int64_t kernels = (int64_t)(t_launches - c0);
        count_launches(-kernels);  // counted again at every executed step
        int64_t post = 0;
        if (loop) {
            // after the loop: the true residual check that every stop of the loop calls for
            // (y from R and g, x = x_0 + Z y, the residual sums), on the device, so that the
            // host reads the stop and the check together
            const uint64_t c1 = t_launches;
            GmresLayout GL(m);
            BAMG_CK(cudaStreamBeginCaptureToGraph(s, g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
            try {
                gmres_solve_y(state.get(), 0, m, s, dj.get());
                form_x<T>(n, x0.get(), Z.get(), n, 0, state.get() + GL.y, xw.get(), s, dj.get());
                residual_norms(B64(), xw.get(), rn.get(), partial.get(), s);
            } catch (...) {
                cudaGraph_t c2 = nullptr;
                cudaStreamEndCapture(s, &c2);
                cudaGraphDestroy(g);
                throw;
            }
            cudaGraph_t c2 = nullptr;
            BAMG_CK(cudaStreamEndCapture(s, &c2));
            post = (int64_t)(t_launches - c1);
            count_launches(-post);
        }
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            if (loop) return false;
            throw Error(BAMG_ECUDA, "cudaGraphInstantiate of the Arnoldi step failed");
        }
        graph = g;
        gexec = ex;
        graph_kernels = kernels;
        graph_post = post;
        graph_loop = loop;
        return true;
    }

    void ensure_private_stream() {
        if (!h_pin) BAMG_CK(cudaMallocHost(&h_pin, 32 * sizeof(double)));
        if (!ps) {
            BAMG_CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
            BAMG_CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
            BAMG_CK(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
        }
    }
    // runs f with s = the private stream, fenced against the caller's stream on both sides
    template <typename F>
    void on_private_stream(F&& f) {
        ensure_private_stream();
        cudaStream_t su = s;
        BAMG_CK(cudaEventRecord(ev_in, su));
        BAMG_CK(cudaStreamWaitEvent(ps, ev_in, 0));
        s = ps;
        try {
            f();
        } catch (...) {
            cudaEventRecord(ev_out, ps);
            cudaStreamWaitEvent(su, ev_out, 0);
            s = su;
            throw;
        }
        BAMG_CK(cudaEventRecord(ev_out, ps));
        BAMG_CK(cudaStreamWaitEvent(su, ev_out, 0));
        s = su;
    }

    void solve(double* x_user, int flags, double tol, bamg_stats* st) override {
        AllocStream as_(s);
        const int n = lv[0]->n;
        m = std::min(std::max(o.gmres_m, 1), GMRES_MMAX);
        GmresLayout GL(m);
        V.ensure((size_t)n * (m + 1));
        Z.ensure((size_t)n * m);
        state.ensure(GL.total);
        const int pb = std::max({dots_partial_blocks(n) * (m + 1), (int)blocks_for(n, 256) * RESNORM_SUMS,
                                 2 * arn_tiles(n) * (m + 1)});
        partial.ensure(pb);
        x0.ensure(n);
        xw.ensure(n);
        rn.ensure(8);
        vin.ensure(n);
        zout.ensure(n);
        dj.ensure(2);  // j and the Arnoldi kernels' last-block ticket
        // all work of the solve runs on the private stream, fenced against the caller's
        on_private_stream([&] { solve_on_private_stream(x_user, flags, tol, st); });
    }

    // --------------------------------------------------------------- pArnoldi (Section 4.3)
    DevBuf<double> Hh, eta, zero;
    void parnoldi(double* x_user, int flags, double tol, bamg_stats* st) override {
        check_setup_flags(false);
        AllocStream as_(s);
        const int n = lv[0]->n;
        const int mp = std::min(std::max(o.gmres_m, 1), PARN_MMAX);
        GmresLayout GL(mp);
        V.ensure((size_t)n * (mp + 1));
        state.ensure(GL.total);
        partial.ensure(std::max({dots_partial_blocks(n) * (mp + 1), (int)blocks_for(n, 256) * RESNORM_SUMS,
                                 2 * arn_tiles(n) * (mp + 1)}));
        x0.ensure(n);
        xw.ensure(n);
        rn.ensure(8);
        vin.ensure(n);
        zout.ensure(n);
        dj.ensure(2);  // j and the Arnoldi kernels' last-block ticket
        Hh.ensure((size_t)(mp + 1) * mp);
        eta.ensure(mp);
        if (zero.n < (size_t)n) {
            zero.ensure(n);
            BAMG_CK(cudaMemsetAsync(zero.get(), 0, sizeof(double) * n, s));
        }
        on_private_stream([&] { parnoldi_on_private_stream(mp, x_user, flags, tol, st); });
    }

    // Arnoldi on C B from y = the setup's state-vector approximation (or the guess); after
    // every step the Ritz vector x = V_k eta of the eigenvalue of H_k closest to 0 and its
    // true residual; after mp steps a restart from the Ritz vector.
    void parnoldi_on_private_stream(int mp, double* x_user, int flags, double tol, bamg_stats* st) {
        auto t0 = std::chrono::steady_clock::now();
        const int n = lv[0]->n;
        GmresLayout GL(mp);
        const MatView<double> B = B64();
        const bool l2 = (flags & BAMG_NORM_L2) != 0;
        if (flags & BAMG_X_GUESS)
            BAMG_CK(cudaMemcpyAsync(x0.get(), x_user, sizeof(double) * n,
                                    (flags & BAMG_X_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        else
            BAMG_CK(cudaMemcpyAsync(x0.get(), x_init.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        std::vector<VLevel<T>> vl = vlevels(vin.get(), zout.get());
        int it = 0, restarts = 0, checks = 0, status = BAMG_ENOCONV;
        residual_norms(B, x0.get(), rn.get(), partial.get(), s);
        read_n(rn.get(), RESNORM_SUMS);
        double ratio1 = h_pin[0] / h_pin[2];
        double ratio = l2 ? std::sqrt(h_pin[1] / h_pin[4]) : ratio1, xsum = h_pin[3];
        double* xfinal = x0.get();
        if (ratio <= tol) status = BAMG_OK;
        while (status != BAMG_OK && it < o.max_it) {
            double* V0 = V.get();
            dots(n, x0.get(), n, 1, x0.get(), state.get() + GL.nrm2, partial.get(), s);
            gmres_init(state.get(), mp, s);
            scale_vec(n, x0.get(), state.get(), GL.hn, true, V0, s);
            BAMG_CK(cudaMemsetAsync(dj.get(), 0, 2 * sizeof(int), s));
            bool stop = false;
            for (int j = 0; j < mp && it < o.max_it; ++j) {
                parnoldi_step<T>(n, B, V.get(), vin.get(), zout.get(), dj.get(), state.get(), mp, Hh.get(), mp + 1,
                                 partial.get(), vl, pinvT.get(), o.omega, o.nu_pre, o.nu_post, s);
                ++it;
                ritz_closest_to_zero(Hh.get(), mp + 1, j + 1, eta.get(), s);
                form_x<double>(n, zero.get(), V.get(), n, j + 1, eta.get(), xw.get(), s);
                residual_norms(B, xw.get(), rn.get(), partial.get(), s);
                BAMG_CK(cudaMemcpyAsync(h_pin + 8, state.get() + GL.hn, sizeof(double), cudaMemcpyDeviceToHost, s));
                read_n(rn.get(), RESNORM_SUMS);
                ++checks;
                xfinal = xw.get();
                ratio1 = h_pin[0] / h_pin[2];
                ratio = l2 ? std::sqrt(h_pin[1] / h_pin[4]) : ratio1;
                xsum = h_pin[3];
                if (!(ratio == ratio)) throw Error(BAMG_ENUMERIC, "NaN in the Arnoldi iteration");
                if (ratio <= tol) {
                    status = BAMG_OK;
                    stop = true;
                    break;
                }
                if (h_pin[8] == 0.0) {  // invariant subspace: the Ritz vector is final
                    stop = true;
                    break;
                }
            }
            if (stop) break;
            BAMG_CK(cudaMemcpyAsync(x0.get(), xw.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            xfinal = x0.get();
            ++restarts;
        }
        TmpBuf<double> out(n, s);
        h_pin[9] = xsum;
        BAMG_CK(cudaMemcpyAsync(rn.get() + 5, h_pin + 9, sizeof(double), cudaMemcpyHostToDevice, s));
        scale_vec(n, xfinal, rn.get(), 5, true, out.get(), s);
        BAMG_CK(cudaMemcpyAsync(x_user, out.get(), sizeof(double) * n,
                                (flags & BAMG_X_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        BAMG_CK(cudaStreamSynchronize(s));
        if (st) {
            std::memset(st, 0, sizeof(*st));
            st->status = status;
            st->iterations = it;
            st->restarts = restarts;
            st->true_checks = checks;
            st->host_waits = checks;
            st->residual_l1 = ratio1;
            st->setup_ms = setup_ms;
            st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        if (status != BAMG_OK) throw Error(status, "pArnoldi did not reach the tolerance within max_it iterations");
    }

    // --------------------------------------------------------------- stand-alone MLE (Section 4.1)
    void mle_setup(const bamg_csr* A, int r_, int levels, double tol, int max_cycles, bool l2, double* x, bool x_host,
                   bamg_stats* st) override {
        int cycles = 0;
        double rat[2] = {INFINITY, INFINITY};
        setup(A, r_, levels, tol, max_cycles, l2, &cycles, rat);
        const int n = lv[0]->n;
        if (x) {  // the last cycle's state vector approximation, 1^T x = 1 (x_init)
            BAMG_CK(cudaMemcpyAsync(x, x_init.get(), sizeof(double) * n,
                                    x_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
            BAMG_CK(cudaStreamSynchronize(s));
        }
        const double ratio = rat[l2 ? 1 : 0];
        if (st) {
            std::memset(st, 0, sizeof(*st));
            st->status = ratio <= tol ? BAMG_OK : BAMG_ENOCONV;
            st->iterations = cycles;
            st->residual_l1 = rat[0];
            st->setup_ms = setup_ms;
        }
        if (!(ratio <= tol)) throw Error(BAMG_ENOCONV, "MLE did not reach the tolerance within max_cycles cycles");
    }

    void solve_on_private_stream(double* x_user, int flags, double tol, bamg_stats* st) {
        auto t0 = std::chrono::steady_clock::now();
        const int n = lv[0]->n;
        GmresLayout GL(m);
        const MatView<double> B = B64();
        if (flags & BAMG_X_GUESS) {
            BAMG_CK(cudaMemcpyAsync(x0.get(), x_user, sizeof(double) * n,
                                    (flags & BAMG_X_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        } else {
            BAMG_CK(cudaMemcpyAsync(x0.get(), x_init.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
        int it = 0, restarts = 0, checks = 0, waits = 0, status = BAMG_ENOCONV;
        const int restarts0 = mle_restarts;
        // stopping test: ||B x||_1 / ||x||_1 <= tol, or with BAMG_NORM_L2 the 2-norm ratio
        // (the criterion of the paper's tables); ratio1 is always the l1 ratio
        const bool l2 = (flags & BAMG_NORM_L2) != 0;
        bool persist = o.persistent != 0;  // steps in one cooperative launch where the hierarchy qualifies
        if (persist) {
            if (!ctl.get()) ctl.alloc(3);
            pbar.ensure(2);
            perr.ensure(1);
        }
        residual_norms(B, x0.get(), rn.get(), partial.get(), s);
        // a restart cycle's start: v_1 = r_0 / ||r_0||, g = beta e_1, j = 0
        auto cycle_start = [&] {
            double* V0 = V.get();
            spmv_f64(B, x0.get(), V0, -1.0, s);
            dots(n, V0, n, 1, V0, state.get() + GL.nrm2, partial.get(), s);
            gmres_init(state.get(), m, s);
            scale_vec(n, V0, state.get(), GL.hn, true, V0, s);
            BAMG_CK(cudaMemsetAsync(dj.get(), 0, 2 * sizeof(int), s));
        };
        // the first cycle's start is queued before the residual is read and the step is
        // captured meanwhile, so the device works while the host captures (the start goes
        // unused when x_0 already meets the tolerance)
        cycle_start();
        bool started = true;
        if (!persist && !gexec) capture_step(n);
        read_n(rn.get(), RESNORM_SUMS);
        check_setup_flags(true);  // the setup's copy preceded this wait on the caller's stream
        double ratio1 = h_pin[0] / h_pin[2];
        double ratio = l2 ? std::sqrt(h_pin[1] / h_pin[4]) : ratio1;
        double x1 = l2 ? std::sqrt(h_pin[4]) : h_pin[2], xsum = h_pin[3], last_x1 = x1;
        double kappa = 1.0;
        bool have_xw = false;
        if (ratio <= tol) status = BAMG_OK;
        while (status != BAMG_OK && it < o.max_it) {
            if (!persist && !gexec) capture_step(n);
            if (!started) cycle_start();
            started = false;
            for (int j = 0; j < m && it < o.max_it; ++j) {
                bool launched = false, checked = false;  // checked: the graph formed the check's sums
                if (persist) {  // steps j .. jn - 1 in one cooperative launch
                    h_pin[12] = kappa;
                    h_pin[13] = tol * x1;
                    h_pin[14] = (double)std::min(m, j + (o.max_it - it));
                    BAMG_CK(cudaMemcpyAsync(ctl.get(), h_pin + 12, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
                    std::vector<VLevel<T>> vl = vlevels(vin.get(), zout.get());
                    launched = arnoldi_cycle_persistent<T>(n, B, V.get(), Z.get(), vin.get(), dj.get(), state.get(), m,
                                                           partial.get(), vl, pinvT.get(), o.omega, o.nu_pre,
                                                           o.nu_post, ctl.get(), pbar.get(), perr.get(), s);
                    if (launched) {
                        BAMG_CK(cudaMemcpyAsync(h_pin, state.get() + GL.est, 2 * sizeof(double),
                                                cudaMemcpyDeviceToHost, s));
                        BAMG_CK(cudaMemcpyAsync(h_pin + 4, dj.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
                        BAMG_CK(cudaMemcpyAsync(h_pin + 5, perr.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
                        BAMG_CK(cudaStreamSynchronize(s));
                        ++waits;
                        BAMG_REQUIRE(*reinterpret_cast<const int*>(h_pin + 5) == 0, BAMG_ETIMEOUT,
                                     "persistent Arnoldi cycle: a grid barrier wait gave up");
                        const int jn = *reinterpret_cast<const int*>(h_pin + 4);
                        BAMG_REQUIRE(jn > j && jn <= (int)h_pin[14], BAMG_ECUDA,
                                     "persistent Arnoldi cycle: bad step count");
                        it += jn - j;
                        j = jn - 1;
                    } else {  // this hierarchy runs the captured step
                        persist = false;
                        if (!gexec) capture_step(n);
                    }
                }
                if (launched) {
                } else if (graph_loop) {  // steps j .. jn - 1 in one launch
                    h_pin[12] = kappa;
                    h_pin[13] = tol * x1;
                    h_pin[14] = (double)std::min(m, j + (o.max_it - it));
                    BAMG_CK(cudaMemcpyAsync(ctl.get(), h_pin + 12, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
                    BAMG_CK(cudaGraphLaunch(gexec, s));
                    BAMG_CK(cudaMemcpyAsync(h_pin, state.get() + GL.est, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                            s));
                    BAMG_CK(cudaMemcpyAsync(h_pin + 4, dj.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
                    BAMG_CK(cudaMemcpyAsync(h_pin + 16, rn.get(), RESNORM_SUMS * sizeof(double), cudaMemcpyDeviceToHost,
                                            s));
                    BAMG_CK(cudaStreamSynchronize(s));
                    ++waits;
                    const int jn = *reinterpret_cast<const int*>(h_pin + 4);
                    BAMG_REQUIRE(jn > j && jn <= (int)h_pin[14], BAMG_ECUDA, "device-side Arnoldi loop: bad step count");
                    count_launches(graph_kernels * (jn - j) + graph_post);
                    checked = true;
                    it += jn - j;
                    j = jn - 1;
                } else {
                    BAMG_CK(cudaGraphLaunch(gexec, s));
                    count_launches(graph_kernels);
                    BAMG_CK(cudaStreamSynchronize(s));
                    ++waits;
                    ++it;
                }
                const double est = h_pin[0], hn = h_pin[1];
                const bool last = (j == m - 1) || it >= o.max_it || hn == 0.0;
                if (est * kappa <= tol * x1 || last) {
                    if (checked) {  // formed by the graph after its loop, read with the stop
                        for (int k = 0; k < RESNORM_SUMS; ++k) h_pin[k] = h_pin[16 + k];
                    } else {
                        gmres_solve_y(state.get(), j, m, s);
                        form_x<T>(n, x0.get(), Z.get(), n, j + 1, state.get() + GL.y, xw.get(), s);
                        residual_norms(B, xw.get(), rn.get(), partial.get(), s);
                        read_n(rn.get(), RESNORM_SUMS);
                    }
                    ++checks;
                    have_xw = true;
                    const double r1 = h_pin[0], r2 = std::sqrt(h_pin[1]);
                    ratio1 = r1 / h_pin[2];
                    ratio = l2 ? r2 / std::sqrt(h_pin[4]) : ratio1;
                    last_x1 = l2 ? std::sqrt(h_pin[4]) : h_pin[2];
                    xsum = h_pin[3];
                    if (r2 > 0.0 && !l2) kappa = std::max(1.0, r1 / r2);
                    if (!(ratio == ratio)) throw Error(BAMG_ENUMERIC, "NaN in the Krylov iteration");
                    if (ratio <= tol) {
                        status = BAMG_OK;
                        break;
                    }
                    if (last) break;
                }
            }
            if (status == BAMG_OK) break;
            if (have_xw) {  // restart from the last iterate
                BAMG_CK(cudaMemcpyAsync(x0.get(), xw.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                x1 = last_x1;
            }
            ++restarts;
            // an imported hierarchy carries no test vectors: plain restarts there
            if (o.mle_restart && it < o.max_it && L_idx >= 0 && nvec > 0) mle_restart(x0.get());
        }
        double* xfinal = have_xw ? xw.get() : x0.get();
        // normalise 1^T x = 1
        TmpBuf<double> out(n, s);
        h_pin[8] = xsum;
        BAMG_CK(cudaMemcpyAsync(rn.get() + 5, h_pin + 8, sizeof(double), cudaMemcpyHostToDevice, s));
        scale_vec(n, xfinal, rn.get(), 5, true, out.get(), s);
        if (flags & BAMG_X_HOST)
            BAMG_CK(cudaMemcpyAsync(x_user, out.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        else
            BAMG_CK(cudaMemcpyAsync(x_user, out.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        BAMG_CK(cudaStreamSynchronize(s));
        if (st) {
            st->status = status;
            st->iterations = it;
            st->restarts = restarts;
            st->true_checks = checks;
            st->host_waits = waits;
            st->mle_restarts = mle_restarts - restarts0;
            st->residual_l1 = ratio1;
            st->setup_ms = setup_ms;
            st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        if (status != BAMG_OK) throw Error(status, "FGMRES did not reach the tolerance within max_it iterations");
    }

    // --------------------------------------------------------------- export
    template <typename S>
    static void to_host_double(const S* d, size_t cnt, double* h, cudaStream_t s) {
        std::vector<S> tmp(cnt);
        if (cnt) BAMG_CK(cudaMemcpyAsync(tmp.data(), d, sizeof(S) * cnt, cudaMemcpyDeviceToHost, s));
        BAMG_CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < cnt; ++i) h[i] = (double)tmp[i];
    }
    void export_obj(int l, int what, void* h_dst, int64_t cap, int64_t* bytes) override {
        check_setup_flags(false);
        BAMG_REQUIRE(l >= 0 && l < (int)lv.size(), BAMG_EINVAL, "export: level out of range");
        LevelT<T>& L = *lv[l];
        int64_t need = 0;
        switch (what) {
            case BAMG_EXPORT_B: need = 4LL * (L.n + 1) + 4LL * L.nnz + 8LL * L.nnz; break;
            case BAMG_EXPORT_T: need = 8LL * L.nnz; break;
            case BAMG_EXPORT_P:
                BAMG_REQUIRE(l + 1 < (int)lv.size(), BAMG_EINVAL, "export: the coarsest level has no P");
                need = 4LL * L.n * o.caliber + 4LL * L.n + 8LL * L.n * o.caliber;
                break;
            case BAMG_EXPORT_CF:
                BAMG_REQUIRE(l + 1 < (int)lv.size(), BAMG_EINVAL, "export: the coarsest level has no splitting");
                need = L.n;
                break;
            case BAMG_EXPORT_X: need = 8LL * L.n * ld; break;
            case BAMG_EXPORT_PINV: need = 8LL * nL * nL; break;
            case BAMG_EXPORT_XINIT: need = 8LL * lv[0]->n; break;
            case BAMG_EXPORT_LAMBDA: need = 8LL * nvec; break;
            default: throw Error(BAMG_EINVAL, "export: unknown object");
        }
        if (bytes) *bytes = need;
        if (cap < need) throw Error(BAMG_ESIZE, "export: capacity too small");
        char* h = (char*)h_dst;
        switch (what) {
            case BAMG_EXPORT_B:
                BAMG_CK(cudaMemcpyAsync(h, L.rp.get(), 4LL * (L.n + 1), cudaMemcpyDeviceToHost, s));
                BAMG_CK(cudaMemcpyAsync(h + 4LL * (L.n + 1), L.ci.get(), 4LL * L.nnz, cudaMemcpyDeviceToHost, s));
                if (l == 0 && b64) {
                    BAMG_CK(cudaMemcpyAsync(h + 4LL * (L.n + 1) + 4LL * L.nnz, b64, 8LL * L.nnz, cudaMemcpyDeviceToHost, s));
                    BAMG_CK(cudaStreamSynchronize(s));
                } else {
                    to_host_double(L.bv.get(), L.nnz, (double*)(h + 4LL * (L.n + 1) + 4LL * L.nnz), s);
                }
                break;
            case BAMG_EXPORT_T: to_host_double(L.tv.get(), L.nnz, (double*)h, s); break;
            case BAMG_EXPORT_P:
                BAMG_CK(cudaMemcpyAsync(h, L.pcol.get(), 4LL * L.n * o.caliber, cudaMemcpyDeviceToHost, s));
                BAMG_CK(cudaMemcpyAsync(h + 4LL * L.n * o.caliber, L.pcnt.get(), 4LL * L.n, cudaMemcpyDeviceToHost, s));
                to_host_double(L.pval.get(), (size_t)L.n * o.caliber, (double*)(h + 4LL * L.n * o.caliber + 4LL * L.n), s);
                break;
            case BAMG_EXPORT_CF: BAMG_CK(cudaMemcpyAsync(h, L.cf.get(), L.n, cudaMemcpyDeviceToHost, s)); break;
            case BAMG_EXPORT_X: to_host_double(L.X.get(), (size_t)L.n * ld, (double*)h, s); break;
            case BAMG_EXPORT_PINV: to_host_double(pinv64.get(), (size_t)nL * nL, (double*)h, s); break;
            case BAMG_EXPORT_XINIT: to_host_double(x_init.get(), (size_t)lv[0]->n, (double*)h, s); break;
            case BAMG_EXPORT_LAMBDA: to_host_double(L.lam.get(), (size_t)nvec, (double*)h, s); break;
        }
        BAMG_CK(cudaStreamSynchronize(s));
    }
};

}  // namespace bamg

// =================================================================== C ABI
using namespace bamg;

struct bamg_handle {
    std::unique_ptr<SolverBase> impl;
};

template <typename F>
static int guarded(F&& f) {
    try {
        f();
        g_err.clear();
        return BAMG_OK;
    } catch (const Error& e) {
        g_err = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return BAMG_ENOMEM;
    } catch (const std::exception& e) {
        g_err = e.what();
        return BAMG_EINVAL;
    }
}

extern "C" {

int bamg_default_opts(bamg_opts* o) {
    if (!o) return BAMG_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->omega = 0.7;
    o->nu_tv = 4;
    o->nu_ev = 2;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->caliber = 2;
    o->z = 2;
    o->mmax = 16;
    o->k_ev = 6;
    o->coarse_max = 64;
    o->gmres_m = 50;
    o->max_it = 500;
    o->precision = BAMG_PREC_FP64;
    o->coarsen = BAMG_COARSEN_GRID;
    o->seed = 0;
    o->tv_lo = 1.0;
    o->tv_hi = 2.0;
    o->ev_change_tol = 1e-3;
    o->ridge = 1e-4;
    o->ridge32 = 1e-4;
    o->weight_floor = 1e-28;
    o->cr_theta = 0.85;
    o->cr_nu = 8;
    o->cr_max_rounds = 20;
    o->cr_omega = 0.7;
    o->stream = nullptr;
    o->interp = BAMG_INTERP_LS;
    o->learned_refit = 1;
    o->model = nullptr;
    o->learned_rho_max = 0.0;
    o->device_loop = 1;
    o->mle_restart = 1;
    o->setup_cycles = 1;
    o->mu = 1;
    o->smoother = BAMG_SMOOTH_JACOBI;
    o->persistent = 0;
    o->coarse_tail = 0;
    return BAMG_OK;
}

static void check_opts(const bamg_opts& o) {
    BAMG_REQUIRE(o.caliber >= 1 && o.caliber <= 4, BAMG_EINVAL, "caliber must be 1..4");
    BAMG_REQUIRE(o.z >= 1 && o.z <= 3, BAMG_EINVAL, "z must be 1..3");
    BAMG_REQUIRE(o.mmax >= 1 && o.mmax <= 16, BAMG_EINVAL, "mmax must be 1..16");
    BAMG_REQUIRE(o.k_ev >= 1 && o.k_ev <= 15, BAMG_EINVAL, "k_ev must be 1..15");
    BAMG_REQUIRE(o.coarse_max >= 1 && o.coarse_max <= 64, BAMG_EINVAL, "coarse_max must be 1..64");
    BAMG_REQUIRE(o.nu_pre >= 0 && o.nu_post >= 0 && o.nu_tv >= 0 && o.nu_ev >= 0, BAMG_EINVAL, "negative sweep count");
    BAMG_REQUIRE(o.gmres_m >= 1 && o.gmres_m <= GMRES_MMAX, BAMG_EINVAL, "gmres_m must be 1..256");
    BAMG_REQUIRE(o.max_it >= 1, BAMG_EINVAL, "max_it must be >= 1");
    BAMG_REQUIRE(o.precision == BAMG_PREC_FP64 || o.precision == BAMG_PREC_MIXED, BAMG_EINVAL, "bad precision");
    BAMG_REQUIRE(o.coarsen == BAMG_COARSEN_GRID || o.coarsen == BAMG_COARSEN_CR, BAMG_EINVAL, "bad coarsening");
    BAMG_REQUIRE(o.omega > 0.0 && o.omega < 2.0, BAMG_EINVAL, "omega must be in (0, 2)");
    BAMG_REQUIRE(o.interp == BAMG_INTERP_LS || o.interp == BAMG_INTERP_LEARNED, BAMG_EINVAL, "bad interp");
    BAMG_REQUIRE(o.interp == BAMG_INTERP_LS || (o.model && o.model->impl), BAMG_EINVAL,
                 "BAMG_INTERP_LEARNED needs a model");
    BAMG_REQUIRE(o.mu == 1 || o.mu == 2, BAMG_EINVAL, "mu must be 1 (V-cycle setup) or 2 (W-cycle setup)");
    BAMG_REQUIRE(o.setup_cycles >= 1 && o.setup_cycles <= 64, BAMG_EINVAL, "setup_cycles must be 1..64");
    BAMG_REQUIRE(o.smoother == BAMG_SMOOTH_JACOBI || o.smoother == BAMG_SMOOTH_MCGS, BAMG_EINVAL, "bad smoother");
    BAMG_REQUIRE(o.coarse_tail == 0 || o.coarse_tail == 1, BAMG_EINVAL, "coarse_tail must be 0 or 1");
}

static void check_setup_args(const bamg_csr* A, int r, int levels, const bamg_opts& o) {
    check_opts(o);
    BAMG_REQUIRE(A->n >= 2 && A->nnz >= 1, BAMG_EINVAL, "A must have n >= 2 and nnz >= 1");
    BAMG_REQUIRE(A->row_ptr && A->col && A->val, BAMG_EINVAL, "null CSR array");
    BAMG_REQUIRE(r >= 1 && r <= 24, BAMG_EINVAL, "r must be 1..24");
    BAMG_REQUIRE(levels >= 0 && levels <= 30, BAMG_EINVAL, "levels must be 0..30");
    if (o.coarsen == BAMG_COARSEN_GRID)
        BAMG_REQUIRE(o.grid_nx >= 1 && o.grid_ny >= 1 && (int64_t)o.grid_nx * o.grid_ny == A->n, BAMG_EINVAL,
                     "full coarsening needs grid_nx * grid_ny == n");
}

// Builds the hierarchy; with the learned interpolation and learned_rho_max > 0, measures
// the V-cycle factor and falls back to least squares when it exceeds the limit.
static std::unique_ptr<SolverBase> make_solver(const bamg_csr* A, int r, int levels, const bamg_opts& o,
                                               bool record = false, float* rec_feat = nullptr,
                                               float* rec_target = nullptr, int64_t rec_cap = 0) {
    std::unique_ptr<SolverBase> sv;
    if (o.precision == BAMG_PREC_FP64) {
        auto p = std::make_unique<Solver<double>>();
        p->o = o;
        p->s = (cudaStream_t)o.stream;
        p->record = record, p->rec_feat = rec_feat, p->rec_target = rec_target, p->rec_cap = rec_cap;
        p->setup(A, r, levels);
        sv = std::move(p);
    } else {
        auto p = std::make_unique<Solver<float>>();
        p->o = o;
        p->s = (cudaStream_t)o.stream;
        p->record = record, p->rec_feat = rec_feat, p->rec_target = rec_target, p->rec_cap = rec_cap;
        p->setup(A, r, levels);
        sv = std::move(p);
    }
    sv->interp_used = o.interp;
    if (o.interp == BAMG_INTERP_LEARNED && o.learned_rho_max > 0.0) {
        const double rho = sv->vcycle_factor(20);
        if (!(rho <= o.learned_rho_max)) {
            bamg_opts ls = o;
            ls.interp = BAMG_INTERP_LS;
            const double ms = sv->setup_ms;
            sv.reset();
            sv = make_solver(A, r, levels, ls);
            sv->setup_ms += ms;
        }
        sv->rho_measured = rho;
    }
    return sv;
}

int bamg_setup(const bamg_csr* A, int r, int levels, const bamg_opts* opts, bamg_handle** h) {
    return guarded([&] {
        BAMG_REQUIRE(A && h, BAMG_EINVAL, "null argument");
        *h = nullptr;
        bamg_opts o;
        if (opts) o = *opts;
        else bamg_default_opts(&o);
        check_setup_args(A, r, levels, o);
        auto hh = std::make_unique<bamg_handle>();
        hh->impl = make_solver(A, r, levels, o);
        *h = hh.release();
    });
}

int bamg_mle_solve(const bamg_csr* A, int r, int levels, const bamg_opts* opts, double tol, int max_cycles,
                   int flags, double* x, bamg_stats* st, bamg_handle** h) {
    return guarded([&] {
        BAMG_REQUIRE(A, BAMG_EINVAL, "null argument");
        if (h) *h = nullptr;
        BAMG_REQUIRE(tol > 0.0 && max_cycles >= 1, BAMG_EINVAL, "tol must be > 0 and max_cycles >= 1");
        BAMG_REQUIRE(!(flags & BAMG_X_GUESS), BAMG_EINVAL, "the MLE takes no initial guess");
        bamg_opts o;
        if (opts) o = *opts;
        else bamg_default_opts(&o);
        check_setup_args(A, r, levels, o);
        std::unique_ptr<SolverBase> sv;
        if (o.precision == BAMG_PREC_FP64) sv = std::make_unique<Solver<double>>();
        else sv = std::make_unique<Solver<float>>();
        sv->o = o;
        sv->s = (cudaStream_t)o.stream;
        sv->interp_used = o.interp;
        int code = BAMG_OK;
        std::string msg;
        try {
            sv->mle_setup(A, r, levels, tol, max_cycles, (flags & BAMG_NORM_L2) != 0, x, (flags & BAMG_X_HOST) != 0,
                          st);
        } catch (const Error& e) {
            if (e.code != BAMG_ENOCONV) throw;
            code = e.code;
            msg = e.what();
        }
        if (h) {
            auto hh = std::make_unique<bamg_handle>();
            hh->impl = std::move(sv);
            *h = hh.release();
        }
        if (code != BAMG_OK) throw Error(code, msg);
    });
}

int bamg_parnoldi(bamg_handle* h, double* x, int flags, double tol, bamg_stats* st) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl && x, BAMG_EINVAL, "null argument");
        BAMG_REQUIRE(tol >= 0.0, BAMG_EINVAL, "tol must be >= 0");
        h->impl->parnoldi(x, flags, tol, st);
    });
}

int bamg_solve(bamg_handle* h, double* x, int flags, double tol, bamg_stats* st) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl && x, BAMG_EINVAL, "null argument");
        BAMG_REQUIRE(tol > 0.0, BAMG_EINVAL, "tol must be positive");
        if (st) std::memset(st, 0, sizeof(*st));
        h->impl->solve(x, flags, tol, st);
    });
}

void bamg_free(bamg_handle* h) { delete h; }

int bamg_solve_batch(int nchains, const bamg_csr* As, const int* r, const int* levels, const bamg_opts* opts,
                     double* const* xs, int flags, double tol, int nworkers, bamg_stats* st) {
    if (nchains < 0 || (nchains > 0 && (!As || !r || !levels || !opts || !xs))) {
        g_err = "bamg_solve_batch: bad arguments";
        return BAMG_EINVAL;
    }
    if (flags & BAMG_X_GUESS) {
        g_err = "bamg_solve_batch: BAMG_X_GUESS is not supported";
        return BAMG_EINVAL;
    }
    if (nchains == 0) return BAMG_OK;
    if (nworkers <= 0) nworkers = std::min(16, std::max(1, (nchains + 3) / 4));
    nworkers = std::min(nworkers, nchains);
    // largest chains first: the queue ends with the short jobs
    std::vector<int> order(nchains);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return As[a].n > As[b].n; });
    std::atomic<int> next{0};
    std::mutex mu;
    int first_code = BAMG_OK;
    int first_chain = nchains;
    std::string first_msg;
    auto worker = [&]() {
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lock(mu);
            if (first_code == BAMG_OK) {
                first_code = BAMG_ECUDA;
                first_msg = "bamg_solve_batch: stream creation failed";
            }
            return;
        }
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= nchains) break;
            const int k = order[q];
            bamg_opts o = opts[k];
            o.stream = ws;
            // with several host threads, graphs holding a WHILE conditional node slowed the
            // other threads' setups about fourfold (512-chain mixture, 8 workers), more than
            // the device-side loop saves: one graph launch per Arnoldi step here
            if (nworkers > 1) {
                o.device_loop = 0;
                o.persistent = 0;  // a cooperative launch holds every SM: the workers' solves would take turns
            }
            bamg_handle* h = nullptr;
            bamg_stats local{};
            int code = bamg_setup(&As[k], r[k], levels[k], &o, &h);
            if (code == BAMG_OK) code = bamg_solve(h, xs[k], flags & BAMG_X_HOST, tol, &local);
            local.status = code;
            if (st) st[k] = local;
            if (code != BAMG_OK) {
                std::lock_guard<std::mutex> lock(mu);
                if (k < first_chain) {
                    first_chain = k;
                    first_code = code;
                    first_msg = "chain " + std::to_string(k) + ": " + g_err;
                }
            }
            bamg_free(h);
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nworkers; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    g_err = first_msg;
    return first_code;
}

const char* bamg_last_error(void) { return g_err.c_str(); }

uint64_t bamg_launch_count(void) { return g_launches.load(); }

int bamg_hierarchy_info(const bamg_handle* h, int* nlevels, int64_t* h_n, int64_t* h_nnz, double* opc) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl, BAMG_EINVAL, "null handle");
        const int L = h->impl->nlevels();
        if (nlevels) *nlevels = L;
        double tot = 0, n0 = 0;
        for (int l = 0; l < L && l < 32; ++l) {
            int64_t n, nnz;
            h->impl->level_size(l, &n, &nnz);
            if (h_n) h_n[l] = n;
            if (h_nnz) h_nnz[l] = nnz;
            tot += (double)nnz;
            if (l == 0) n0 = (double)nnz;
        }
        if (opc) *opc = tot / n0;
    });
}

int bamg_level_export(const bamg_handle* h, int level, int what, void* h_dst, int64_t cap, int64_t* h_bytes) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl, BAMG_EINVAL, "null handle");
        h->impl->export_obj(level, what, h_dst, cap, h_bytes);
    });
}

int bamg_hierarchy_layout(const bamg_handle* h, int level, int* ld, int* r, int* v_col0, int* nvec) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl, BAMG_EINVAL, "null handle");
        h->impl->layout(level, ld, r, v_col0, nvec);
    });
}

int bamg_import(int nlevels, const bamg_level_in* levels, const double* h_pinv, const double* h_x_init,
                const bamg_opts* opts, bamg_handle** h) {
    return guarded([&] {
        BAMG_REQUIRE(levels && h && h_pinv && h_x_init && nlevels >= 1 && nlevels <= 30, BAMG_EINVAL, "bad import args");
        *h = nullptr;
        bamg_opts o;
        if (opts) o = *opts;
        else bamg_default_opts(&o);
        check_opts(o);
        BAMG_REQUIRE(levels[nlevels - 1].n <= 64, BAMG_EINVAL, "import: coarsest level must have <= 64 states");
        auto hh = std::make_unique<bamg_handle>();
        if (o.precision == BAMG_PREC_FP64) {
            auto sv = std::make_unique<Solver<double>>();
            sv->o = o;
            sv->s = (cudaStream_t)o.stream;
            sv->import(nlevels, levels, h_pinv, h_x_init);
            hh->impl = std::move(sv);
        } else {
            auto sv = std::make_unique<Solver<float>>();
            sv->o = o;
            sv->s = (cudaStream_t)o.stream;
            sv->import(nlevels, levels, h_pinv, h_x_init);
            hh->impl = std::move(sv);
        }
        *h = hh.release();
    });
}

int bamg_smooth_apply(bamg_handle* h, int level, int sweeps, const void* b, void* x, void* work) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl && b && x && work, BAMG_EINVAL, "null argument");
        h->impl->smooth_apply(level, sweeps, b, x, work);
    });
}

int bamg_hierarchy_precision(const bamg_handle* h) { return h && h->impl ? h->impl->precision() : BAMG_EINVAL; }

int bamg_vcycle_factor(bamg_handle* h, int iters, double* rho) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl && rho && iters >= 2, BAMG_EINVAL, "bad vcycle_factor arguments");
        *rho = h->impl->vcycle_factor(iters);
        BAMG_CK(cudaStreamSynchronize(h->impl->s));
    });
}

int bamg_hierarchy_interp(const bamg_handle* h, double* h_rho) {
    if (!h || !h->impl) return BAMG_EINVAL;
    if (h_rho) *h_rho = h->impl->rho_measured;
    return h->impl->interp_used;
}

int bamg_interp_dataset(const bamg_csr* A, int r, int levels, const bamg_opts* opts, float* d_feat, float* d_target,
                        int64_t cap_rows, int64_t* h_rows) {
    return guarded([&] {
        BAMG_REQUIRE(A && h_rows && cap_rows >= 0 && (cap_rows == 0 || (d_feat && d_target)), BAMG_EINVAL,
                     "bad interp_dataset arguments");
        bamg_opts o;
        if (opts) o = *opts;
        else bamg_default_opts(&o);
        o.interp = BAMG_INTERP_LS;
        check_setup_args(A, r, levels, o);
        auto sv = make_solver(A, r, levels, o, true, d_feat, d_target, cap_rows);
        *h_rows = sv->rec_rows;
        BAMG_CK(cudaStreamSynchronize((cudaStream_t)o.stream));
        BAMG_REQUIRE(*h_rows <= cap_rows, BAMG_ESIZE, "interp_dataset: cap_rows too small");
    });
}

int bamg_vcycle_apply(bamg_handle* h, const double* v, double* z) {
    return guarded([&] {
        BAMG_REQUIRE(h && h->impl && v && z, BAMG_EINVAL, "null argument");
        h->impl->vcycle_apply(v, z);
        BAMG_CK(cudaStreamSynchronize(h->impl->s));
    });
}

}  // extern "C"
