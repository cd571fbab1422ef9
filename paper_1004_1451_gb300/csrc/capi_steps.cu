// C ABI of the single setup steps (bamg.h, "Step entry points"): thin wrappers that
// validate the arguments and run the same launchers the hierarchy uses.
#include <cstring>
#include <memory>

#include "kernels.cuh"

using namespace bamg;

namespace bamg {
template <typename F>
static int guard(F&& f) {
    try {
        f();
        set_last_error("");
        return BAMG_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return BAMG_EINVAL;
    }
}

template <typename T>
static MatView<T> view(const bamg_mat* B) {
    BAMG_REQUIRE(B && B->n >= 1 && B->nnz >= 0 && B->row_ptr && B->col && B->val, BAMG_EINVAL, "bad matrix");
    return MatView<T>{B->n, B->nnz, B->row_ptr, B->col, (const T*)B->val};
}

template <typename T>
static void check_block(const void* X, int ncols, int ld, int col0) {
    constexpr int W = V16<T>::W;
    BAMG_REQUIRE(X != nullptr, BAMG_EINVAL, "null vector block");
    BAMG_REQUIRE(((uintptr_t)X & 15) == 0, BAMG_EINVAL, "vector block must be 16-byte aligned");
    BAMG_REQUIRE(col0 >= 0 && ld >= W, BAMG_EINVAL, "col0 must be >= 0 and ld at least one 16-byte chunk");
    BAMG_REQUIRE(ld % W == 0 && col0 % W == 0, BAMG_EINVAL, "ld and col0 must be multiples of 2 (FP64) or 4 (FP32)");
    BAMG_REQUIRE(ncols >= 1 && col0 + (ncols + W - 1) / W * W <= ld, BAMG_EINVAL, "columns exceed the leading dimension");
}

template <typename T>
static void relax_step(const bamg_mat* Bm, const void* T_val, const double* lam, int ncols, int ld, int col0,
                       double omega, int nu, void* X, void* work, cudaStream_t s) {
    MatView<T> B = view<T>(Bm);
    check_block<T>(X, ncols, ld, col0);
    BAMG_REQUIRE(work && ((uintptr_t)work & 15) == 0, BAMG_EINVAL, "work must be 16-byte aligned");
    TmpBuf<T> dB(B.n, s), dT(B.n, s), dinv(B.n, s);
    launch_diag<T>(B, dB.get(), s);
    launch_reciprocal<T>(B.n, dB.get(), dinv.get(), s);
    if (T_val) launch_diag_vals<T>(B.n, B.rp, B.ci, (const T*)T_val, dT.get(), s);
    relax<T>(B, (const T*)T_val, dB.get(), dinv.get(), T_val ? dT.get() : nullptr, lam, ncols, ld, col0, (T)omega, nu,
             (T*)X, (T*)work, s);
    BAMG_CK(cudaStreamSynchronize(s));
}
}  // namespace bamg

extern "C" {

int bamg_tv_init(int dtype, int n, int ncols, int ld, int col0, uint64_t seed, double lo, double hi, void* X,
                 void* stream) {
    return guard([&] {
        cudaStream_t s = (cudaStream_t)stream;
        BAMG_REQUIRE(n >= 0 && ncols >= 0 && (X || n == 0) && col0 >= 0 && col0 + ncols <= ld, BAMG_EINVAL,
                     "bad tv_init args");
        if (dtype == BAMG_F64) launch_tv_init<double>(n, ncols, ld, col0, seed, lo, hi, (double*)X, s);
        else if (dtype == BAMG_F32) launch_tv_init<float>(n, ncols, ld, col0, seed, lo, hi, (float*)X, s);
        else throw Error(BAMG_EINVAL, "bad dtype");
        BAMG_CK(cudaStreamSynchronize(s));
    });
}

int bamg_relax(int dtype, const bamg_mat* B, const void* T_val, const double* d_lambda, int ncols, int ld, int col0,
               double omega, int nu, void* X, void* work, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(nu >= 0, BAMG_EINVAL, "nu must be >= 0");
        if (dtype == BAMG_F64) relax_step<double>(B, T_val, d_lambda, ncols, ld, col0, omega, nu, X, work, (cudaStream_t)stream);
        else if (dtype == BAMG_F32) relax_step<float>(B, T_val, d_lambda, ncols, ld, col0, omega, nu, X, work, (cudaStream_t)stream);
        else throw Error(BAMG_EINVAL, "bad dtype");
    });
}

int bamg_autotune_report(int32_t* h_rows, int max_rows) {
    if (!h_rows || max_rows < 0) return BAMG_EINVAL;
    return jacobi_tuned_shapes(h_rows, max_rows);
}

int bamg_tv_weights(int dtype, const bamg_mat* B, int ncols, int ld, int col0, const uint8_t* d_active, double floor,
                    void* X, double* d_w, void* stream) {
    return guard([&] {
        cudaStream_t s = (cudaStream_t)stream;
        BAMG_REQUIRE(d_w && ncols <= 32, BAMG_EINVAL, "bad weights args");
        if (dtype == BAMG_F64) {
            check_block<double>(X, ncols, ld, col0);
            tv_weights<double>(view<double>(B), ncols, ld, col0, d_active, floor, (double*)X, d_w, s);
        } else if (dtype == BAMG_F32) {
            check_block<float>(X, ncols, ld, col0);
            tv_weights<float>(view<float>(B), ncols, ld, col0, d_active, floor, (float*)X, d_w, s);
        } else
            throw Error(BAMG_EINVAL, "bad dtype");
        BAMG_CK(cudaStreamSynchronize(s));
    });
}

int bamg_coarsen_grid(int nx, int ny, uint8_t* cf, int32_t* cidx, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(nx >= 1 && ny >= 1 && cf && cidx, BAMG_EINVAL, "bad coarsen_grid args");
        coarsen_grid(nx, ny, cf, cidx, (cudaStream_t)stream);
        BAMG_CK(cudaStreamSynchronize((cudaStream_t)stream));
    });
}

int bamg_coarsen_cr(const bamg_mat* B, int level, uint64_t seed, double theta, int nu, double omega, int max_rounds,
                    uint8_t* cf, int32_t* cidx, int* h_nc, int* h_rounds, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(cf && cidx && nu >= 1 && max_rounds >= 0 && level >= 0 && level < 256, BAMG_EINVAL,
                     "bad coarsen_cr args");
        int nc = 0;
        const int rounds = coarsen_cr<double>(view<double>(B), level, seed, theta, nu, omega, max_rounds, cf, cidx, &nc,
                                              (cudaStream_t)stream);
        if (h_nc) *h_nc = nc;
        if (h_rounds) *h_rounds = rounds;
    });
}

int bamg_interp_ls(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols,
                   int ld, const double* d_w, int z, int mmax, int c, double ridge, int32_t* pcol, void* pval,
                   int32_t* pcnt, void* stream) {
    return guard([&] {
        cudaStream_t s = (cudaStream_t)stream;
        BAMG_REQUIRE(B && cf && cidx && X && d_w && pcol && pval && pcnt && ncols <= ld, BAMG_EINVAL,
                     "bad interp_ls args");
        int e;
        if (dtype == BAMG_F64)
            e = interp_ls<double>(B->n, B->row_ptr, B->col, (const double*)B->val, cf, cidx, (const double*)X, ncols,
                                  ld, d_w, z, mmax, c,
                                  ridge, pcol, (double*)pval, pcnt, s);
        else if (dtype == BAMG_F32)
            e = interp_ls<float>(B->n, B->row_ptr, B->col, (const float*)B->val, cf, cidx, (const float*)X, ncols, ld,
                                 d_w, z, mmax, c,
                                 ridge, pcol, (float*)pval, pcnt, s);
        else
            throw Error(BAMG_EINVAL, "bad dtype");
        BAMG_REQUIRE(e == 0, BAMG_EOVERFLOW, "neighbourhood search: a fine point needs more than 2048 recorded states");
    });
}

}  // extern "C"

namespace bamg {
template <typename T>
static void galerkin_step(const bamg_mat* Bm, const void* T_val, int nc, const int32_t* pcol, const void* pval,
                          const int32_t* pcnt, int c, int32_t* out_rp, int32_t* out_ci, void* out_bv, void* out_tv,
                          int64_t cap, int64_t* h_nnz, cudaStream_t s) {
    MatView<T> B = view<T>(Bm);
    EllView<T> P{B.n, c, pcol, (const T*)pval, pcnt};
    cudaStream_t prev = alloc_stream();
    alloc_stream() = s;
    struct Restore {
        cudaStream_t p;
        ~Restore() { alloc_stream() = p; }
    } restore_{prev};
    DevBuf<int32_t> qrp, qci;
    DevBuf<T> qv;
    build_restriction<T>(P, nc, qrp, qci, qv, s);
    GalerkinOut<T> go;
    galerkin<T>(B, (const T*)T_val, qrp.get(), qci.get(), qv.get(), P, nc, go, s);
    if (h_nnz) *h_nnz = go.nnz;
    if (cap < go.nnz) throw Error(BAMG_ESIZE, "galerkin: output capacity too small");
    BAMG_REQUIRE(out_rp && out_ci && out_bv, BAMG_EINVAL, "null output");
    BAMG_CK(cudaMemcpyAsync(out_rp, go.rp.get(), sizeof(int32_t) * (nc + 1), cudaMemcpyDeviceToDevice, s));
    BAMG_CK(cudaMemcpyAsync(out_ci, go.ci.get(), sizeof(int32_t) * go.nnz, cudaMemcpyDeviceToDevice, s));
    BAMG_CK(cudaMemcpyAsync(out_bv, go.bv.get(), sizeof(T) * go.nnz, cudaMemcpyDeviceToDevice, s));
    if (out_tv) BAMG_CK(cudaMemcpyAsync(out_tv, go.tv.get(), sizeof(T) * go.nnz, cudaMemcpyDeviceToDevice, s));
    BAMG_CK(cudaStreamSynchronize(s));
}
}  // namespace bamg

namespace bamg {
template <typename T>
static void features_step(const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols, int ld,
                          const double* d_w, int z, int mmax, int c, double ridge, float* d_feat, float* d_target,
                          int32_t* d_cand, cudaStream_t s) {
    AllocStream as_(s);
    const MatView<T> Bv = view<T>(B);
    TmpBuf<int32_t> pcol((size_t)Bv.n * c, s), pcnt(Bv.n, s);
    TmpBuf<T> pval((size_t)Bv.n * c, s);
    LsOut ex;
    ex.feat = d_feat;
    ex.target = d_target;
    ex.cand = d_cand;
    ex.greedy = d_target != nullptr;
    const int e = interp_ls<T>(Bv.n, Bv.rp, Bv.ci, Bv.v, cf, cidx, (const T*)X, ncols, ld, d_w, z, mmax, c, ridge,
                               pcol.get(), pval.get(), pcnt.get(), s, nullptr, ex);
    BAMG_REQUIRE(e == 0, BAMG_EOVERFLOW, "neighbourhood search: a fine point needs more than 2048 recorded states");
    BAMG_CK(cudaStreamSynchronize(s));
}

template <typename T>
static void learned_step(const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols, int ld,
                         const double* d_w, int z, int mmax, int c, double ridge, const bamg_model* m, int refit,
                         int32_t* pcol, void* pval, int32_t* pcnt, cudaStream_t s) {
    AllocStream as_(s);
    const MatView<T> Bv = view<T>(B);
    TmpBuf<int> err(1, s);
    BAMG_CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    interp_learned<T>(Bv.n, Bv.rp, Bv.ci, Bv.v, cf, cidx, (const T*)X, ncols, ld, d_w, z, mmax, c, ridge, m->impl,
                      refit != 0, pcol, (T*)pval, pcnt, s, err.get());
    int h = 0;
    BAMG_CK(cudaMemcpyAsync(&h, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CK(cudaStreamSynchronize(s));
    BAMG_REQUIRE(h == 0, BAMG_EOVERFLOW, "neighbourhood search: a fine point needs more than 2048 recorded states");
}

}  // namespace bamg

extern "C" {

int bamg_galerkin(int dtype, const bamg_mat* B, const void* T_val, int nc, const int32_t* pcol, const void* pval,
                  const int32_t* pcnt, int c, int32_t* out_row_ptr, int32_t* out_col, void* out_bv, void* out_tv,
                  int64_t cap, int64_t* h_nnz, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(nc >= 1 && c >= 1 && c <= 4 && pcol && pval && pcnt, BAMG_EINVAL, "bad galerkin args");
        if (dtype == BAMG_F64)
            galerkin_step<double>(B, T_val, nc, pcol, pval, pcnt, c, out_row_ptr, out_col, out_bv, out_tv, cap, h_nnz,
                                  (cudaStream_t)stream);
        else if (dtype == BAMG_F32)
            galerkin_step<float>(B, T_val, nc, pcol, pval, pcnt, c, out_row_ptr, out_col, out_bv, out_tv, cap, h_nnz,
                                 (cudaStream_t)stream);
        else
            throw Error(BAMG_EINVAL, "bad dtype");
    });
}

int bamg_coarse_eig(int dtype, int n, const double* d_B, const double* d_T, int k_ev, double* d_lam, double* d_V,
                    int32_t* d_kind, int* h_nvec, double* d_pinv, void* stream) {
    return guard([&] {
        cudaStream_t s = (cudaStream_t)stream;
        BAMG_REQUIRE(d_B && d_T && d_lam && d_V && d_kind, BAMG_EINVAL, "bad coarse_eig args");
        BAMG_REQUIRE(dtype == BAMG_F64 || dtype == BAMG_F32, BAMG_EINVAL, "bad dtype");
        const int nv = coarse_eig(n, d_B, d_T, k_ev, d_lam, d_V, d_kind, dtype == BAMG_F32, s);
        BAMG_REQUIRE(nv > 0, BAMG_ENUMERIC, "coarsest eigensolve did not converge");
        if (h_nvec) *h_nvec = nv;
        if (d_pinv)
            BAMG_REQUIRE(coarse_pinv(n, d_B, d_pinv, dtype == BAMG_F32, s) == 0, BAMG_ENUMERIC,
                         "singular coarsest factor");
        BAMG_CK(cudaStreamSynchronize(s));
    });
}


int bamg_interp_features(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols,
                         int ld, const double* d_w, int z, int mmax, int c, double ridge, float* d_feat,
                         float* d_target, int32_t* d_cand, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(B && cf && cidx && X && d_w && ncols <= ld && mmax <= 16, BAMG_EINVAL, "bad interp_features args");
        if (dtype == BAMG_F64)
            features_step<double>(B, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, d_feat, d_target, d_cand,
                                  (cudaStream_t)stream);
        else if (dtype == BAMG_F32)
            features_step<float>(B, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, d_feat, d_target, d_cand,
                                 (cudaStream_t)stream);
        else
            throw Error(BAMG_EINVAL, "bad dtype");
    });
}

int bamg_interp_learned(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols,
                        int ld, const double* d_w, int z, int mmax, int c, double ridge, const bamg_model* m, int refit,
                        int32_t* pcol, void* pval, int32_t* pcnt, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(B && cf && cidx && X && d_w && m && m->impl && pcol && pval && pcnt && ncols <= ld,
                     BAMG_EINVAL, "bad interp_learned args");
        if (dtype == BAMG_F64)
            learned_step<double>(B, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, m, refit, pcol, pval, pcnt,
                                 (cudaStream_t)stream);
        else if (dtype == BAMG_F32)
            learned_step<float>(B, cf, cidx, X, ncols, ld, d_w, z, mmax, c, ridge, m, refit, pcol, pval, pcnt,
                                (cudaStream_t)stream);
        else
            throw Error(BAMG_EINVAL, "bad dtype");
    });
}

// ------------------------------------------------------------------ the model
int bamg_model_create(uint64_t seed, bamg_model** m) {
    return guard([&] {
        BAMG_REQUIRE(m, BAMG_EINVAL, "null model pointer");
        *m = nullptr;
        auto h = std::make_unique<bamg_model>();
        h->impl = mlp_create(seed, nullptr);
        BAMG_CK(cudaStreamSynchronize(nullptr));
        *m = h.release();
    });
}

void bamg_model_free(bamg_model* m) {
    if (!m) return;
    mlp_destroy(m->impl);
    delete m;
}

int64_t bamg_model_param_count(void) { return mlp_param_count(); }

int bamg_model_set(bamg_model* m, const float* h_params, int64_t count) {
    return guard([&] {
        BAMG_REQUIRE(m && m->impl && h_params && count == mlp_param_count(), BAMG_EINVAL, "bad model_set args");
        mlp_set(m->impl, h_params, nullptr);
        BAMG_CK(cudaStreamSynchronize(nullptr));
    });
}

int bamg_model_get(const bamg_model* m, float* h_params, int64_t count) {
    return guard([&] {
        BAMG_REQUIRE(m && m->impl && h_params && count == mlp_param_count(), BAMG_EINVAL, "bad model_get args");
        mlp_get(m->impl, h_params, nullptr);
    });
}

int bamg_model_forward(const bamg_model* m, const float* d_feat, int64_t rows, float* d_out, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(m && m->impl && rows >= 0 && (rows == 0 || (d_feat && d_out)), BAMG_EINVAL,
                     "bad model_forward args");
        mlp_forward(m->impl, rows, d_feat, d_out, (cudaStream_t)stream);
    });
}

int bamg_model_gradients(bamg_model* m, const float* d_feat, const float* d_target, int64_t rows, float* h_grad,
                         double* h_loss, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(m && m->impl && rows > 0 && d_feat && d_target, BAMG_EINVAL, "bad model_gradients args");
        const double l = mlp_gradients(m->impl, rows, d_feat, d_target, h_grad, (cudaStream_t)stream);
        if (h_loss) *h_loss = l;
    });
}

int bamg_model_train(bamg_model* m, const float* d_feat, const float* d_target, int64_t rows, int epochs, int batch,
                     double lr, double* h_epoch_loss, void* stream) {
    return guard([&] {
        BAMG_REQUIRE(m && m->impl && rows > 0 && d_feat && d_target && epochs >= 0 && batch > 0 && lr > 0.0,
                     BAMG_EINVAL, "bad model_train args");
        mlp_train(m->impl, rows, d_feat, d_target, epochs, batch, lr, h_epoch_loss, (cudaStream_t)stream);
    });
}

}  // extern "C"
