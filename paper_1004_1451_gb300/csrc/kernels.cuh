// Host launchers of the device kernels (one translation unit per family).
#pragma once

#include "common.cuh"

namespace bamg {

template <typename T>
struct MatView {
    int n = 0, nnz = 0;
    const int32_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const T* v = nullptr;
};

// Interpolation in ELL form: row i has pcnt[i] <= c entries (pcol[i*c+t], pval[i*c+t]).
template <typename T>
struct EllView {
    int n = 0, c = 0;
    const int32_t* pcol = nullptr;
    const T* pval = nullptr;
    const int32_t* pcnt = nullptr;
};

// Lanes per row for sparse row walks on a matrix with nnz entries in n rows: 1 (one thread
// per row) below 12 entries per row on average, then 4, 8, 16 or 32.
inline int lanes_per_row(int n, int64_t nnz) {
    const double avg = n > 0 ? (double)nnz / n : 0.0;
    return avg < 12.0 ? 1 : avg < 24.0 ? 4 : avg < 48.0 ? 8 : avg < 96.0 ? 16 : 32;
}

// ------------------------------------------------------------------ k_relax.cu
template <typename T>
void launch_tv_init(int n, int ncols, int ld, int col0, uint64_t seed, double lo, double hi, T* X, cudaStream_t s);
template <typename T>
void launch_diag(const MatView<T>& M, T* d, cudaStream_t s);
template <typename T>
void launch_diag_vals(int n, const int32_t* rp, const int32_t* ci, const T* vals, T* d, cudaStream_t s);
template <typename T>
void launch_reciprocal(int n, const T* d, T* dinv, cudaStream_t s);
// dB = diag(B), dT = diag(T) (skipped when tv is null), dinv = 1 / dB, one launch
template <typename T>
void launch_diagonals(int n, const int32_t* rp, const int32_t* ci, const T* bv, const T* tv, T* dB, T* dT, T* dinv,
                      cudaStream_t s);
template <typename T>
void launch_identity_on_pattern(int n, const int32_t* rp, const int32_t* ci, T* tv, cudaStream_t s);
// nu sweeps; T_val/dT/d_lambda may be null (no shift).  work: n*ld scratch.  tune: on large
// levels, time the launch shapes once per shape key (jacobi_tuned_shapes lists the choices).
template <typename T>
void relax(const MatView<T>& B, const T* T_val, const T* dB, const T* dinvB, const T* dT, const double* d_lambda,
           int ncols, int ld, int col0, T omega, int nu, T* X, T* work, cudaStream_t s, bool tune = true);
// Rows (precision bytes, shift, entry batch, 16-byte chunks per row, log2 n, chunks per
// thread, blocks per SM) of the tuned sweep shapes, at most max_rows; returns the count.
int jacobi_tuned_shapes(int* out, int max_rows);
// Normalise active columns and write LS weights (ncols doubles).
template <typename T>
void tv_weights(const MatView<T>& B, int ncols, int ld, int col0, const uint8_t* d_active, double floor, T* X,
                double* d_w, cudaStream_t s);
// Rayleigh quotients lambda_k = <Bx,x>/<Tx,x> (k >= 1; lambda_0 = 0), selection flags.
template <typename T>
void rayleigh_update(const MatView<T>& B, const T* T_val, const T* X, int ncols, int ld, int col0, double tol,
                     double* d_lam, uint8_t* d_sel, cudaStream_t s);
template <typename T>
void inject_cols(int nc, const int32_t* c2f, const T* X, T* Xc, int ld, int col0, int ncols, cudaStream_t s);
template <typename T>
void prolong_cols(const EllView<T>& P, const T* Xc, T* X, int ld, int col0, int ncols, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_convert(int64_t n, const Tin* a, Tout* b, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_strided_to_vec(int n, const Tin* X, int ld, int col, Tout* y, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_vecs_to_strided(int n, int nv, const Tin* y, Tout* X, int ld, int col0, cudaStream_t s);

// Build B = I - A (diagonal always stored) from A (sorted CSR); checks column sums,
// signs and a_ii < 1.  Returns the status flags (bit 0: negative entry, bit 1: colsum,
// bit 2: a_ii = 1, bit 3: unsorted/out-of-range column).
int build_system_matrix(int n, int nnzA, const int32_t* rpA, const int32_t* ciA, const double* vA,
                        DevBuf<int32_t>& rpB, DevBuf<int32_t>& ciB, DevBuf<double>& vB, cudaStream_t s);

// ------------------------------------------------------------------ learned interpolation
constexpr int MLP_S = 16;       // candidate slots (m_max)
constexpr int MLP_NF_SLOT = 6;  // features per slot
constexpr int MLP_F = 112;      // features per point: 16 x 6 + 2, zero-padded
constexpr int MLP_H = 128;      // hidden width
struct Model;                   // the MLP (k_mlp.cu)
Model* mlp_create(uint64_t seed, cudaStream_t s);
void mlp_destroy(Model* m);
int64_t mlp_param_count();
void mlp_set(Model* m, const float* h_params, cudaStream_t s);
void mlp_get(const Model* m, float* h_params, cudaStream_t s);
void mlp_forward(const Model* m, int64_t rows, const float* feat, float* Y, cudaStream_t s);
double mlp_gradients(Model* m, int64_t rows, const float* feat, const float* target, float* h_grad, cudaStream_t s);
void mlp_train(Model* m, int64_t rows, const float* feat, const float* target, int epochs, int batch, double lr,
               double* h_loss, cudaStream_t s);
// Optional outputs of the LS kernel: per point MLP_F features, the LS row on the MLP_S
// slots, the candidate of each slot (-1 padded); greedy = false skips Algorithm 2.
struct LsOut {
    float* feat = nullptr;
    float* target = nullptr;
    int32_t* cand = nullptr;
    bool greedy = true;
};

// ------------------------------------------------------------------ k_interp.cu
void coarsen_grid(int nx, int ny, uint8_t* cf, int32_t* cidx, cudaStream_t s);
void coarse_to_fine(int n, const uint8_t* cf, const int32_t* cidx, int32_t* c2f, cudaStream_t s);
// Returns an error flag (BAMG_EOVERFLOW if a neighbourhood search overflowed).
template <typename T>
int interp_ls(int n, const int32_t* rp, const int32_t* ci, const T* bv, const uint8_t* cf, const int32_t* cidx,
              const T* X, int ncols, int ld, const double* d_w, int z, int mmax, int c, double ridge, int32_t* pcol,
              T* pval, int32_t* pcnt, cudaStream_t s, int* d_err = nullptr, const LsOut& ex = LsOut());
// Learned interpolation of one level: candidates and features (the LS kernel's search),
// the MLP, then per fine point the c slots of largest |y| with weights y or, with refit,
// the Eq. (3.6) minimiser over them.  Coarse rows are unit rows.
template <typename T>
int interp_learned(int n, const int32_t* rp, const int32_t* ci, const T* bv, const uint8_t* cf, const int32_t* cidx,
                   const T* X, int ncols, int ld, const double* d_w, int z, int mmax, int c, double ridge,
                   const Model* model, bool refit, int32_t* pcol, T* pval, int32_t* pcnt, cudaStream_t s,
                   int* d_err = nullptr);
// Q rows (CSR by coarse rows, sorted by fine index) from the ELL interpolation.
template <typename T>
void build_restriction(const EllView<T>& P, int nc, DevBuf<int32_t>& qrp, DevBuf<int32_t>& qci, DevBuf<T>& qv,
                       cudaStream_t s);
// Galerkin: outputs allocated by the callback once nnz is known.
template <typename T>
struct GalerkinOut {
    DevBuf<int32_t> rp, ci;
    DevBuf<T> bv, tv;
    int nnz = 0;  // -1 while the count is on its way to the host (galerkin with defer)
};
// With defer (taken while the bound's arrays stay within 64 MB) the coarse arrays get room for
// the product count's bound and the compaction is queued without waiting for the entry count;
// galerkin_nnz(out, s) then waits for it (no other count may be read on this host thread in
// between).
template <typename T>
void galerkin(const MatView<T>& B, const T* T_val, const int32_t* qrp, const int32_t* qci, const T* qv,
              const EllView<T>& P, int nc, GalerkinOut<T>& out, cudaStream_t s, bool defer = false);
template <typename T>
void galerkin_nnz(GalerkinOut<T>& out, cudaStream_t s);
template <typename T>
void csr_to_dense(int n, const int32_t* rp, const int32_t* ci, const T* v, double* D, cudaStream_t s);

// ------------------------------------------------------------------ k_cr.cu
// Compatible relaxation coarsening (Algorithm 1).  Returns the number of rounds.
template <typename T>
int coarsen_cr(const MatView<T>& B, int level, uint64_t seed, double theta, int nu, double omega, int max_rounds,
               uint8_t* cf, int32_t* cidx, int* nc_out, cudaStream_t s);

// ------------------------------------------------------------------ k_coarse.cu
// Eigenpairs of B x = lambda T x (dense FP64 input, n <= 64); the eigenvectors are
// refined in FP32 when fp32_vectors is set, else in FP64.  Returns the number of vector
// columns written (<= k_ev + 1) or a negative status.
int coarse_eig(int n, const double* dB, const double* dT, int k_ev, double* d_lam, double* d_V, int32_t* d_kind,
               bool fp32_vectors, cudaStream_t s);
// Minimal-norm inverse of the rank n-1 matrix B (dense FP64 in and out, row-major),
// computed in FP32 arithmetic when fp32 is set, else in FP64.
// with d_fail: a failed factorisation sets bit 2 of *d_fail and the call returns 0 without
// waiting for the device; else it returns BAMG_ENUMERIC after reading the blocks' status
int coarse_pinv(int n, const double* dB, double* dP, bool fp32, cudaStream_t s, int* d_fail = nullptr);

// Colour classes of the multicolour Gauss-Seidel smoother for the pattern (n, rp, ci):
// repeated independent sets of the uncoloured states; rows sorted by (colour, state), host
// offsets ptr[0..ncolours].
void colour_classes(int n, int nnz, const int32_t* rp, const int32_t* ci, int level, uint64_t seed,
                    std::vector<int>& ptr, DevBuf<int32_t>& rows, cudaStream_t s);

// ------------------------------------------------------------------ k_solve.cu
template <typename T>
struct VLevel {  // one level of the V-cycle
    MatView<T> B;
    const T* dinv = nullptr;
    EllView<T> P;                  // to the next coarser level
    const int32_t* qrp = nullptr;  // Q by coarse rows
    const int32_t* qci = nullptr;
    const T* qv = nullptr;
    int qnnz = 0;                  // entries of Q
    T *b = nullptr, *x = nullptr, *r = nullptr;  // work vectors of n entries
    // multicolour Gauss-Seidel smoother (gs_ncol > 0): rows sorted by colour (device) and
    // the colour offsets gs_ptr[0..gs_ncol] (host memory owned by the hierarchy)
    const int32_t* gs_rows = nullptr;
    const int* gs_ptr = nullptr;
    int gs_ncol = 0;
    // read on lv[0] only: the form of the coarse end of the V-cycle, 0 = the levels from the
    // first one with at most 4096 rows on a thread-block cluster (where the device has
    // clusters), 1 = the levels from the first one with at most 1024 rows in one block
    int tail_form = 0;
};
// One V-cycle: lv[0].b -> lv[0].x.  With Z != null the result is also stored at
// Z + (*dj) * n_0.
// sweeps x <- x + omega D^{-1} (b - B x) on one level (y: work array of n); result in x.
template <typename T>
void smooth_sweeps(const VLevel<T>& v, const T* b, T* x, T* y, double omega, int sweeps, cudaStream_t s);
template <typename T>
void vcycle(const std::vector<VLevel<T>>& lv, const T* pinv, double omega, int nu_pre, int nu_post, cudaStream_t s,
            T* Z = nullptr, const int* dj = nullptr);

void spmv_f64(const MatView<double>& B, const double* x, double* y, double alpha, cudaStream_t s);  // y = alpha B x
void spmv_f64_from_f32(const MatView<double>& B, const float* x, double* y, cudaStream_t s);
// Column dots h[q] = sum_i V[q*ldv + i] w[i], q < nv (deterministic two-level reduction).
void dots(int n, const double* V, int64_t ldv, int nv, const double* w, double* d_h, double* d_partial,
          cudaStream_t s);
int dots_partial_blocks(int n);
int arn_tiles(int n);  // row tiles of the fused Arnoldi kernels
void update_minus(int n, const double* V, int64_t ldv, int nv, const double* d_h, double* w, cudaStream_t s);
template <typename TZ>
void form_x(int n, const double* x0, const TZ* Z, int64_t ldz, int nz, const double* d_y, double* x, cudaStream_t s,
            const int* dnz = nullptr);  // with dnz the column count is *dnz (device memory)
// sum |B x|, sum (B x)^2, sum |x|, sum x into d_out[4] (deterministic).
// FGMRES Arnoldi steps *dj .. (until the stop test of ctl) in one cooperative launch with
// grid-wide barriers (same iterates as the captured step); false, launching nothing, when
// the hierarchy or device does not qualify.  bar: 2 unsigned, err: 1 int (device).
template <typename T>
bool arnoldi_cycle_persistent(int n, const MatView<double>& B, double* V, T* Z, T* vin, int* dj, double* st, int m,
                              double* partial, const std::vector<VLevel<T>>& lv, const T* pinv, double omega,
                              int nu_pre, int nu_post, const double* ctl, unsigned* bar, int* err, cudaStream_t s);
// Section 4.3 (preconditioned Arnoldi): one step on C B with the index j in *dj (raw
// Hessenberg column into H, ld ldh), and the eigenvector of H_k for the eigenvalue closest
// to 0 (inverse iteration with shift 0; k <= PARN_MMAX).
constexpr int PARN_MMAX = 64;
template <typename T>
void parnoldi_step(int n, const MatView<double>& B, double* V, T* vin, T* zout, int* dj, double* st, int m,
                   double* H, int ldh, double* partial, const std::vector<VLevel<T>>& lv, const T* pinv, double omega,
                   int nu_pre, int nu_post, cudaStream_t s);
void ritz_closest_to_zero(const double* H, int ldh, int k, double* eta, cudaStream_t s);
// d_out[0..4] = sum |Bx|, sum (Bx)^2, sum |x|, sum x, sum x^2 (FP64, fixed order);
// d_partial: blocks_for(n, 256) * RESNORM_SUMS doubles
constexpr int RESNORM_SUMS = 5;
void residual_norms(const MatView<double>& B, const double* x, double* d_out, double* d_partial, cudaStream_t s);
void scale_vec(int n, double* x, const double* d_num, int num_idx, bool reciprocal, double* y, cudaStream_t s);
void gmres_init(double* d_state, int m, cudaStream_t s);
// One Arnoldi step of flexible GMRES whose index j lives in device memory (*dj), so the
// whole sequence can be captured once in a CUDA graph and replayed.  With cond == 0,
// h_est (pinned host memory) receives {residual estimate, h_{j+1,j}} after the step.
// With a WHILE conditional handle the step is the body of a device-side loop: its last
// kernel sets the handle to 0 once j + 1 >= ctl[2], h_{j+1,j} = 0, or
// estimate * ctl[0] <= ctl[1] (ctl in device memory: kappa, tol ||x||_1, last j + 1).
template <typename T>
void arnoldi_step_graphable(int n, const MatView<double>& B, double* V, T* Z, T* vin, T* zout, int* dj, double* st,
                            int m, double* partial, const std::vector<VLevel<T>>& lv, const T* pinv, double omega,
                            int nu_pre, int nu_post, double* h_est, const double* ctl,
                            cudaGraphConditionalHandle cond, cudaStream_t s);
void gmres_solve_y(double* d_state, int j, int m, cudaStream_t s, const int* dj = nullptr);  // with dj: j = *dj - 1

}  // namespace bamg

// The opaque model handle of the C ABI.
struct bamg_model {
    bamg::Model* impl = nullptr;
};
