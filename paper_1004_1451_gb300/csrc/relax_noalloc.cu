// Allocation-free variant of the omega-Jacobi relaxation entry point.
//
// Some callers cannot let a library allocate device memory: services that reserve a
// fixed device-memory budget at start-up and refuse any later cudaMalloc, frameworks
// whose caching allocator owns the whole device and must not be bypassed, and
// latency-critical loops where cudaMalloc or cudaFree would block on the device.  For
// them bamg_relax_noalloc keeps its working memory (the second copy of the vector block
// used by the out-of-place sweeps, and the diagonals of B and T) in one file-scope
// device array instead of allocating it per call.
#include <mutex>

#include "kernels.cuh"

namespace bamg {

// Size of the shared scratch array.  Every GPU that loads the library holds it until
// the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device memory, so the
// device address is looked up once per device (with that device current) and cached.
static void* noalloc_scratch(int dev) {
    static std::mutex mu;
    static void* addr[256] = {};
    BAMG_REQUIRE(dev >= 0 && dev < 256, BAMG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        BAMG_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = p;
    }
    return addr[dev];
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
static void relax_noalloc(const bamg_mat* Bm, const void* T_val, const double* lam, int ncols, int ld, int col0,
                          double omega, int nu, void* X, cudaStream_t s) {
    constexpr int W = V16<T>::W;
    BAMG_REQUIRE(Bm && Bm->n >= 1 && Bm->nnz >= 0 && Bm->row_ptr && Bm->col && Bm->val, BAMG_EINVAL, "bad matrix");
    BAMG_REQUIRE(X != nullptr && ((uintptr_t)X & 15) == 0, BAMG_EINVAL, "vector block must be 16-byte aligned");
    BAMG_REQUIRE(col0 >= 0 && ld >= W, BAMG_EINVAL, "col0 must be >= 0 and ld at least one 16-byte chunk");
    BAMG_REQUIRE(ld % W == 0 && col0 % W == 0, BAMG_EINVAL, "ld and col0 must be multiples of 2 (FP64) or 4 (FP32)");
    BAMG_REQUIRE(ncols >= 1 && col0 + (ncols + W - 1) / W * W <= ld, BAMG_EINVAL, "columns exceed the leading dimension");
    BAMG_REQUIRE(nu >= 0, BAMG_EINVAL, "nu must be >= 0");
    const size_t n = (size_t)Bm->n;
    const size_t work_b = align256(n * (size_t)ld * sizeof(T));
    const size_t vec_b = align256(n * sizeof(T));
    const size_t need = work_b + 3 * vec_b;
    BAMG_REQUIRE(need <= NOALLOC_SCRATCH_BYTES, BAMG_EINVAL,
                 "bamg_relax_noalloc: n * (ld + 3) elements exceed its 8 MiB scratch; use bamg_relax");
    int dev = 0;
    BAMG_CK(cudaGetDevice(&dev));
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(dev));
    T* work = reinterpret_cast<T*>(base);
    T* dB = reinterpret_cast<T*>(base + work_b);
    T* dinv = reinterpret_cast<T*>(base + work_b + vec_b);
    T* dT = reinterpret_cast<T*>(base + work_b + 2 * vec_b);
    // every scratch word read below is written first in the same call: no clearing needed
    MatView<T> B{Bm->n, Bm->nnz, Bm->row_ptr, Bm->col, (const T*)Bm->val};
    launch_diag<T>(B, dB, s);
    launch_reciprocal<T>(B.n, dB, dinv, s);
    if (T_val) launch_diag_vals<T>(B.n, B.rp, B.ci, (const T*)T_val, dT, s);
    relax<T>(B, (const T*)T_val, dB, dinv, T_val ? dT : nullptr, lam, ncols, ld, col0, (T)omega, nu, (T*)X, work, s,
             false);
    BAMG_CK(cudaStreamSynchronize(s));
}

}  // namespace bamg

extern "C" int bamg_relax_noalloc(int dtype, const bamg_mat* B, const void* T_val, const double* d_lambda, int ncols,
                                  int ld, int col0, double omega, int nu, void* X, void* stream) {
    using namespace bamg;
    try {
        if (dtype == BAMG_F64)
            relax_noalloc<double>(B, T_val, d_lambda, ncols, ld, col0, omega, nu, X, (cudaStream_t)stream);
        else if (dtype == BAMG_F32)
            relax_noalloc<float>(B, T_val, d_lambda, ncols, ld, col0, omega, nu, X, (cudaStream_t)stream);
        else
            throw Error(BAMG_EINVAL, "bad dtype");
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
