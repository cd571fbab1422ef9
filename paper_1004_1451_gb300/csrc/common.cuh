// Shared host/device helpers of the GB300 Bootstrap AMG library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bamg.h"

namespace bamg {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void count_launch();
void count_launches(int64_t k);  // adds k (may be negative: graph capture bookkeeping)
void set_last_error(const std::string& msg);

#define BAMG_CK(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            throw ::bamg::Error(e_ == cudaErrorMemoryAllocation ? BAMG_ENOMEM : BAMG_ECUDA,        \
                                std::string(#call) + ": " + cudaGetErrorString(e_));               \
        }                                                                                          \
    } while (0)

#define BAMG_REQUIRE(cond, code, msg)                                                              \
    do {                                                                                           \
        if (!(cond)) throw ::bamg::Error((code), (msg));                                           \
    } while (0)

// Programmatic dependent launch: while pdl_enabled() is set (the default; BAMG_PDL=0 in
// the environment clears it) every launch lets the kernel start before its predecessor in
// the stream finishes.  Every kernel of the library calls pdl_begin() before its first
// access to memory written by earlier work: it waits until the predecessor grid has
// completed and its writes are visible, and signals that its own dependents may launch.
// Without the attribute both instructions return at once.
bool& pdl_enabled();
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}
struct PdlScope {
    bool prev;
    PdlScope() : prev(pdl_enabled()) { pdl_enabled() = true; }
    ~PdlScope() { pdl_enabled() = prev; }
};
#define BAMG_LAUNCH_PDL(kernel, grid, block, smem, strm_, ...)                                      \
    do {                                                                                           \
        if (::bamg::pdl_enabled()) {                                                               \
            cudaLaunchConfig_t cfg_ = {};                                                          \
            cfg_.gridDim = dim3(grid);                                                             \
            cfg_.blockDim = dim3(block);                                                           \
            cfg_.dynamicSmemBytes = (smem);                                                        \
            cfg_.stream = (strm_);                                                                  \
            cudaLaunchAttribute at_[1];                                                            \
            at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                        \
            at_[0].val.programmaticStreamSerializationAllowed = 1;                                 \
            cfg_.attrs = at_;                                                                      \
            cfg_.numAttrs = 1;                                                                     \
            BAMG_CK(cudaLaunchKernelEx(&cfg_, kernel, __VA_ARGS__));                               \
        } else {                                                                                   \
            kernel<<<(grid), (block), (smem), (strm_)>>>(__VA_ARGS__);                              \
        }                                                                                          \
        ::bamg::count_launch();                                                                    \
        BAMG_CK(cudaGetLastError());                                                               \
    } while (0)
// Every kernel of the library goes through this macro so the process-wide launch
// counter is exact.
#define BAMG_LAUNCH(kernel, grid, block, smem, stream, ...) \
    BAMG_LAUNCH_PDL(kernel, grid, block, smem, stream, __VA_ARGS__)

inline unsigned blocks_for(int64_t work, int per_block) {
    int64_t b = (work + per_block - 1) / per_block;
    return (unsigned)(b < 1 ? 1 : b);
}

// Stream on which DevBuf allocations are ordered (set by the owner of the work: the
// handle's stream during setup and solve).  Thread-local.
cudaStream_t& alloc_stream();
// Sets alloc_stream() for a scope.
struct AllocStream {
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocStream() { alloc_stream() = prev; }
};

// Owning device buffer from the stream-ordered pool (cudaMallocAsync on alloc_stream()),
// so building a hierarchy does not synchronise the device for every allocation.
// Callers synchronise their streams before the owner is destroyed.
template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    explicit DevBuf(size_t n_) { alloc(n_); }
    void alloc(size_t n_) {
        release();
        s = alloc_stream();
        if (n_) BAMG_CK(cudaMallocAsync((void**)&p, n_ * sizeof(T), s));
        n = n_;
    }
    void ensure(size_t n_) {
        if (n_ > n) alloc(n_);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        release();
        p = o.p;
        n = o.n;
        s = o.s;
        o.p = nullptr;
        o.n = 0;
        return *this;
    }
    T* get() const { return p; }
};

// Stack allocator for the temporaries of one stream: chunks from the stream-ordered pool,
// handed out in 256-byte aligned slices and taken back when the slices are released (any
// order; space is reclaimed from the top).  A slice released here can be handed out again
// at once: its next user is ordered after its last one on the same stream.  Spares the
// pool calls of the many short-lived buffers of a setup.
struct StackArena {
    struct Chunk {
        char* base;
        size_t cap, top;
    };
    struct Slice {
        int chunk;
        size_t prev;
        char* p;
        bool live;
    };
    cudaStream_t s;
    std::vector<Chunk> chunks;
    std::vector<Slice> stack;
    static constexpr size_t MIN_CHUNK = size_t(64) << 20;
    explicit StackArena(cudaStream_t st) : s(st) {}
    void* push(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        size_t c = stack.empty() ? 0 : (size_t)stack.back().chunk;
        while (c < chunks.size() && chunks[c].top + bytes > chunks[c].cap) ++c;
        if (c == chunks.size()) {
            Chunk k{nullptr, bytes > MIN_CHUNK ? bytes : MIN_CHUNK, 0};
            BAMG_CK(cudaMallocAsync((void**)&k.base, k.cap, s));
            chunks.push_back(k);
        }
        Chunk& k = chunks[c];
        stack.push_back(Slice{(int)c, k.top, k.base + k.top, true});
        k.top += bytes;
        return stack.back().p;
    }
    void pop(void* p) {
        for (size_t q = stack.size(); q-- > 0;)
            if (stack[q].p == p && stack[q].live) {
                stack[q].live = false;
                break;
            }
        while (!stack.empty() && !stack.back().live) {
            chunks[stack.back().chunk].top = stack.back().prev;
            stack.pop_back();
        }
    }
    // returns the chunks to the pool once no slice is live
    void release() {
        if (!stack.empty()) return;
        for (Chunk& k : chunks) cudaFreeAsync(k.base, s);
        chunks.clear();
    }
    ~StackArena() {
        stack.clear();
        release();
    }
    StackArena(const StackArena&) = delete;
    StackArena& operator=(const StackArena&) = delete;
};
// The arena that TmpBufs on its stream draw from (thread-local; null: the pool directly).
StackArena*& tmp_arena();
struct ArenaScope {  // sets tmp_arena() for a scope and releases the arena's chunks after
    StackArena* prev;
    StackArena& a;
    explicit ArenaScope(StackArena& a_) : prev(tmp_arena()), a(a_) { tmp_arena() = &a; }
    ~ArenaScope() {
        tmp_arena() = prev;
        a.release();
    }
};

// Stream-ordered temporary: a slice of the current StackArena when it serves this stream,
// else cudaMallocAsync / cudaFreeAsync.
template <typename T>
struct TmpBuf {
    T* p = nullptr;
    cudaStream_t s = nullptr;
    StackArena* a = nullptr;
    TmpBuf(size_t n, cudaStream_t st) : s(st) {
        if (!n) return;
        StackArena* cur = tmp_arena();
        if (cur && cur->s == st) {
            a = cur;
            p = static_cast<T*>(a->push(n * sizeof(T)));
        } else {
            BAMG_CK(cudaMallocAsync((void**)&p, n * sizeof(T), s));
        }
    }
    ~TmpBuf() {
        if (!p) return;
        if (a)
            a->pop(p);
        else
            cudaFreeAsync(p, s);
    }
    TmpBuf(const TmpBuf&) = delete;
    TmpBuf& operator=(const TmpBuf&) = delete;
    T* get() const { return p; }
};

// ------------------------------------------------------------------ device helpers
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state s + t * gamma, then the published
// 64-bit finaliser.  Draw number (stream * 2^40 + idx + 1) of `seed`.
__host__ __device__ __forceinline__ uint64_t splitmix64_output(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t counter_u64(uint64_t seed, uint64_t stream, uint64_t idx) {
    uint64_t ctr = stream * (1ull << 40) + idx + 1ull;
    return splitmix64_output(seed + ctr * 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ double counter_uniform(uint64_t seed, uint64_t stream, uint64_t idx) {
    return (double)(counter_u64(seed, stream, idx) >> 11) * 0x1.0p-53;
}

constexpr uint64_t STREAM_TV = 0;
constexpr uint64_t STREAM_CR = 1ull << 22;
constexpr uint64_t STREAM_MIS = 1ull << 23;
constexpr uint64_t STREAM_COLOUR = 1ull << 21;  // + (level << 8) + colour: the smoother's colouring

// 16-byte vector of T: 2 doubles or 4 floats.
template <typename T>
struct V16;
template <>
struct V16<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ static void load(const double* p, double* o) {
        double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    }
    __device__ static void store(double* p, const double* o) { *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]); }
};
template <>
struct V16<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ static void load(const float* p, float* o) {
        float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    __device__ static void store(float* p, const float* o) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Multiply and add with rounding after each operation (no contraction into an FMA),
// so that sums computed in the same order match a plain CPU evaluation bit for bit.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// w / h rounded to nearest, given r = 1 / h rounded to nearest: q0 = w r lies within an ulp
// of the quotient, the remainder w - q0 h is exact in one fma, and q0 + rem r rounded once is
// the correctly rounded quotient (Markstein's theorem: P. Markstein, IBM J. Res. Dev. 34(1),
// 1990).  Three FP64 operations instead of a full division, for the many quotients by one
// divisor; it holds for quotients in the normal range.  A zero remainder keeps q0, and with
// it the sign of a zero quotient.
__device__ __forceinline__ double div_by_recip(double w, double h, double r) {
    const double q0 = __dmul_rn(w, r);
    const double rem = __fma_rn(-q0, h, w);
    return rem == 0.0 ? q0 : __fma_rn(rem, r, q0);
}

// ------------------------------------------------------------------ host helpers
// d_out has n + 1 entries; with h_total (the device address of mapped host memory) the total
// is also stored there
void exclusive_scan(const int32_t* d_in, int32_t* d_out, int n, cudaStream_t s, int32_t* h_total = nullptr);
int32_t exclusive_scan_total(const int32_t* d_in, int32_t* d_out, int n, cudaStream_t s);  // the total, to the host
int32_t read_int(const int32_t* d_p, cudaStream_t s);  // a device int, to the host (after s's earlier work)

}  // namespace bamg
