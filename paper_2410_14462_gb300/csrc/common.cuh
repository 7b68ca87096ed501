// Internal declarations shared by the libludvig translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "ludvig.h"

namespace ludvig {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

// ---------------------------------------------------------------- tracing
void count_launch();
bool fault_launch_now();   // host-side fault injection (LUDVIG_OPT_FAULT_LAUNCH)
bool trace_on();
int trace_begin(int stage, cudaStream_t st);   // returns a slot or -1
void trace_end(int slot, cudaStream_t st);

// Brackets a scope with stage events when tracing is on.
struct StageScope {
    int slot;
    cudaStream_t st;
    StageScope(int stage, cudaStream_t s) : slot(trace_on() ? trace_begin(stage, s) : -1), st(s) {}
    ~StageScope() {
        if (slot >= 0) trace_end(slot, st);
    }
};

#define LV_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            ::ludvig::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                  \
                                cudaGetErrorString(_e));                                   \
            return _e == cudaErrorMemoryAllocation ? LUDVIG_ERR_OOM : LUDVIG_ERR_CUDA;      \
        }                                                                                  \
    } while (0)

#define LV_LAUNCH()                                                                        \
    do {                                                                                   \
        ::ludvig::count_launch();                                                          \
        if (::ludvig::fault_launch_now()) {                                                \
            ::ludvig::set_error("%s:%d kernel launch: injected failure", __FILE__, __LINE__); \
            return LUDVIG_ERR_CUDA;                                                        \
        }                                                                                  \
        cudaError_t _e = cudaGetLastError();                                               \
        if (_e != cudaSuccess) {                                                           \
            ::ludvig::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,              \
                                cudaGetErrorString(_e));                                   \
            return LUDVIG_ERR_CUDA;                                                        \
        }                                                                                  \
    } while (0)

#define LV_TRY(expr)                                                                       \
    do {                                                                                   \
        ludvig_status _s = (expr);                                                         \
        if (_s != LUDVIG_OK) return _s;                                                    \
    } while (0)

#define LV_ARG(cond, ...)                                                                  \
    do {                                                                                   \
        if (!(cond)) {                                                                     \
            ::ludvig::set_error(__VA_ARGS__);                                              \
            return LUDVIG_ERR_ARG;                                                         \
        }                                                                                  \
    } while (0)

// ---------------------------------------------------------------- workspace
// Grow-only named device buffers.  A buffer keeps its contents only until the
// next call that grows it; callers treat workspace as scratch.
class Arena {
  public:
    Arena() = default;
    Arena(const Arena&) = delete;              // buffers have one owner
    Arena& operator=(const Arena&) = delete;
    ~Arena();
    // Exchanges the buffers of two workspaces (lending a pooled workspace).
    void swap(Arena& o) noexcept {
        dev_.swap(o.dev_);
        host_.swap(o.host_);
        const size_t a = bytes_.load(), b = o.bytes_.load();
        bytes_.store(b);
        o.bytes_.store(a);
    }
    // Device bytes held (readable from any thread while another grows it).
    size_t device_bytes() const { return bytes_.load(std::memory_order_relaxed); }
    // Returns a device buffer of at least `bytes` bytes (256-byte aligned).
    ludvig_status get(const char* name, size_t bytes, void** out);
    template <class T>
    ludvig_status get(const char* name, size_t count, T** out) {
        void* p = nullptr;
        ludvig_status s = get(name, count * sizeof(T), &p);
        *out = static_cast<T*>(p);
        return s;
    }
    ludvig_status pinned(const char* name, size_t bytes, void** out);   // host, page-locked
    void release();

  private:
    struct Buf {
        void* ptr = nullptr;
        size_t bytes = 0;
    };
    std::unordered_map<std::string, Buf> dev_, host_;
    std::atomic<size_t> bytes_{0};
};

// Device-side sizes of one group of views of an asynchronous uplift, copied
// back to the host with the call's status: the (tile, Gaussian) pairs the
// group needed and the weight chunks it filled.
struct GroupDiag {
    uint64_t pairs;
    int32_t chunks;
    int32_t pad;
};

// An asynchronous uplift call whose device-side capacity checks have not been
// read yet (ludvig_sync, or the next call on the scene, reads them).  The
// arguments are kept so that groups which did not fit the workspace can be
// redone once it has grown.
struct PendingCall {
    bool active = false;
    int kind = 0;                      // 0: accumulate into num/den, 1: uplift (+ normalise)
    int src = 0;                       // 0: plain features, 1: zero-padded to 32 channels, 2: FP8 codes
    std::vector<ludvig_camera> cams;
    int n_views = 0, width = 0, height = 0, dtype = 0, d = 0;
    const void* feats = nullptr;       // features or FP8 codes
    const float* scales = nullptr;     // FP8 per-view scales
    float* num = nullptr;
    float* den = nullptr;
    std::vector<int> v0, nv;                    // the groups' views
    std::vector<int64_t> pair_cap, chunk_cap;   // the capacities each group ran with
};

}  // namespace ludvig

// The opaque scene: a device copy of the Gaussians with the view-independent
// 3D covariance precomputed.
struct ludvig_scene {
    int64_t n = 0;
    int device = 0;
    float4* geo = nullptr;     // [n] (mean.x, mean.y, mean.z, opacity)
    float4* cov_a = nullptr;   // [n] (S00, S01, S02, S11)
    float2* cov_b = nullptr;   // [n] (S12, S22)
    float* means = nullptr;    // [n,3] copy (kNN, graph)
    cudaStream_t copy_stream = nullptr;   // host-feature uploads (created on first use)
    cudaEvent_t ev_ready[2] = {nullptr, nullptr};
    cudaEvent_t ev_free[2] = {nullptr, nullptr};
    int64_t tc_chunk_cap = 0;             // tensor-core path: weight chunks kept in ws
    int64_t pair_cap = 0;                 // (tile, Gaussian) pairs per group kept in ws
    bool onesweep = false;                // sorts with the one-sweep radix sort (packed batch contexts)
    // asynchronous uplift: front-end and aggregation streams, their events,
    // the device status words ([0] bounded-wait status, [1] capacity overflow)
    // and their host mirror with the groups' sizes
    cudaStream_t st_front = nullptr, st_agg = nullptr;
    cudaEvent_t ev_call = nullptr, ev_front[2] = {nullptr, nullptr}, ev_agg[2] = {nullptr, nullptr};
    cudaEvent_t ev_join[2] = {nullptr, nullptr}, ev_done = nullptr;
    int* dstat = nullptr;                 // device [2]
    int* hstat = nullptr;                 // pinned [2], written at the end of each call
    ludvig::GroupDiag* ddiag = nullptr;   // device [diag_cap]
    ludvig::GroupDiag* hdiag = nullptr;   // pinned [diag_cap]
    int diag_cap = 0;
    ludvig::PendingCall pending;
    ludvig::Arena ws;
};

struct ludvig_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int device = 0;
    int64_t* row_ptr = nullptr;   // [n+1]
    int32_t* col = nullptr;       // [nnz]
    float* val = nullptr;         // [nnz]
    float* d2 = nullptr;          // [nnz] ||f^_i - f^_j||^2 (RBF graphs only)
    float s_f = 0.f;              // median edge feature distance (RBF graphs only)
    int val_version = 0;          // bumped whenever val changes
    int sell_version = -1;        // val_version of the sliced copy in ws ("sell.*"), -1: none
    int64_t sell_slices = 0;
    int32_t* perm = nullptr;      // [n] node at position r of the kNN grid's cell order (null: identity)
    int32_t* inv = nullptr;       // [n] position of each node in that order
    ludvig::Arena ws;
};

namespace ludvig {

// ---------------------------------------------------------------- primitives
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;   // keys per sort block

// Exclusive prefix sum of n uint32 values (in-place allowed).  *total_dev
// (device, may be null) receives the exact 64-bit sum; the uint32 prefixes are
// meaningful only while that sum stays below 2^32.
ludvig_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total_dev,
                                 Arena& ws, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on key bits [0, nbits), applied
// independently to nseg consecutive segments of seg_len entries each
// (seg_len % kRadixTile == 0).  Sorted data ends in (*keys, *vals), which may
// be swapped with (keys_alt, vals_alt).
ludvig_status radix_sort_pairs(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt,
                               uint32_t* vals_alt, int64_t nseg, int64_t seg_len, int nbits,
                               Arena& ws, cudaStream_t st);

// The same for one segment whose valid length is read on the device: `len`
// (device, may be null = all of seg_len) entries of the seg_len-entry buffers
// are sorted; the output holds them first, then (up to the next multiple of
// kRadixTile) largest-key fillers.  The caller guarantees that the rounded-up
// length fits the buffers.
ludvig_status radix_sort_pairs_len(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt,
                                   uint32_t* vals_alt, int64_t nseg, int64_t seg_len, const uint64_t* len,
                                   int nbits, Arena& ws, cudaStream_t st);

// radix_sort_pairs_len with 16-bit keys (nbits <= 16): less traffic per pass.
ludvig_status radix_sort_pairs_len16(uint16_t** keys, uint32_t** vals, uint16_t* keys_alt, uint32_t* vals_alt,
                                     int64_t nseg, int64_t seg_len, const uint64_t* len, int nbits, Arena& ws,
                                     cudaStream_t st);

// The same sort (and the same device-length rule) with one kernel per pass
// after an up-front histogram of every pass; the passes chain their prefix
// through the blocks.  A wait that runs past its bound records
// LUDVIG_ERR_TIMEOUT in *err (device, may be null).
ludvig_status radix_sort_onesweep(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                  int64_t nseg, int64_t seg_len, const uint64_t* len, int nbits, int* err,
                                  Arena& ws, cudaStream_t st);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

}  // namespace ludvig
