// Scene lifetime, workspace arena and error reporting of libludvig.
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

namespace ludvig {

namespace {
thread_local char g_last_error[1024] = "";
}

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

// ---------------------------------------------------------------- tracing
namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_trace{false};
struct TraceRec {
    int stage;
    cudaEvent_t a, b;
};
std::mutex g_trace_mu;
std::vector<TraceRec> g_recs;        // recorded, not yet read
std::vector<cudaEvent_t> g_free_ev;  // reusable events
double g_ms[16];
int64_t g_calls[16];

cudaEvent_t take_event() {
    if (!g_free_ev.empty()) {
        cudaEvent_t e = g_free_ev.back();
        g_free_ev.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Host-side fault injection: an armed counter k > 0 makes the k-th event from
// now fail once (then disarms).  Nothing reaches the GPU.
namespace {
std::atomic<int64_t> g_fault_alloc{0}, g_fault_launch{0};
bool fault_tick(std::atomic<int64_t>& c) {
    int64_t v = c.load();
    while (v > 0) {
        if (c.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}
}  // namespace
bool fault_launch_now() { return g_fault_launch.load(std::memory_order_relaxed) > 0 && fault_tick(g_fault_launch); }
bool trace_on() { return g_trace.load(std::memory_order_relaxed); }

int trace_begin(int stage, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return -1;
    if (cudaEventRecord(a, st) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    g_recs.push_back({stage, a, b});
    return (int)g_recs.size() - 1;
}

void trace_end(int slot, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (slot < 0 || slot >= (int)g_recs.size()) return;
    if (cudaEventRecord(g_recs[slot].b, st) != cudaSuccess) cudaGetLastError();
}

Arena::~Arena() { release(); }

void Arena::release() {
    for (auto& kv : dev_)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (auto& kv : host_)
        if (kv.second.ptr) cudaFreeHost(kv.second.ptr);
    dev_.clear();
    host_.clear();
    bytes_.store(0);
}

ludvig_status Arena::get(const char* name, size_t bytes, void** out) {
    Buf& b = dev_[name];
    if (bytes == 0) bytes = 1;
    if (b.bytes < bytes) {
        if (b.ptr) {
            // a kernel queued earlier may still read the old buffer
            LV_CUDA(cudaDeviceSynchronize());
            LV_CUDA(cudaFree(b.ptr));
            bytes_.fetch_sub(b.bytes);
            b.ptr = nullptr;
            b.bytes = 0;
        }
        const size_t want = bytes + bytes / 8;   // grow with some headroom
        if (g_fault_alloc.load(std::memory_order_relaxed) > 0 && fault_tick(g_fault_alloc)) {
            set_error("workspace '%s': injected allocation failure", name);
            return LUDVIG_ERR_OOM;
        }
        cudaError_t e = cudaMalloc(&b.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&b.ptr, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b.ptr = nullptr;
                set_error("workspace '%s': cudaMalloc of %zu bytes failed: %s", name, bytes,
                          cudaGetErrorString(e));
                return LUDVIG_ERR_OOM;
            }
            b.bytes = bytes;
        } else {
            b.bytes = want;
        }
        bytes_.fetch_add(b.bytes);
    }
    *out = b.ptr;
    return LUDVIG_OK;
}

ludvig_status Arena::pinned(const char* name, size_t bytes, void** out) {
    Buf& b = host_[name];
    if (b.bytes < bytes) {
        if (b.ptr) {
            LV_CUDA(cudaDeviceSynchronize());
            LV_CUDA(cudaFreeHost(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        LV_CUDA(cudaMallocHost(&b.ptr, bytes));
        b.bytes = bytes;
    }
    *out = b.ptr;
    return LUDVIG_OK;
}

ludvig_status scene_init(ludvig_scene* s, const float* means, const float* scales, const float* quats,
                         const float* opac, int scales_are_linear, cudaStream_t st);
void scene_release_async(ludvig_scene* s);

}  // namespace ludvig

using namespace ludvig;

extern "C" int32_t ludvig_abi_version(void) { return LUDVIG_ABI_VERSION; }

extern "C" const char* ludvig_last_error(void) { return g_last_error; }

extern "C" ludvig_status ludvig_scene_create(const float* means, const float* scales, const float* quats,
                                             const float* opacity, int64_t n, const ludvig_scene_opts* opts,
                                             void* stream, ludvig_scene_t* out) {
    LV_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    LV_ARG(n >= 0 && n < ((int64_t)1 << 31), "n must be in [0, 2^31)");
    LV_ARG(n == 0 || (means && scales && quats && opacity), "NULL input array");
    ludvig_scene* s = new (std::nothrow) ludvig_scene();
    LV_ARG(s != nullptr, "host allocation failed");
    s->n = n;
    LV_CUDA(cudaGetDevice(&s->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n > 0) {
        const size_t nn = (size_t)n;
        if (cudaMalloc(&s->geo, nn * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&s->cov_a, nn * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&s->cov_b, nn * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&s->means, nn * 3 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            ludvig_scene_destroy(s);
            set_error("scene allocation failed for n=%lld", (long long)n);
            return LUDVIG_ERR_OOM;
        }
        const int linear = opts ? (opts->scales_are_linear != 0) : 0;
        ludvig_status r = scene_init(s, means, scales, quats, opacity, linear, st);
        if (r != LUDVIG_OK) {
            ludvig_scene_destroy(s);
            return r;
        }
    }
    *out = s;
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_scene_destroy(ludvig_scene_t s) {
    if (!s) return LUDVIG_OK;
    cudaDeviceSynchronize();
    cudaFree(s->geo);
    cudaFree(s->cov_a);
    cudaFree(s->cov_b);
    cudaFree(s->means);
    for (int b = 0; b < 2; ++b) {
        if (s->ev_ready[b]) cudaEventDestroy(s->ev_ready[b]);
        if (s->ev_free[b]) cudaEventDestroy(s->ev_free[b]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    scene_release_async(s);
    s->ws.release();
    delete s;
    return LUDVIG_OK;
}

extern "C" int64_t ludvig_scene_size(ludvig_scene_t s) { return s ? s->n : -1; }

extern "C" int64_t ludvig_scene_workspace_bytes(ludvig_scene_t s) { return s ? (int64_t)s->ws.device_bytes() : -1; }

namespace ludvig {
namespace {
std::atomic<int64_t> g_opt_f32_tc{1};
std::atomic<int64_t> g_opt_count{0};
std::atomic<int64_t> g_opt_agg_config{0};
std::atomic<int64_t> g_opt_group_mb{2048};
std::atomic<int64_t> g_opt_batch_tune{1};
std::atomic<int64_t> g_opt_batch_pack{1};
std::atomic<int64_t> g_opt_agg_sms{0};
}
bool option_f32_tensor_cores() { return g_opt_f32_tc.load() != 0; }
bool option_count_normalise() { return g_opt_count.load() != 0; }
int option_agg_config() { return (int)g_opt_agg_config.load(); }
int64_t option_group_bytes() { return g_opt_group_mb.load() << 20; }
bool option_batch_tune() { return g_opt_batch_tune.load() != 0; }
bool option_batch_pack() { return g_opt_batch_pack.load() != 0; }
int option_agg_sms() { return (int)g_opt_agg_sms.load(); }
}  // namespace ludvig

extern "C" ludvig_status ludvig_set_option(int32_t option, int64_t value) {
    switch (option) {
        case LUDVIG_OPT_F32_TENSOR_CORES:
            g_opt_f32_tc.store(value != 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_COUNT_NORMALISE:
            g_opt_count.store(value != 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_FAULT_ALLOC:
            g_fault_alloc.store(value > 0 ? value : 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_FAULT_LAUNCH:
            g_fault_launch.store(value > 0 ? value : 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_AGG_CONFIG:
            if (value < 0 || value > 1) {
                set_error("LUDVIG_OPT_AGG_CONFIG must be 0 or 1");
                return LUDVIG_ERR_ARG;
            }
            g_opt_agg_config.store(value);
            return LUDVIG_OK;
        case LUDVIG_OPT_GROUP_MB:
            if (value < 1 || value > (64 << 10)) {
                set_error("LUDVIG_OPT_GROUP_MB must be in [1, 65536]");
                return LUDVIG_ERR_ARG;
            }
            g_opt_group_mb.store(value);
            return LUDVIG_OK;
        case LUDVIG_OPT_BATCH_TUNE:
            g_opt_batch_tune.store(value != 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_BATCH_PACK:
            g_opt_batch_pack.store(value != 0);
            return LUDVIG_OK;
        case LUDVIG_OPT_AGG_SMS:
            if (value < 0 || value > 4096) {
                set_error("LUDVIG_OPT_AGG_SMS must be in [0, 4096]");
                return LUDVIG_ERR_ARG;
            }
            g_opt_agg_sms.store(value);
            return LUDVIG_OK;
        default:
            set_error("unknown option %d", option);
            return LUDVIG_ERR_ARG;
    }
}

extern "C" int64_t ludvig_get_option(int32_t option) {
    switch (option) {
        case LUDVIG_OPT_F32_TENSOR_CORES: return g_opt_f32_tc.load();
        case LUDVIG_OPT_COUNT_NORMALISE: return g_opt_count.load();
        case LUDVIG_OPT_FAULT_ALLOC: return g_fault_alloc.load();
        case LUDVIG_OPT_FAULT_LAUNCH: return g_fault_launch.load();
        case LUDVIG_OPT_AGG_CONFIG: return g_opt_agg_config.load();
        case LUDVIG_OPT_GROUP_MB: return g_opt_group_mb.load();
        case LUDVIG_OPT_BATCH_TUNE: return g_opt_batch_tune.load();
        case LUDVIG_OPT_BATCH_PACK: return g_opt_batch_pack.load();
        case LUDVIG_OPT_AGG_SMS: return g_opt_agg_sms.load();
        default: return -1;
    }
}

extern "C" ludvig_status ludvig_trace_enable(int32_t on) {
    g_trace.store(on != 0);
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_trace_read(ludvig_trace* out, int32_t reset) {
    LV_ARG(out != nullptr, "out is NULL");
    std::lock_guard<std::mutex> lk(g_trace_mu);
    for (auto& r : g_recs) {
        LV_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        LV_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.stage >= 0 && r.stage < 16) {
            g_ms[r.stage] += ms;
            g_calls[r.stage] += 1;
        }
        g_free_ev.push_back(r.a);
        g_free_ev.push_back(r.b);
    }
    g_recs.clear();
    for (int i = 0; i < 16; ++i) {
        out->ms[i] = g_ms[i];
        out->calls[i] = g_calls[i];
    }
    out->kernel_launches = g_launches.load();
    if (reset) {
        for (int i = 0; i < 16; ++i) {
            g_ms[i] = 0.0;
            g_calls[i] = 0;
        }
        g_launches.store(0);
    }
    return LUDVIG_OK;
}
