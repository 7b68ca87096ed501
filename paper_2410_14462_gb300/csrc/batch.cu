// Batched uplift: many independent uplifts (Sec. 3.2, Eq. 5, one per job) of
// uneven size on one GPU.  The paper runs one uplift at a time; this is the
// executor that keeps the GPU busy across jobs.
//
// Packed jobs (the tensor-core path: bfloat16, or float32 with the
// tensor-core option, and d < 32 through the zero-padded path) share their
// launches.  Jobs with the same feature dtype, channel count and image size
// whose feature arrays lie at whole-view offsets from one another form a
// class; the views of a class's jobs are packed, largest scene first, into
// common groups (views of several jobs in one group: each view carries its
// own scene, camera, feature coordinate and output in the kernels'
// parameters), so that a launch of each pipeline stage serves up to 128
// views of many jobs.  The group size (views per group under a bound on the
// per-view Gaussian scratch and the pixels) is picked per class by a tuner
// that times candidate sizes on the class's own jobs the first time it meets
// the class (LUDVIG_OPT_BATCH_TUNE), and kept for later batches.  The classes
// run one after another, largest first, on one pooled context (a workspace,
// two streams and their events) driven by the calling thread: each class
// fills the GPU with its groups, and one context bounds the weight-row
// memory.
//
// Other jobs (the CUDA-core float32 path) run as ludvig_uplift calls on
// `slots` host threads (the calling thread joins them after the classes),
// each with its own stream and a pooled workspace lent to the job's scene for
// the call (swapped in and back out), longest job first.
//
// Every slot stream waits for an event recorded on the caller's stream before
// its first job, and the caller's stream waits for every slot's final event,
// so the batch is ordered on `stream` like one call.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "uplift_int.cuh"

namespace ludvig {

bool option_batch_tune();
bool option_batch_pack();
int64_t option_group_bytes();

namespace {

double job_cost(const ludvig_uplift_job& j) {
    // pixels x Gaussians x channels, with a floor on the channels for the
    // D-independent walk
    return (double)ludvig_scene_size(j.scene) * (double)j.n_views * (double)j.width * (double)j.height *
           (double)std::max<int32_t>(j.d, 32);
}

// Idle slot workspaces and packed contexts per device.  Never destroyed at
// exit: no CUDA call may run from a static destructor; process exit returns
// the memory.
std::mutex g_pool_mu;
using Pool = std::unordered_map<int, std::vector<std::unique_ptr<Arena>>>;
using CtxPool = std::unordered_map<int, std::vector<ludvig_scene*>>;
Pool& pool() {
    static Pool* p = new Pool();
    return *p;
}
CtxPool& ctx_pool() {
    static CtxPool* p = new CtxPool();
    return *p;
}

std::unique_ptr<Arena> take_workspace(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto& v = pool()[dev];
    if (v.empty()) return std::make_unique<Arena>();
    std::unique_ptr<Arena> a = std::move(v.back());
    v.pop_back();
    return a;
}

void return_workspace(int dev, std::unique_ptr<Arena> a) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool()[dev].push_back(std::move(a));
}

// A packed context: a scene object without Gaussians, used for its
// workspace, streams, events and status words.
ludvig_scene* take_context(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto& v = ctx_pool()[dev];
    if (!v.empty()) {
        ludvig_scene* c = v.back();
        v.pop_back();
        return c;
    }
    ludvig_scene* c = new (std::nothrow) ludvig_scene();
    if (c) {
        c->device = dev;
        c->onesweep = true;   // many groups: one kernel per radix pass
    }
    return c;
}

void return_context(int dev, ludvig_scene* c) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    ctx_pool()[dev].push_back(c);
}

struct SlotResources {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    ~SlotResources() {
        // both are released by the runtime once pending work completes
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : done)
            if (e) cudaEventDestroy(e);
        if (start) cudaEventDestroy(start);
    }
};

// ------------------------------------------------------------ classes

size_t elem_size(int dtype) { return dtype == LUDVIG_F32 ? 4 : 2; }

// Jobs that may share groups: same dtype, d and image size, features at
// whole-view offsets from one another (same address modulo the view size).
struct ClassKey {
    int dtype, d, width, height;
    uint64_t residue;
    bool operator<(const ClassKey& o) const {
        return std::tie(dtype, d, width, height, residue) < std::tie(o.dtype, o.d, o.width, o.height, o.residue);
    }
};

struct JobClass {
    ClassKey key;
    std::vector<int32_t> jobs;   // largest scene first
    const char* base = nullptr;  // lowest feature address of the class
    double cost = 0.0;
    int groups = 0;
    int64_t group_bytes = 0;
    bool tuned = false;
};

// ------------------------------------------------------------ tuner
// Group size per (dtype, d, image size, scene size class): the fastest of
// the candidate scratch budgets on a sample of the class's own jobs.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int64_t>& tune_table() {
    static auto* t = new std::map<std::tuple<int, int, int, int, int>, int64_t>();
    return *t;
}

constexpr int64_t kMiB = (int64_t)1 << 20;
// (a group's weight rows grow with its views too: a 2 GiB scratch bound
// keeps a context near 10 GiB at paper scale)
const int64_t kCandidates[] = {256 * kMiB, 512 * kMiB, 1024 * kMiB, 2048 * kMiB};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

// Frees a context's workspace and forgets its capacities (after a failed
// allocation: the next call sizes them again on its first group).
void reset_context(ludvig_scene* ctx) {
    cudaDeviceSynchronize();
    cudaGetLastError();
    ctx->ws.release();
    ctx->pair_cap = 0;
    ctx->tc_chunk_cap = 0;
}

std::tuple<int, int, int, int, int> tune_key(const ludvig_uplift_job* jobs, const JobClass& c) {
    double sum = 0.0;
    for (int32_t j : c.jobs) sum += (double)ludvig_scene_size(jobs[j].scene);
    const double mean = std::max(1.0, sum / (double)c.jobs.size());
    return std::make_tuple(c.key.dtype, c.key.d, c.key.width, c.key.height, (int)std::floor(std::log2(mean)));
}

// Times each candidate on up to 4 jobs of the class (spread over its scene
// sizes) and up to 64 views of each, outputs in the context's scratch (the
// jobs' outputs are untouched);
// one run at the largest candidate first grows the workspace.  A candidate
// that runs out of device memory is dropped with every larger one.
ludvig_status tune_class(ludvig_scene* ctx, const ludvig_uplift_job* jobs, const JobClass& c, cudaStream_t st,
                         int64_t* best) {
    const size_t vb = (size_t)c.key.width * c.key.height * c.key.d * elem_size(c.key.dtype);
    std::vector<PackedJob> sample;
    int64_t out_elems = 0, beta_elems = 0;
    int views = 0;
    // up to 4 jobs spread over the class's sizes (largest first), 64 views each
    std::vector<int32_t> pick;
    const size_t nj = c.jobs.size();
    for (size_t q = 0; q < 4 && q < nj; ++q) {
        const int32_t j = c.jobs[nj <= 4 ? q : q * (nj - 1) / 3];
        if (pick.empty() || pick.back() != j) pick.push_back(j);
    }
    for (int32_t j : pick) {
        if (views >= 256) break;
        const ludvig_uplift_job& J = jobs[j];
        const int nv = std::min(std::min(J.n_views, 64), 256 - views);
        if (nv <= 0 || J.scene->n == 0) continue;
        // scratch outputs of at most about 2 GiB (the first job always)
        if (!sample.empty() && out_elems + J.scene->n * (int64_t)c.key.d > ((int64_t)1 << 29)) break;
        PackedJob p{J.scene, J.cams, nv, (int)((static_cast<const char*>(J.feats) - c.base) / vb), nullptr, nullptr};
        sample.push_back(p);
        out_elems += round_up(J.scene->n * c.key.d, 64);
        beta_elems += round_up(J.scene->n, 64);
        views += nv;
    }
    *best = option_group_bytes();
    if (sample.empty()) return LUDVIG_OK;
    // the scratch outputs live in the context's workspace: bound again after
    // every reset of the context
    auto bind_scratch = [&]() -> ludvig_status {
        float *out, *beta;
        LV_TRY(ctx->ws.get("tune.out", (size_t)out_elems, &out));
        LV_TRY(ctx->ws.get("tune.beta", (size_t)beta_elems, &beta));
        for (PackedJob& p : sample) {
            p.out = out;
            p.beta = beta;
            out += round_up(p.scene->n * c.key.d, 64);
            beta += round_up(p.scene->n, 64);
        }
        return LUDVIG_OK;
    };
    LV_TRY(bind_scratch());
    cudaEvent_t e0, e1;
    LV_CUDA(cudaEventCreate(&e0));
    LV_CUDA(cudaEventCreate(&e1));
    struct Events {
        cudaEvent_t a, b;
        ~Events() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    // the largest candidate that fits in memory grows the workspace first;
    // larger ones are dropped
    int top = kNumCandidates - 1;
    for (;; --top) {
        const ludvig_status r = uplift_packed(ctx, sample.data(), (int)sample.size(), c.base, c.key.dtype, c.key.d,
                                              c.key.width, c.key.height, kCandidates[top], st, nullptr);
        if (r == LUDVIG_OK) break;
        if (r != LUDVIG_ERR_OOM || top == 0) return r;
        reset_context(ctx);
        LV_TRY(bind_scratch());
    }
    float best_ms = 0.f;
    for (int k = 0; k <= top; ++k) {
        LV_CUDA(cudaEventRecord(e0, st));
        LV_TRY(uplift_packed(ctx, sample.data(), (int)sample.size(), c.base, c.key.dtype, c.key.d, c.key.width,
                             c.key.height, kCandidates[k], st, nullptr));
        LV_CUDA(cudaEventRecord(e1, st));
        LV_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (k == 0 || ms < best_ms) {
            best_ms = ms;
            *best = kCandidates[k];
        }
    }
    // the real run sizes the workspace for the choice
    reset_context(ctx);
    return LUDVIG_OK;
}

ludvig_status class_group_bytes(ludvig_scene* ctx, const ludvig_uplift_job* jobs, JobClass& c, cudaStream_t st) {
    c.group_bytes = option_group_bytes();
    c.tuned = false;
    if (!option_batch_tune()) return LUDVIG_OK;
    const auto key = tune_key(jobs, c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = tune_table().find(key);
        if (it != tune_table().end()) {
            c.group_bytes = it->second;
            c.tuned = true;
            return LUDVIG_OK;
        }
    }
    int64_t best = 0;
    LV_TRY(tune_class(ctx, jobs, c, st, &best));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_table()[key] = best;
    c.group_bytes = best;
    c.tuned = true;
    return LUDVIG_OK;
}

// The plan of the last batch (ludvig_batch_last_plan).
std::mutex g_plan_mu;
std::vector<ludvig_batch_class>& last_plan() {
    static auto* p = new std::vector<ludvig_batch_class>();
    return *p;
}

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_uplift_batch(const ludvig_uplift_job* jobs, int32_t n_jobs, int32_t slots,
                                             int32_t* job_status, void* stream) {
    LV_ARG(n_jobs >= 0, "n_jobs must be >= 0");
    LV_ARG(n_jobs == 0 || jobs != nullptr, "jobs is NULL");
    LV_ARG(slots >= 1 && slots <= LUDVIG_MAX_BATCH_SLOTS, "slots must be in [1, %d]", LUDVIG_MAX_BATCH_SLOTS);
    if (n_jobs == 0) return LUDVIG_OK;
    std::vector<ludvig_scene_t> scenes((size_t)n_jobs);
    for (int32_t j = 0; j < n_jobs; ++j) {
        LV_ARG(jobs[j].scene != nullptr, "job %d: scene is NULL", j);
        scenes[(size_t)j] = jobs[j].scene;
    }
    std::sort(scenes.begin(), scenes.end());
    LV_ARG(std::adjacent_find(scenes.begin(), scenes.end()) == scenes.end(),
           "two jobs share a scene (a scene serves one stream at a time)");

    std::vector<ludvig_status> status((size_t)n_jobs, LUDVIG_OK);
    std::vector<std::string> message((size_t)n_jobs);
    // a job with invalid arguments fails alone; the scenes' pending calls complete first
    for (int32_t j = 0; j < n_jobs; ++j) {
        const ludvig_uplift_job& J = jobs[j];
        ludvig_status r = check_uplift_args(J.scene, J.cams, J.n_views, J.width, J.height, J.feats, J.dtype, J.d,
                                            J.out);
        if (r == LUDVIG_OK) r = scene_sync(J.scene);
        if (r != LUDVIG_OK) {
            status[(size_t)j] = r;
            message[(size_t)j] = ludvig_last_error();
        }
    }

    // classes of packed jobs; the rest run as single calls
    std::map<ClassKey, JobClass> by_key;
    std::vector<int32_t> plain;
    for (int32_t j = 0; j < n_jobs; ++j) {
        if (status[(size_t)j] != LUDVIG_OK) continue;
        const ludvig_uplift_job& J = jobs[j];
        const size_t vb = (size_t)J.width * J.height * J.d * elem_size(J.dtype);
        const bool packable = option_batch_pack() && packed_supported(J.dtype, J.d) && J.n_views > 0 &&
                              J.scene->n > 0 &&
                              (reinterpret_cast<uintptr_t>(J.feats) & 15) == 0 && vb % 16 == 0;
        if (!packable) {
            plain.push_back(j);
            continue;
        }
        ClassKey k{J.dtype, J.d, J.width, J.height, (uint64_t)(reinterpret_cast<uintptr_t>(J.feats) % vb)};
        JobClass& c = by_key[k];
        c.key = k;
        c.jobs.push_back(j);
        const char* f = static_cast<const char*>(J.feats);
        if (!c.base || f < c.base) c.base = f;
        c.cost += job_cost(J);
    }
    std::vector<JobClass> classes;
    for (auto& kv : by_key) {
        JobClass& c = kv.second;
        const size_t vb = (size_t)c.key.width * c.key.height * c.key.d * elem_size(c.key.dtype);
        // view coordinates must fit the tensor map and an int
        std::vector<int32_t> keep;
        for (int32_t j : c.jobs) {
            const size_t off = (size_t)(static_cast<const char*>(jobs[j].feats) - c.base) / vb;
            if (off + (size_t)jobs[j].n_views < ((size_t)1 << 31))
                keep.push_back(j);
            else
                plain.push_back(j);
        }
        c.jobs.swap(keep);
        if (c.jobs.empty()) continue;
        std::stable_sort(c.jobs.begin(), c.jobs.end(), [&](int32_t a, int32_t b) {
            return ludvig_scene_size(jobs[a].scene) > ludvig_scene_size(jobs[b].scene);
        });
        classes.push_back(std::move(c));
    }
    std::stable_sort(classes.begin(), classes.end(),
                     [](const JobClass& a, const JobClass& b) { return a.cost > b.cost; });
    std::stable_sort(plain.begin(), plain.end(),
                     [&](int32_t a, int32_t b) { return job_cost(jobs[a]) > job_cost(jobs[b]); });

    // the classes run in the calling thread on one context, largest first
    // (each fills the GPU with groups of many views; one context bounds the
    // weight-row memory); the single jobs run on every slot thread, the
    // calling thread joining them after the classes
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const int nslots = std::max(1, std::min<int>(slots, (int)plain.size() + (classes.empty() ? 0 : 1)));
    SlotResources res;
    res.streams.assign((size_t)nslots, nullptr);
    res.done.assign((size_t)nslots, nullptr);
    LV_CUDA(cudaEventCreateWithFlags(&res.start, cudaEventDisableTiming));
    for (int k = 0; k < nslots; ++k) {
        LV_CUDA(cudaStreamCreateWithFlags(&res.streams[(size_t)k], cudaStreamNonBlocking));
        LV_CUDA(cudaEventCreateWithFlags(&res.done[(size_t)k], cudaEventDisableTiming));
    }
    LV_CUDA(cudaEventRecord(res.start, caller));
    for (int k = 0; k < nslots; ++k) LV_CUDA(cudaStreamWaitEvent(res.streams[(size_t)k], res.start, 0));

    std::atomic<int> next{0};
    std::vector<cudaError_t> slot_err((size_t)nslots, cudaSuccess);
    std::vector<PackedStats> cstats(classes.size());
    std::vector<float> cms(classes.size(), 0.f);
    std::vector<int64_t> cws(classes.size(), 0);
    auto fail = [&](int32_t j, ludvig_status r) {
        status[(size_t)j] = r;
        message[(size_t)j] = ludvig_last_error();
    };
    auto run_classes = [&](cudaStream_t st) {
        if (classes.empty()) return;
        ludvig_scene* ctx = nullptr;
        try {
            ctx = take_context(dev);
        } catch (...) {
        }
        for (size_t i = 0; i < classes.size(); ++i) {
            JobClass& c = classes[i];
            ludvig_status r = LUDVIG_ERR_OOM;
            if (!ctx) set_error("no context for the packed jobs");
            try {
                const auto t0 = std::chrono::steady_clock::now();
                if (ctx) r = class_group_bytes(ctx, jobs, c, st);
                if (ctx && r == LUDVIG_OK) {
                    const size_t vb = (size_t)c.key.width * c.key.height * c.key.d * elem_size(c.key.dtype);
                    std::vector<PackedJob> pj;
                    for (int32_t j : c.jobs) {
                        const ludvig_uplift_job& J = jobs[j];
                        pj.push_back(PackedJob{J.scene, J.cams, J.n_views,
                                               (int)((static_cast<const char*>(J.feats) - c.base) / vb), J.out,
                                               J.beta});
                    }
                    r = uplift_packed(ctx, pj.data(), (int)pj.size(), c.base, c.key.dtype, c.key.d, c.key.width,
                                      c.key.height, c.group_bytes, st, &cstats[i]);
                    // out of device memory: smaller groups (the outputs are zeroed again)
                    while (r == LUDVIG_ERR_OOM && c.group_bytes > 64 * kMiB) {
                        reset_context(ctx);
                        c.group_bytes /= 2;
                        r = uplift_packed(ctx, pj.data(), (int)pj.size(), c.base, c.key.dtype, c.key.d, c.key.width,
                                          c.key.height, c.group_bytes, st, &cstats[i]);
                    }
                    c.groups = cstats[i].groups;
                }
                cms[i] = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (ctx) cws[i] = (int64_t)ctx->ws.device_bytes();
            } catch (...) {
                set_error("internal error in a packed class");
                r = LUDVIG_ERR_INTERNAL;
            }
            if (r != LUDVIG_OK)
                for (int32_t j : c.jobs) fail(j, r);
        }
        if (ctx) {
            cudaStreamSynchronize(st);   // the context returns to the pool once idle
            try {
                return_context(dev, ctx);
            } catch (...) {
            }
        }
    };
    auto worker = [&](int k) {
        cudaError_t e = cudaSetDevice(dev);
        cudaStream_t st = res.streams[(size_t)k];
        if (k == 0 && e == cudaSuccess) run_classes(st);
        std::unique_ptr<Arena> ws;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= (int)plain.size()) break;
            const int32_t j = plain[(size_t)i];
            try {   // nothing may escape a std::thread
                const ludvig_uplift_job& J = jobs[j];
                if (!ws) ws = take_workspace(dev);
                ludvig_status r = LUDVIG_ERR_CUDA;
                if (e == cudaSuccess) {
                    J.scene->ws.swap(*ws);   // lend the slot's workspace to the job
                    r = ludvig_uplift(J.scene, J.cams, J.n_views, J.width, J.height, J.feats, J.dtype, J.d,
                                      J.out, J.beta, st);
                    // complete it (a redo of what did not fit uses the lent workspace too)
                    if (r == LUDVIG_OK) r = ludvig_sync(J.scene);
                    J.scene->ws.swap(*ws);
                } else {
                    set_error("slot setup failed");
                }
                if (r != LUDVIG_OK) fail(j, r);
            } catch (...) {
                status[(size_t)j] = LUDVIG_ERR_INTERNAL;
            }
        }
        slot_err[(size_t)k] = cudaEventRecord(res.done[(size_t)k], st);
        // the workspace returns to the pool once its stream is idle
        const cudaError_t se = cudaStreamSynchronize(st);
        if (slot_err[(size_t)k] == cudaSuccess) slot_err[(size_t)k] = se;
        try {
            if (ws) return_workspace(dev, std::move(ws));
        } catch (...) {
        }
    };
    std::vector<std::thread> threads;
    for (int k = 1; k < nslots; ++k) {
        try {
            threads.emplace_back(worker, k);
        } catch (...) {
            // fewer threads still drain the shared counter; this slot's
            // stream only records its (empty) final event
            slot_err[(size_t)k] = cudaEventRecord(res.done[(size_t)k], res.streams[(size_t)k]);
        }
    }
    worker(0);
    for (std::thread& t : threads) t.join();
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        std::vector<ludvig_batch_class>& plan = last_plan();
        plan.clear();
        for (size_t i = 0; i < classes.size(); ++i) {
            const JobClass& c = classes[i];
            ludvig_batch_class b{};
            b.redone = cstats[i].redone;
            b.workspace_mb = (int32_t)(cws[i] >> 20);
            b.ms = cms[i];
            b.dtype = c.key.dtype;
            b.d = c.key.d;
            b.width = c.key.width;
            b.height = c.key.height;
            b.jobs = (int32_t)c.jobs.size();
            for (int32_t j : c.jobs) b.views += jobs[j].n_views;
            b.groups = c.groups;
            b.group_mb = (int32_t)(c.group_bytes >> 20);
            b.tuned = c.tuned ? 1 : 0;
            plan.push_back(b);
        }
        ludvig_batch_class single{};
        single.jobs = (int32_t)plain.size();
        for (int32_t j : plain) single.views += jobs[j].n_views;
        single.groups = -1;
        plan.push_back(single);
    }
    for (int k = 0; k < nslots; ++k) {
        LV_CUDA(slot_err[(size_t)k]);
        LV_CUDA(cudaStreamWaitEvent(caller, res.done[(size_t)k], 0));
    }
    if (job_status)
        for (int32_t j = 0; j < n_jobs; ++j) job_status[j] = (int32_t)status[(size_t)j];
    for (int32_t j = 0; j < n_jobs; ++j) {
        if (status[(size_t)j] != LUDVIG_OK) {
            set_error("job %d: %s", j, message[(size_t)j].c_str());
            return status[(size_t)j];
        }
    }
    return LUDVIG_OK;
}

extern "C" int32_t ludvig_batch_last_plan(ludvig_batch_class* out, int32_t cap) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const std::vector<ludvig_batch_class>& plan = last_plan();
    if (out)
        for (int32_t k = 0; k < cap && k < (int32_t)plan.size(); ++k) out[k] = plan[(size_t)k];
    return (int32_t)plan.size();
}

extern "C" ludvig_status ludvig_batch_release_workspaces(void) {
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    std::vector<std::unique_ptr<Arena>> idle;
    std::vector<ludvig_scene*> ctxs;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        idle.swap(pool()[dev]);
        ctxs.swap(ctx_pool()[dev]);
    }
    idle.clear();   // every pooled workspace's stream finished before it was pooled
    for (ludvig_scene* c : ctxs) ludvig_scene_destroy(c);
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_batch_forget_tuning(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_table().clear();
    return LUDVIG_OK;
}
