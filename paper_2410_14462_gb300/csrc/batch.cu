// Batched uplift: many independent uplifts (Sec. 3.2, Eq. 5, one per job) of
// uneven size on one GPU.  The paper runs one uplift at a time; this is the
// executor that keeps the GPU busy across jobs.
//
// Each job is exactly a ludvig_uplift call.  An uplift waits for its own
// stream a few times (pair counts size the sort and the weight rows), so jobs
// overlap only if their host sides run concurrently: `slots` host threads (the
// calling thread is one of them) each own a non-blocking stream and take jobs
// from a shared counter in order of decreasing estimated cost (the longest
// jobs start first and the short ones fill the tail).  Every slot stream
// waits for an event recorded on the caller's stream before its first job,
// and the caller's stream waits for every slot's final event, so the batch is
// ordered on `stream` like one call.
//
// Workspaces: a scene's workspace grows to the largest uplift it has run, so
// many resident scenes would each hold one.  Instead every slot lends its own
// pooled workspace to the job it runs (swapped into the scene for the call
// and back out after it), and the pool keeps the slot workspaces for the next
// batch: device memory scales with the slots, not with the jobs.  A slot's
// workspace is used on its slot's stream only, and each slot waits for its
// stream before its workspace goes back to the pool.
#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace ludvig {

namespace {

double job_cost(const ludvig_uplift_job& j) {
    // pixels x Gaussians x channels, with a floor on the channels for the
    // D-independent walk
    return (double)ludvig_scene_size(j.scene) * (double)j.n_views * (double)j.width * (double)j.height *
           (double)std::max<int32_t>(j.d, 32);
}

// Idle slot workspaces per device.  Never destroyed: no CUDA call may run
// from a static destructor at exit; process exit returns the memory.
std::mutex g_pool_mu;
using Pool = std::unordered_map<int, std::vector<std::unique_ptr<Arena>>>;
Pool& pool() {
    static Pool* p = new Pool();
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

    std::vector<int32_t> order((size_t)n_jobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return job_cost(jobs[a]) > job_cost(jobs[b]); });

    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const int nslots = std::min<int>(slots, n_jobs);
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

    std::atomic<int32_t> next{0};
    std::vector<ludvig_status> status((size_t)n_jobs, LUDVIG_OK);
    std::vector<std::string> message((size_t)n_jobs);
    std::vector<cudaError_t> slot_err((size_t)nslots, cudaSuccess);
    auto worker = [&](int k) {
        cudaError_t e = cudaSetDevice(dev);
        cudaStream_t st = res.streams[(size_t)k];
        std::unique_ptr<Arena> ws;
        try {
            ws = take_workspace(dev);
        } catch (...) {
            e = cudaErrorMemoryAllocation;
        }
        for (;;) {
            const int32_t i = next.fetch_add(1);
            if (i >= n_jobs) break;
            const int32_t j = order[(size_t)i];
            const ludvig_uplift_job& J = jobs[j];
            try {   // nothing may escape a std::thread
                ludvig_status r = LUDVIG_ERR_CUDA;
                if (e == cudaSuccess) {
                    J.scene->ws.swap(*ws);   // lend the slot's workspace to the job
                    r = ludvig_uplift(J.scene, J.cams, J.n_views, J.width, J.height, J.feats, J.dtype, J.d,
                                      J.out, J.beta, st);
                    // complete it (a redo of what did not fit uses the lent workspace too)
                    if (r == LUDVIG_OK) r = ludvig_sync(J.scene);
                    J.scene->ws.swap(*ws);
                }
                status[(size_t)j] = r;
                if (r != LUDVIG_OK)
                    message[(size_t)j] = e == cudaSuccess ? ludvig_last_error() : "slot setup failed";
            } catch (...) {
                status[(size_t)j] = LUDVIG_ERR_INTERNAL;
            }
        }
        slot_err[(size_t)k] = cudaEventRecord(res.done[(size_t)k], st);
        // the workspace returns to the pool once its stream has finished with it
        const cudaError_t se = cudaStreamSynchronize(st);
        if (slot_err[(size_t)k] == cudaSuccess) slot_err[(size_t)k] = se;
        if (ws) {
            try {
                return_workspace(dev, std::move(ws));
            } catch (...) {
            }
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

extern "C" ludvig_status ludvig_batch_release_workspaces(void) {
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    std::vector<std::unique_ptr<Arena>> idle;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        idle.swap(pool()[dev]);
    }
    idle.clear();   // every pooled workspace's stream finished before it was pooled
    return LUDVIG_OK;
}
