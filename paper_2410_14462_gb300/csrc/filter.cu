// Gaussian filtering by importance (Sec. 3.2, "Gaussian filtering"): beta_i,
// the sum of the Gaussian's rendering weights over the training views (the
// uplift's normaliser), estimates its importance, and the method keeps the
// more important half of the Gaussians (Sec. 4 keeps half).
//
//   ludvig_beta_select   indices of the `keep` largest beta_i (ties to the
//                        lower index), ascending: one stable LSD radix sort of
//                        (descending-beta key, index), a mark of the first
//                        `keep` entries, and a compaction by exclusive scan;
//   ludvig_scene_subset  a new scene holding the selected Gaussians, gathered
//                        from the source scene's device arrays (the
//                        precomputed 3D covariances are copied, so the new
//                        scene projects exactly as the old one did).
#include "common.cuh"

namespace ludvig {

namespace {

// Ascending key = descending beta: for beta > 0 the IEEE bits order like the
// values, so their complement orders them downwards; beta <= 0, NaN and the
// padding take the largest key.  The sort is stable, so equal keys stay in
// index order.
__global__ void k_beta_keys(const float* __restrict__ beta, int64_t n, int64_t npad, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    uint32_t k = 0xffffffffu;
    if (i < n) {
        const float b = beta[i];
        if (b > 0.f) k = ~__float_as_uint(b);
    }
    keys[i] = k;
    vals[i] = (uint32_t)i;
}

__global__ void k_mark_kept(const uint32_t* __restrict__ vals, int64_t keep, uint32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < keep) flag[vals[i]] = 1u;
}

__global__ void k_compact(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos, int64_t n,
                          int32_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (int32_t)i;
}

// dst Gaussian j = src Gaussian idx[j]; an index outside [0, n) sets *bad and
// leaves the entry zero.
__global__ void k_gather_scene(const float4* __restrict__ geo, const float4* __restrict__ cov_a,
                               const float2* __restrict__ cov_b, const float* __restrict__ means,
                               const int32_t* __restrict__ idx, int64_t m, int64_t n, float4* __restrict__ geo2,
                               float4* __restrict__ cov_a2, float2* __restrict__ cov_b2,
                               float* __restrict__ means2, int* __restrict__ bad) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t g = idx[j];
    if (g < 0 || (int64_t)g >= n) {
        atomicExch(bad, 1);
        geo2[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        cov_a2[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        cov_b2[j] = make_float2(0.f, 0.f);
        means2[3 * j] = means2[3 * j + 1] = means2[3 * j + 2] = 0.f;
        return;
    }
    geo2[j] = geo[g];
    cov_a2[j] = cov_a[g];
    cov_b2[j] = cov_b[g];
    means2[3 * j] = means[3 * (int64_t)g];
    means2[3 * j + 1] = means[3 * (int64_t)g + 1];
    means2[3 * j + 2] = means[3 * (int64_t)g + 2];
}

unsigned blocks_for(int64_t work) { return (unsigned)ceil_div(std::max<int64_t>(work, 1), 256); }

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_beta_select(ludvig_scene_t scene, const float* beta, int64_t keep, int32_t* kept,
                                            void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    const int64_t n = scene->n;
    LV_ARG(keep >= 0 && keep <= n, "keep must be in [0, n]");
    if (keep == 0) return LUDVIG_OK;
    LV_ARG(beta != nullptr && kept != nullptr, "NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena& ws = scene->ws;
    const int64_t npad = round_up(n, kRadixTile);
    uint32_t *keys, *vals, *keys2, *vals2, *flag;
    LV_TRY(ws.get("filter.keys", (size_t)npad, &keys));
    LV_TRY(ws.get("filter.vals", (size_t)npad, &vals));
    LV_TRY(ws.get("filter.keys2", (size_t)npad, &keys2));
    LV_TRY(ws.get("filter.vals2", (size_t)npad, &vals2));
    LV_TRY(ws.get("filter.flag", (size_t)n, &flag));
    StageScope scope(LUDVIG_STAGE_FILTER, st);
    k_beta_keys<<<blocks_for(npad), 256, 0, st>>>(beta, n, npad, keys, vals);
    LV_LAUNCH();
    uint32_t *sk = keys, *sv = vals;
    LV_TRY(radix_sort_pairs(&sk, &sv, keys2, vals2, 1, npad, 32, ws, st));
    LV_CUDA(cudaMemsetAsync(flag, 0, sizeof(uint32_t) * (size_t)n, st));
    k_mark_kept<<<blocks_for(keep), 256, 0, st>>>(sv, keep, flag);
    LV_LAUNCH();
    // positions of the kept Gaussians: the sorted keys are no longer needed
    uint32_t* pos = sk == keys ? keys2 : keys;
    LV_TRY(scan_exclusive_u32(flag, pos, n, nullptr, ws, st));
    k_compact<<<blocks_for(n), 256, 0, st>>>(flag, pos, n, kept);
    LV_LAUNCH();
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_scene_subset(ludvig_scene_t scene, const int32_t* idx, int64_t m, void* stream,
                                             ludvig_scene_t* out) {
    LV_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(m >= 0 && m < ((int64_t)1 << 31), "m must be in [0, 2^31)");
    LV_ARG(m == 0 || idx != nullptr, "idx is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ludvig_scene* s = new (std::nothrow) ludvig_scene();
    LV_ARG(s != nullptr, "host allocation failed");
    s->n = m;
    LV_CUDA(cudaGetDevice(&s->device));
    if (m > 0) {
        const size_t mm = (size_t)m;
        if (cudaMalloc(&s->geo, mm * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&s->cov_a, mm * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&s->cov_b, mm * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&s->means, mm * 3 * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            ludvig_scene_destroy(s);
            set_error("scene allocation failed for n=%lld", (long long)m);
            return LUDVIG_ERR_OOM;
        }
        int* bad = nullptr;
        void* hb = nullptr;
        ludvig_status r = scene->ws.get("subset.bad", 1, &bad);
        if (r == LUDVIG_OK) r = scene->ws.pinned("subset.bad_h", 16, &hb);
        if (r != LUDVIG_OK) {
            ludvig_scene_destroy(s);
            return r;
        }
        if (cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) {
            ludvig_scene_destroy(s);
            set_error("cudaMemsetAsync failed");
            return LUDVIG_ERR_CUDA;
        }
        k_gather_scene<<<blocks_for(m), 256, 0, st>>>(scene->geo, scene->cov_a, scene->cov_b, scene->means, idx, m,
                                                      scene->n, s->geo, s->cov_a, s->cov_b, s->means, bad);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            ludvig_scene_destroy(s);
            set_error("scene subset: CUDA failure");
            return LUDVIG_ERR_CUDA;
        }
        count_launch();
        if (*static_cast<int*>(hb) != 0) {
            ludvig_scene_destroy(s);
            set_error("scene subset: an index lies outside [0, %lld)", (long long)scene->n);
            return LUDVIG_ERR_ARG;
        }
    }
    *out = s;
    return LUDVIG_OK;
}
