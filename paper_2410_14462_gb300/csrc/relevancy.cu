// Relevancy of uplifted CLIP features to text queries (appendix, "Relevancy
// scores", after LERF): with s_iq = f^_i . phi^_q and s_ik = f^_i . phi^_k
// (l2-normalised feature, query and canonical-phrase embeddings),
//   r_iq = min_k exp(T s_iq) / (exp(T s_iq) + exp(T s_ik))
//        = min_k 1 / (1 + exp(T (s_ik - s_iq))).
//
// The work streams the feature rows once and does m = queries + phrases dot
// products per row: memory-bound, so CUDA cores, not a GEMM.  One warp per row
// (grid-stride): lane l holds channels l, l + 32, ... of the row and of every
// embedding (normalised once per block into shared memory), the m partial
// dots and the squared norm are reduced across the warp, and lane q < queries
// writes r_iq.
#include <algorithm>

#include "common.cuh"

namespace ludvig {

namespace {

constexpr int kRelMaxM = 64;                   // queries + phrases
constexpr int kRelMaxSmemFloats = 48 * 1024;   // embeddings in shared memory (192 KB)

template <int M>
__global__ void __launch_bounds__(256) k_relevancy(const float* __restrict__ f, int64_t n, int d,
                                                   const float* __restrict__ phi, int nq, int m, float T,
                                                   float* __restrict__ r) {
    extern __shared__ float sphi[];   // [m][d], rows normalised
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // normalise the embeddings: warp w takes rows w, w + 8, ...
    for (int e = warp; e < m; e += 8) {
        float s = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float v = phi[(int64_t)e * d + c];
            s = fmaf(v, v, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float inv = s > 0.f ? 1.0f / sqrtf(s) : 0.f;
        for (int c = lane; c < d; c += 32) sphi[e * d + c] = phi[(int64_t)e * d + c] * inv;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < n; i += (int64_t)gridDim.x * 8) {
        const float* fi = f + i * d;
        float acc[M];
#pragma unroll
        for (int e = 0; e < M; ++e) acc[e] = 0.f;
        float nn = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float x = fi[c];
            nn = fmaf(x, x, nn);
#pragma unroll
            for (int e = 0; e < M; ++e)
                if (e < m) acc[e] = fmaf(x, sphi[e * d + c], acc[e]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
#pragma unroll
        for (int e = 0; e < M; ++e) {
            if (e < m) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
            }
        }
        const float inv = nn > 0.f ? 1.0f / sqrtf(nn) : 0.f;
        // lane q (< nq) takes query q: s_q and the phrases' s_k from the reduced dots
        for (int q0 = 0; q0 < nq; q0 += 32) {
            const int q = q0 + lane;
            float sq = 0.f;
#pragma unroll
            for (int e = 0; e < M; ++e)
                if (e == q) sq = acc[e];
            float best = 1.f;
#pragma unroll
            for (int e = 0; e < M; ++e) {
                if (e >= nq && e < m) {
                    const float v = 1.0f / (1.0f + expf(T * inv * (acc[e] - sq)));
                    best = fminf(best, v);
                }
            }
            if (q < nq) r[i * nq + q] = best;
        }
    }
}

template <int M>
ludvig_status launch_relevancy(const float* f, int64_t n, int d, const float* phi, int nq, int m, float T, float* r,
                               cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)m * d;
    static bool configured = false;
    if (!configured) {
        LV_CUDA(cudaFuncSetAttribute(k_relevancy<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float) * kRelMaxSmemFloats)));
        configured = true;
    }
    int dev = 0, sms = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = ceil_div(n, 8);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    k_relevancy<M><<<grid, 256, smem, st>>>(f, n, d, phi, nq, m, T, r);
    LV_LAUNCH();
    return LUDVIG_OK;
}

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_relevancy(const float* feats, int64_t n, int32_t d, const float* phi, int32_t n_queries,
                                          int32_t n_canon, float temperature, float* r, void* stream) {
    LV_ARG(n >= 0 && d >= 1, "bad sizes");
    LV_ARG(n_queries >= 1 && n_canon >= 1 && n_queries + n_canon <= kRelMaxM,
           "need 1 <= queries, 1 <= phrases, queries + phrases <= %d", kRelMaxM);
    LV_ARG((int64_t)(n_queries + n_canon) * d <= kRelMaxSmemFloats, "(queries + phrases) x d must be <= %d",
           kRelMaxSmemFloats);
    LV_ARG(temperature > 0.f, "temperature must be positive");
    if (n == 0) return LUDVIG_OK;
    LV_ARG(feats != nullptr && phi != nullptr && r != nullptr, "NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StageScope scope(LUDVIG_STAGE_RELEVANCY, st);
    const int m = n_queries + n_canon;
    if (m <= 8) return launch_relevancy<8>(feats, n, d, phi, n_queries, m, temperature, r, st);
    if (m <= 16) return launch_relevancy<16>(feats, n, d, phi, n_queries, m, temperature, r, st);
    if (m <= 32) return launch_relevancy<32>(feats, n, d, phi, n_queries, m, temperature, r, st);
    return launch_relevancy<64>(feats, n, d, phi, n_queries, m, temperature, r, st);
}
