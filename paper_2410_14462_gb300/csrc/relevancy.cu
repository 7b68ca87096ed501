// Relevancy of uplifted CLIP features to text queries (appendix, "Relevancy
// scores", after LERF): with s_iq = f^_i . phi^_q and s_ik = f^_i . phi^_k
// (l2-normalised feature, query and canonical-phrase embeddings),
//   r_iq = min_k exp(T s_iq) / (exp(T s_iq) + exp(T s_ik))
//        = min_k 1 / (1 + exp(T (s_ik - s_iq))).
//
// The work streams the feature rows once and does m = queries + phrases dot
// products per row: memory-bound, so CUDA cores, not a GEMM.  One thread per
// row keeps the row's m dots in registers (no cross-lane reductions): a warp
// takes 32 rows and walks their channels 32 at a time, staging each 32 x 32
// slab through shared memory (coalesced 128-byte row loads in, one padded row
// per thread out); the embeddings sit normalised and transposed in shared
// memory ([channel][M]), so every thread reads the same values (broadcast).
#include <algorithm>

#include "common.cuh"

namespace ludvig {

namespace {

constexpr int kRelMaxM = 64;                   // queries + phrases
constexpr int kRelMaxSmemFloats = 40 * 1024;   // transposed embeddings in shared memory (160 KB)

template <int M>
__global__ void __launch_bounds__(256) k_relevancy(const float* __restrict__ f, int64_t n, int d,
                                                   const float* __restrict__ phi, int nq, int m, float T,
                                                   float* __restrict__ r) {
    extern __shared__ float smem[];
    float* sphi = smem;                            // [d][M], rows of phi normalised, zero past m
    float (*tile)[32 * 33] = reinterpret_cast<float (*)[32 * 33]>(smem + (size_t)d * M);   // per warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = warp; e < M; e += 8) {
        float s = 0.f;
        if (e < m)
            for (int c = lane; c < d; c += 32) {
                const float v = phi[(int64_t)e * d + c];
                s = fmaf(v, v, s);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float inv = s > 0.f ? 1.0f / sqrtf(s) : 0.f;
        for (int c = lane; c < d; c += 32) sphi[c * M + e] = e < m ? phi[(int64_t)e * d + c] * inv : 0.f;
    }
    __syncthreads();
    float* t = tile[warp];
    for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 32; base < n; base += (int64_t)gridDim.x * 256) {
        const int64_t i = base + lane;
        const int rows = (int)(n - base < 32 ? n - base : 32);
        float acc[M];
#pragma unroll
        for (int e = 0; e < M; ++e) acc[e] = 0.f;
        float nn = 0.f;
        for (int c0 = 0; c0 < d; c0 += 32) {
            // slab: rows base .. base + 31, channels c0 .. c0 + 31 (lane = channel)
            const int c = c0 + lane;
            float v[32];   // all 32 row loads in flight before the stores
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) v[rr] = (rr < rows && c < d) ? f[(base + rr) * d + c] : 0.f;
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) t[rr * 33 + lane] = v[rr];
            __syncwarp();
            const int cw = min(32, d - c0);
            for (int cc = 0; cc < cw; ++cc) {
                const float x = t[lane * 33 + cc];
                nn = fmaf(x, x, nn);
                const float4* p = reinterpret_cast<const float4*>(sphi + (size_t)(c0 + cc) * M);
#pragma unroll
                for (int e4 = 0; e4 < M / 4; ++e4) {
                    const float4 ph = p[e4];
                    acc[4 * e4] = fmaf(x, ph.x, acc[4 * e4]);
                    acc[4 * e4 + 1] = fmaf(x, ph.y, acc[4 * e4 + 1]);
                    acc[4 * e4 + 2] = fmaf(x, ph.z, acc[4 * e4 + 2]);
                    acc[4 * e4 + 3] = fmaf(x, ph.w, acc[4 * e4 + 3]);
                }
            }
            __syncwarp();
        }
        if (lane >= rows) continue;
        const float inv = nn > 0.f ? 1.0f / sqrtf(nn) : 0.f;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            if (q < nq) {
                float best = 1.f;
#pragma unroll
                for (int e = 0; e < M; ++e)
                    if (e >= nq && e < m) best = fminf(best, 1.0f / (1.0f + expf(T * inv * (acc[e] - acc[q]))));
                r[i * nq + q] = best;
            }
        }
    }
}

template <int M>
size_t relevancy_smem(int d) {
    return sizeof(float) * ((size_t)d * M + 8 * 32 * 33);
}

template <int M>
ludvig_status launch_relevancy(const float* f, int64_t n, int d, const float* phi, int nq, int m, float T, float* r,
                               cudaStream_t st) {
    const size_t smem = relevancy_smem<M>(d);
    // set once per process; a function-local static is initialised by one thread
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_relevancy<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)relevancy_smem<M>(kRelMaxSmemFloats / M));
    LV_CUDA(configured);
    int dev = 0, sms = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = ceil_div(n, 256);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 4));
    k_relevancy<M><<<grid, 256, smem, st>>>(f, n, d, phi, nq, m, T, r);
    LV_LAUNCH();
    return LUDVIG_OK;
}

int relevancy_bucket(int m) { return m <= 8 ? 8 : m <= 16 ? 16 : m <= 32 ? 32 : 64; }

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_relevancy(const float* feats, int64_t n, int32_t d, const float* phi, int32_t n_queries,
                                          int32_t n_canon, float temperature, float* r, void* stream) {
    LV_ARG(n >= 0 && d >= 1, "bad sizes");
    LV_ARG(n_queries >= 1 && n_canon >= 1 && n_queries + n_canon <= kRelMaxM,
           "need 1 <= queries, 1 <= phrases, queries + phrases <= %d", kRelMaxM);
    LV_ARG((int64_t)relevancy_bucket(n_queries + n_canon) * d <= kRelMaxSmemFloats,
           "(queries + phrases, rounded up to 8, 16, 32 or 64) x d must be <= %d", kRelMaxSmemFloats);
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
