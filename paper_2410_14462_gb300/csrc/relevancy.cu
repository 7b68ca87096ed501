// Relevancy of uplifted CLIP features to text queries (appendix, "Relevancy
// scores", after LERF): with s_iq = f^_i . phi^_q and s_ik = f^_i . phi^_k
// (l2-normalised feature, query and canonical-phrase embeddings),
//   r_iq = min_k exp(T s_iq) / (exp(T s_iq) + exp(T s_ik))
//        = min_k 1 / (1 + exp(T (s_ik - s_iq))).
//
// The work streams the feature rows once and does m = queries + phrases dot
// products of length d per row: a skinny product S = F Phi^T (n x d times
// d x m) with its epilogue.  A CTA takes 128 rows and computes their 128 x M
// block of S on CUDA cores with register tiles: thread (row group, query
// group) holds 4 rows x M/8 queries, and per channel reads 4 features of its
// rows (one 16-byte load of the chunk staged transposed in shared memory) and
// M/8 normalised embedding values (one or two 16-byte loads, the same for the
// whole warp), for 4 M/8 fused multiply-adds.  Channels are
// staged 32 at a time, the next chunk's global loads in flight while the
// current one is used.  The feature norms are summed from the staged chunks
// (two threads per row, each over half of every chunk).  Each dot product is
// one fmaf chain over the channels in order.  The epilogue writes the block of S to shared memory and takes
// the minimum over the phrases for every (row, query).
#include <algorithm>

#include "common.cuh"

namespace ludvig {

namespace {

constexpr int kRelMaxM = 64;                   // queries + phrases
constexpr int kRelMaxSmemFloats = 40 * 1024;   // normalised embeddings in shared memory (160 KB)
constexpr int kRelRows = 128;                  // rows per CTA
constexpr int kRelPitch = kRelRows + 4;        // transposed chunk: [channel][row], 16-byte aligned rows

template <int M>
__global__ void __launch_bounds__(256, M == 32 ? 3 : 2) k_relevancy(const float* __restrict__ f, int64_t n, int d,
                                                   const float* __restrict__ phi, int nq, int m, float T,
                                                   float* __restrict__ r) {
    constexpr int QPT = M / 8;                 // queries per thread
    constexpr int kStage = 32 * kRelPitch > kRelRows * (M + 1) ? 32 * kRelPitch : kRelRows * (M + 1);
    extern __shared__ __align__(16) float smem[];
    float* sphi = smem;                                        // [d][M], normalised, zero past m
    float* As = sphi + (size_t)d * M;                          // [32][kRelPitch]
    float* Cs = As;                                            // epilogue: [kRelRows][M + 1], in As's place
    float* nrm = As + kStage;                                  // [kRelRows] squared norms
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
    // query group (QPT queries, the same for a warp: its embedding loads are
    // broadcasts) and row group (4 rows; a warp's 32 groups read one 512-byte
    // run of the staged chunk)
    const int qg = tid >> 5, rg = tid & 31;
    const int64_t base = (int64_t)blockIdx.x * kRelRows;
    // staging: element t + 256 j of a chunk is row (t + 256 j) / 32, channel lane
    const int64_t stride8 = 8 * (int64_t)d;                       // 8 rows
    const float* frow = f + (base + (tid >> 5)) * (int64_t)d + lane;   // row warp, channel lane
    const int64_t rows_left = n - base - (tid >> 5);                   // rows warp + 8 jj exist for 8 jj < this
    auto load_chunk = [&](int c0, float* v) {
        const bool cin = c0 + lane < d;
        const float* p = frow + c0;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) v[jj] = (cin && 8 * jj < rows_left) ? p[jj * stride8] : 0.f;
    };
    float v[16];
    load_chunk(0, v);
    float acc[4][QPT];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < QPT; ++b) acc[a][b] = 0.f;
    float nn = 0.f;   // row (tid % 128)'s squared norm over half of each chunk's channels
    for (int c0 = 0; c0 < d; c0 += 32) {
        __syncthreads();   // the previous chunk is consumed (and sphi is written, first time)
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) As[lane * kRelPitch + (tid >> 5) + 8 * jj] = v[jj];
        __syncthreads();
        if (c0 + 32 < d) load_chunk(c0 + 32, v);   // in flight during this chunk
        const int cw = min(32, d - c0);
        {
            // this thread's half of row (tid % 128)'s channels in the chunk
            const int h0 = 16 * (tid >> 7), h1 = min(cw, h0 + 16);
            for (int cc = h0; cc < h1; ++cc) {
                const float x = As[cc * kRelPitch + (tid & (kRelRows - 1))];
                nn = fmaf(x, x, nn);
            }
        }
        auto step = [&](int cc) {
            const float4 a4 = *reinterpret_cast<const float4*>(&As[cc * kRelPitch + 4 * rg]);
            const float* pr = sphi + (size_t)(c0 + cc) * M + QPT * qg;
            float bq[QPT];
            if constexpr (QPT >= 4) {
#pragma unroll
                for (int b = 0; b < QPT; b += 4) {
                    const float4 p4 = *reinterpret_cast<const float4*>(pr + b);
                    bq[b] = p4.x;
                    bq[b + 1] = p4.y;
                    bq[b + 2] = p4.z;
                    bq[b + 3] = p4.w;
                }
            } else {
#pragma unroll
                for (int b = 0; b < QPT; ++b) bq[b] = pr[b];
            }
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < QPT; ++b) acc[a][b] = fmaf(av[a], bq[b], acc[a][b]);
        };
        if (cw == 32) {
#pragma unroll 8
            for (int cc = 0; cc < 32; ++cc) step(cc);
        } else {
            for (int cc = 0; cc < cw; ++cc) step(cc);
        }
    }
    __syncthreads();   // As is free: the block of S goes to Cs
    if (tid < kRelRows) nrm[tid] = nn;   // first halves; the second halves are added below
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < QPT; ++b) Cs[(4 * rg + a) * (M + 1) + QPT * qg + b] = acc[a][b];
    __syncthreads();
    if (tid >= kRelRows) nrm[tid - kRelRows] += nn;
    __syncthreads();
    const int rows = n - base < kRelRows ? (int)(n - base) : kRelRows;
    for (int o = tid; o < rows * nq; o += 256) {
        const int row = o / nq, q = o - row * nq;
        const float* cr = Cs + row * (M + 1);
        const float nsq = nrm[row];
        const float inv = nsq > 0.f ? 1.0f / sqrtf(nsq) : 0.f;
        float best = 1.f;
        for (int e = nq; e < m; ++e) best = fminf(best, 1.0f / (1.0f + expf(T * inv * (cr[e] - cr[q]))));
        r[(base + row) * nq + q] = best;
    }
}

template <int M>
size_t relevancy_smem(int d) {
    // embeddings, then the chunk [32][kRelPitch] (or the epilogue's [128][M + 1]), then the norms
    const size_t stage = std::max<size_t>((size_t)32 * kRelPitch, (size_t)kRelRows * (M + 1));
    return sizeof(float) * ((size_t)d * M + stage + kRelRows);
}

template <int M>
ludvig_status launch_relevancy(const float* f, int64_t n, int d, const float* phi, int nq, int m, float T, float* r,
                               cudaStream_t st) {
    const size_t smem = relevancy_smem<M>(d);
    // set once per process; a function-local static is initialised by one thread
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_relevancy<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)relevancy_smem<M>(kRelMaxSmemFloats / M));
    LV_CUDA(configured);
    const unsigned grid = (unsigned)ceil_div(n, kRelRows);
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
