// Tensor-core aggregation for float32 features (the plain form of the uplift,
// Sec. 3.2 Eq. 3) at float32-level accuracy.
//
// Both operands are split into two bfloat16 terms, w = W1 + W2 and
// F = F1 + F2 (16 significant bits each), and the product is formed from
// F1 W1 + F1 W2 + F2 W1 on the tensor cores with float32 accumulation (the
// dropped F2 W2 term and the residuals are below 2^-16 relative); beta sums the
// same W1 + W2.
//
// Layout per (view, tile) item, one persistent CTA of 8 warps per SM:
//   * compositing as in the other paths (float32 rules, 8x4-pixel warp
//     blocks), with the next batch's records prefetched while the current
//     batch is composited;
//   * Gaussians with a non-zero weight in the tile become rows of two
//     128 x 256 bfloat16 W tiles (W1, W2) in shared memory, K-major with the
//     128-byte swizzle: the MMA's B operand (N = 128 Gaussians, K = 256 pixels);
//   * per 128-channel block the tile's features are read with coalesced loads
//     (lane = channel), split, and written to tensor memory as the transposed
//     A operand (M = 128 channels, K = 256 pixels; F1 and F2 at columns 0 and
//     128);
//   * tcgen05.mma (kind::f16, M = 128, N = 128, K = 16, A from tensor memory)
//     accumulates D = F^T W into columns 256..383;
//   * the accumulator is read back with lanes = channels, so the additions into
//     num[gid, c] are coalesced: 32 consecutive channels per warp and Gaussian.
// Every mbarrier wait is bounded (LUDVIG_ERR_TIMEOUT on expiry).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "spec.cuh"
#include "tc_ptx.cuh"

namespace ludvig {

namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kRows = 128;                       // Gaussians per W tile (MMA N)
constexpr int kBatch = 32;
constexpr uint32_t kWTermBytes = kRows * 256 * 2;   // 64 KB per bfloat16 term
constexpr uint32_t kColF1 = 0, kColF2 = 128, kColD = 256;

struct Smem32 {
    uint8_t W[2][kWTermBytes];                   // W1, W2 (1024-aligned)
    uint64_t mma_done;
    float4 ra[2][kBatch];
    float2 rb[2][kBatch];
    uint32_t gid[2][kBatch];
    uint32_t row_gid[kRows];
    float row_den[kRows];
    float denpart[8][kBatch];
    uint32_t rowmask[2];
    uint32_t tmem_base;
    int item;
    int abort_flag;
};

constexpr size_t kSmemBytes = sizeof(Smem32) + 1024;

// kind::f16, D float32, A and B bfloat16, both K-major, N = 128, M = 128.
constexpr uint32_t kIdescTS = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t w_off(int r, int k) {
    const int ka = k >> 6, kk = k & 63;
    return (uint32_t)(ka * (kRows * 128) + r * 128 + ((((kk >> 3) ^ (r & 7))) << 4) + ((kk & 7) << 1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct T32Args {
    const float4* rec_a;
    const float2* rec_b;
    int64_t n;
    const uint2* ranges;
    const uint32_t* list;
    int ntiles, TX, width, height, d, nitems;
    const float* feats;   // chunk's first view, [nv, H, W, d]
    float* num;
    float* den;
    int* counter;
    int* status;
};

__device__ void fail(Smem32& S, int* status) {
    S.abort_flag = 1;
    atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
}

// MMA + read-back of the W tile rows [0, nrows) for every 128-channel block.
__device__ __noinline__ void flush32(Smem32& S, const T32Args& a, int nrows, uint32_t& mma_phase, int v, int tx, int ty) {
    fence_proxy_async();   // W tiles written with generic stores, read by the tensor core
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, h = warp >> 2;
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const int d = a.d;
    const float* fv = a.feats + (int64_t)v * a.height * a.width * d;
    const int nblk = (d + 127) / 128;
    for (int cb = 0; cb < nblk; ++cb) {
        // features of 128 channels x 256 pixels -> F1^T, F2^T in tensor memory
        const int c = 128 * cb + 32 * q + lane;
        const bool cvalid = c < d;
#pragma unroll 1
        for (int chunk = 0; chunk < 2; ++chunk) {
            const int p0 = 128 * h + 64 * chunk;
            uint32_t r1[32], r2[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float x[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int p = p0 + 2 * i + e;
                    const int px = tx * kTile + (p & 15), py = ty * kTile + (p >> 4);
                    x[e] = (cvalid && px < a.width && py < a.height) ? __ldg(fv + ((int64_t)py * a.width + px) * d + c)
                                                                      : 0.f;
                }
                const __nv_bfloat16 a1 = __float2bfloat16_rn(x[0]), b1 = __float2bfloat16_rn(x[1]);
                const __nv_bfloat16 a2 = __float2bfloat16_rn(x[0] - __bfloat162float(a1));
                const __nv_bfloat16 b2 = __float2bfloat16_rn(x[1] - __bfloat162float(b1));
                r1[i] = pack_bf16x2(a1, b1);
                r2[i] = pack_bf16x2(a2, b2);
            }
            tmem_st32(tmem + lane_off + kColF1 + p0 / 2, r1);
            tmem_st32(tmem + lane_off + kColF2 + p0 / 2, r2);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t w1 = saddr(S.W[0]), w2 = saddr(S.W[1]);
#pragma unroll
            for (int ks = 0; ks < 16; ++ks) {
                const uint32_t koff = (ks >> 2) * (kRows * 128) + (ks & 3) * 32;
                const uint64_t d1 = sw128_desc(w1 + koff, 16, 1024);
                const uint64_t d2 = sw128_desc(w2 + koff, 16, 1024);
                mma_bf16_ts(tmem + kColD, tmem + kColF1 + ks * 8, d1, kIdescTS, ks > 0 ? 1u : 0u);
                mma_bf16_ts(tmem + kColD, tmem + kColF1 + ks * 8, d2, kIdescTS, 1u);
                mma_bf16_ts(tmem + kColD, tmem + kColF2 + ks * 8, d1, kIdescTS, 1u);
            }
            mma_commit(&S.mma_done);
        }
        if (!mbar_wait(&S.mma_done, mma_phase)) fail(S, a.status);
        mma_phase ^= 1u;
        __syncthreads();
        if (S.abort_flag) return;
        tc_fence_after();
        // D[channel, slot]: warps (q, h) read lanes 32q.., slots 64h..64h+63
#pragma unroll 1
        for (int u = 0; u < 2; ++u) {
            float val[32];
            const int s0 = 64 * h + 32 * u;
            tmem_ld32(tmem + lane_off + kColD + s0, val);
            if (cvalid) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (s0 + j < nrows) red_add_f32(a.num + (int64_t)S.row_gid[s0 + j] * d + c, val[j]);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (tid < nrows) atomicAdd(a.den + S.row_gid[tid], S.row_den[tid]);
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) k_composite_tc32(T32Args a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    Smem32& S = *reinterpret_cast<Smem32*>(smem_raw + pad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    if (tid == 0) {
        mbar_init(&S.mma_done, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&S.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t mma_phase = 0;

    const int bx = (warp & 1) * 8, by = (warp >> 1) * 4;
    const int lx = bx + (lane & 7), ly = by + (lane >> 3);
    const int pix = ly * kTile + lx;
    for (;;) {
        if (tid == 0) S.item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = S.item;
        if (item >= a.nitems || S.abort_flag) break;
        const int v = item / a.ntiles, tile = item - v * a.ntiles;
        const int tx = tile % a.TX, ty = tile / a.TX;
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        const bool inside = px < a.width && py < a.height;
        const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
        const float bxa = (float)(tx * kTile + bx) + 0.5f, bya = (float)(ty * kTile + by) + 0.5f;
        const uint2 range = a.ranges[item];
        const float4* rec_a = a.rec_a + (int64_t)v * a.n;
        const float2* rec_b = a.rec_b + (int64_t)v * a.n;
        // records of the first batch
        if (tid < kBatch && range.x + tid < range.y) {
            const uint32_t g = a.list[range.x + tid];
            S.gid[0][tid] = g;
            S.ra[0][tid] = rec_a[g];
            S.rb[0][tid] = rec_b[g];
        }
        if (tid == 0) {
            S.rowmask[0] = 0u;
            S.rowmask[1] = 0u;
        }
        __syncthreads();
        float T = 1.0f;
        bool done = !inside;
        int nrows = 0;
        int buf = 0;
        for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch, buf ^= 1) {
            if (__syncthreads_count(!done) == 0) break;
            // make room for up to 32 new rows before any weight is live in registers
            if (nrows + kBatch > kRows) {
                flush32(S, a, nrows, mma_phase, v, tx, ty);
                nrows = 0;
                if (S.abort_flag) break;
            }
            const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
            // prefetch the next batch's records (stored at the end of this batch)
            const uint32_t nb0 = b0 + kBatch;
            const bool pf = tid < kBatch && nb0 + tid < range.y;
            uint32_t pg = 0;
            float4 pra;
            float2 prb;
            if (pf) {
                pg = a.list[nb0 + tid];
                pra = rec_a[pg];
                prb = rec_b[pg];
            }
            uint32_t rel;
            {
                bool rr = false;
                if (lane < cnt) {
                    const float4 ra = S.ra[buf][lane];
                    const float2 rb = S.rb[buf][lane];
                    rr = reaches_rect(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, bxa, bxa + 7.0f, bya, bya + 3.0f);
                }
                rel = __ballot_sync(0xffffffffu, rr);
                if (!__any_sync(0xffffffffu, !done)) rel = 0u;
            }
            float w[kBatch];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                w[j] = 0.f;
                if (((rel >> j) & 1u) && !done) {
                    const float4 ra = S.ra[buf][j];
                    const float2 rb = S.rb[buf][j];
                    const float al = alpha_at(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, pxf, pyf);
                    if (al > 0.f) {
                        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
                        if (Tn < kTransMin) {
                            done = true;
                        } else {
                            w[j] = __fmul_rn(al, T);
                            T = Tn;
                        }
                    }
                }
            }
            uint32_t mine = 0u;
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const uint32_t m = __ballot_sync(0xffffffffu, w[j] != 0.f);
                float sj = 0.f;
                if (m) {
                    mine |= 1u << j;
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(w[j]);
                    sj = __bfloat162float(h1) + __bfloat162float(__float2bfloat16_rn(w[j] - __bfloat162float(h1)));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
                }
                if (lane == 0) S.denpart[warp][j] = sj;
            }
            if (lane == 0 && mine) atomicOr(&S.rowmask[buf], mine);
            if (tid == 0) S.rowmask[buf ^ 1] = 0u;
            __syncthreads();
            const uint32_t rowmask = S.rowmask[buf];
            const int nnew = __popc(rowmask);
            if (nnew) {
#pragma unroll
                for (int j = 0; j < kBatch; ++j) {
                    if ((rowmask >> j) & 1u) {
                        const int slot = nrows + __popc(rowmask & ((1u << j) - 1u));
                        const __nv_bfloat16 h1 = __float2bfloat16_rn(w[j]);
                        const __nv_bfloat16 h2 = __float2bfloat16_rn(w[j] - __bfloat162float(h1));
                        const uint32_t o = w_off(slot, pix);
                        *reinterpret_cast<__nv_bfloat16*>(S.W[0] + o) = h1;
                        *reinterpret_cast<__nv_bfloat16*>(S.W[1] + o) = h2;
                    }
                }
                if (tid < kBatch && ((rowmask >> tid) & 1u)) {
                    const int slot = nrows + __popc(rowmask & lt_mask);
                    float s = 0.f;
#pragma unroll
                    for (int wi = 0; wi < 8; ++wi) s += S.denpart[wi][tid];
                    S.row_gid[slot] = S.gid[buf][tid];
                    S.row_den[slot] = s;
                }
                nrows += nnew;
            }
            if (pf) {
                S.gid[buf ^ 1][tid] = pg;
                S.ra[buf ^ 1][tid] = pra;
                S.rb[buf ^ 1][tid] = prb;
            }
            __syncthreads();
        }
        if (S.abort_flag) break;
        if (nrows > 0) flush32(S, a, nrows, mma_phase, v, tx, ty);
        if (S.abort_flag) break;
        __syncthreads();   // every thread has read S.item before thread 0 takes the next one
    }
    __syncthreads();
    if (S.abort_flag && tid == 0) mbar_wait(&S.mma_done, mma_phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(S.tmem_base, 512);
}

}  // namespace

bool tc32_supported(int dtype, int d) { return dtype == LUDVIG_F32 && d >= 32; }

ludvig_status composite_tc32(const float4* rec_a, const float2* rec_b, int64_t n, const uint2* ranges,
                             const uint32_t* list, int nv, int width, int height, const float* feats, int d,
                             float* num, float* den, Arena& ws, int* status, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        LV_CUDA(cudaFuncSetAttribute(k_composite_tc32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
        configured = true;
    }
    int* counter;
    LV_TRY(ws.get("tc32.counter", 1, &counter));
    LV_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    int dev = 0, sms = 148;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    T32Args a;
    a.rec_a = rec_a;
    a.rec_b = rec_b;
    a.n = n;
    a.ranges = ranges;
    a.list = list;
    a.ntiles = TX * TY;
    a.TX = TX;
    a.width = width;
    a.height = height;
    a.d = d;
    a.nitems = nv * TX * TY;
    a.feats = feats;
    a.num = num;
    a.den = den;
    a.counter = counter;
    a.status = status;
    k_composite_tc32<<<std::min(sms, a.nitems), kThreads, kSmemBytes, st>>>(a);
    LV_LAUNCH();
    return LUDVIG_OK;
}

}  // namespace ludvig
