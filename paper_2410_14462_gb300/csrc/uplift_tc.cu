// Tensor-core aggregation of the uplift (Sec. 3.2, Eq. 3):
// num[i,:] += sum_p w_i(p) F[p,:] and den[i] += sum_p w_i(p) per 16x16 tile,
// as the dense product W_tile F_tile on the 5th-generation tensor cores, for
// bfloat16 features (NT = 1) and float32 features (NT = 2, float32-level
// accuracy).
//
// NT = 2: the float32 features are split beforehand into two bfloat16 arrays
// F = F1 + F2 (k_split_f32) and the weights into w = W1 + W2; the product keeps
// W1 F1 + W2 F1 + W1 F2 (16 significant bits per operand, the dropped W2 F2 and
// the residuals are below 2^-16 relative).  den sums the same W terms, so each
// f_i stays a convex combination of the features.
//
// Two kernels per chunk of views:
//
//  k_weights (CUDA cores, one CTA of 8 warps per (view, tile), several CTAs
//  per SM): walks the tile's depth-ordered list in batches of 32 Gaussians
//  (float32 rules of Eq. 1: alpha, 1/255 skip, 1e-4 stop), one 8x4 pixel block
//  per warp, the list records streaming in by bulk copies kRing - 1 batches
//  ahead.  The batch's weights go to 32 staging rows in shared memory; the
//  Gaussians with a non-zero weight somewhere in the tile are then appended,
//  as dense bfloat16 rows of 256 pixels, to the tile's "chunks" of 128 rows in
//  global memory (chunk ids from an atomic counter; row count, Gaussian ids
//  and the tile's next chunk recorded per chunk, the first chunk per tile).
//
//  k_aggregate_tc (one persistent CTA per SM, warp-specialised, tiles taken
//  round-robin with each tile's chunks back to back):
//    warp 0     TMA producer: the chunk's W rows (4 x 16 KB per term, 128-byte
//               swizzle, K-major) and the tile's feature blocks (256 pixels x
//               64 channels, MN-major) into rings of stages;
//    warp 1     MMA issuer: tcgen05.mma kind::f16, M = 128 rows, N = 64
//               channels, K = 256 pixels, one 64-column TMEM slot (of 8) per
//               channel block;
//    warps 2-5  epilogue: den from the W rows in shared memory, then each slot
//               read back (tcgen05.ld), turned through shared memory so that
//               a warp's vector reductions cover two 256-byte row segments
//               each, and added into num.
//  mbarriers hand every stage between the roles, so loads, MMAs and the
//  epilogue of neighbouring blocks and chunks overlap.
//
// Every mbarrier wait is bounded: on expiry the kernel records
// LUDVIG_ERR_TIMEOUT, stops taking work, waits (bounded) for what it issued,
// frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "spec.cuh"
#include "tc_ptx.cuh"

namespace ludvig {

namespace {

using namespace tc;

constexpr int kTcBatch = 32;                           // Gaussians composited per step
constexpr int kRing = 8;                               // list-record batches in flight
constexpr int kCRows = 128;                            // rows per chunk (MMA M)
constexpr int kRowBytes = 256 * 2;                     // one row: 256 pixels, bfloat16
constexpr uint32_t kChunkBytes = kCRows * kRowBytes;   // 64 KB per term
constexpr uint32_t kAtomBytes = kCRows * 128;          // 64-pixel K atom of a chunk: 16 KB
constexpr uint32_t kFBlockBytes = 256 * 64 * 2;        // 32 KB: 256 pixels x 64 channels
constexpr int kSlots = 8;                              // TMEM: 8 slots of 64 float32 columns
constexpr int kAggThreads = 192;                       // producer, MMA, 4 epilogue warps

// kind::f16 instruction descriptor: D float32, A and B bfloat16, A K-major,
// B MN-major, M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((64u >> 3) << 17) |
                            ((128u >> 4) << 24);

// ------------------------------------------------------------ weights

struct WeightsArgs {
    const PairRec* pairs;   // list records in list order
    const uint2* ranges;
    int ntiles, TX, width, height;
    uint8_t* wg1;           // [cap][128][256] bfloat16: W (NT = 1) or W1
    uint8_t* wg2;           // W2 (NT = 2)
    uint32_t* chunk_gid;    // [cap][128]
    int* chunk_rows;        // [cap]
    int* chunk_next;        // [cap]: the tile's next chunk, or -1
    int* item_first;        // [nitems]: the tile's first chunk, or -1 (set to -1 before the launch)
    int* chunk_counter;
    int cap;
    int* status;
};

template <int NT>
struct WeightsSmem {
    uint64_t rec_full[kRing];
    alignas(16) PairRec rec[kRing][kTcBatch];
    alignas(16) uint8_t stage[NT][kTcBatch * kRowBytes];   // [term][j][256 pixels]
    uint32_t rowmask[2];
    int cur_chunk, cur_start, next_chunk;
    int abort_flag;
};

__device__ __forceinline__ void finish_chunk(const WeightsArgs& a, int c, int rows, int next) {
    if (c >= 0 && c < a.cap) {
        a.chunk_rows[c] = rows;
        a.chunk_next[c] = next;
    }
}

template <int NT>
__global__ void __launch_bounds__(256, 4) k_weights(WeightsArgs a) {
    __shared__ WeightsSmem<NT> S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int item = blockIdx.x;
    const int v = item / a.ntiles, tile = item - v * a.ntiles;
    const int tx = tile % a.TX, ty = tile / a.TX;
    const uint2 range = a.ranges[item];
    const uint32_t nb = (range.y - range.x + kTcBatch - 1) / kTcBatch;
    if (nb == 0) return;
    // warp w covers the 8x4 pixel block ((w & 1) * 8, (w >> 1) * 4) of the tile
    const int lx = (warp & 1) * 8 + (lane & 7), ly = (warp >> 1) * 4 + (lane >> 3);
    const int pix = ly * kTile + lx;
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;

    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) mbar_init(&S.rec_full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.rowmask[0] = 0u;
        S.rowmask[1] = 0u;
        S.cur_chunk = -1;
        S.cur_start = 0;
        S.next_chunk = -1;
        S.abort_flag = 0;
    }
    for (int e = tid; e < (int)(NT * kTcBatch * kRowBytes / 16); e += 256)
        reinterpret_cast<uint4*>(&S.stage[0][0])[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    // batch k of the list goes to ring slot k % kRing
    uint32_t rissue = 0, rcons = 0;
    auto issue_records = [&](uint32_t k) {
        if (tid == 0) {
            const uint32_t s = k % kRing;
            const uint32_t b0 = range.x + k * kTcBatch;
            const uint32_t bytes = min((uint32_t)kTcBatch, range.y - b0) * (uint32_t)sizeof(PairRec);
            mbar_expect_tx(&S.rec_full[s], bytes);
            bulk_load(S.rec[s], a.pairs + b0, bytes, &S.rec_full[s]);
        }
        ++rissue;
    };
    for (uint32_t k = 0; k < nb && k + 1 < (uint32_t)kRing; ++k) issue_records(k);

    float T = 1.0f;
    bool done = !(px < a.width && py < a.height);
    int nrows = 0;   // rows of this tile written so far
    int buf = 0;
    for (uint32_t k = 0; k < nb; ++k, buf ^= 1) {
        const uint32_t slot = k % kRing;
        if (!mbar_wait(&S.rec_full[slot], (k / kRing) & 1u)) {
            S.abort_flag = 1;
            atomicExch(a.status, (int)LUDVIG_ERR_TIMEOUT);
        }
        ++rcons;
        if (__syncthreads_count(!done) == 0 || S.abort_flag) break;
        // every thread is past batch k-1: its slot takes batch k + kRing - 1
        if (k + kRing - 1 < nb) issue_records(k + kRing - 1);
        if (tid == 0) {
            // rows [nrows, nrows + 32) must have chunks; a chunk filled to
            // exactly 128 rows may not have its successor yet
            if (nrows >= S.cur_start + kCRows) {
                if (S.next_chunk < 0) S.next_chunk = atomicAdd(a.chunk_counter, 1);
                finish_chunk(a, S.cur_chunk, kCRows, S.next_chunk);
                S.cur_chunk = S.next_chunk;
                S.cur_start += kCRows;
                S.next_chunk = -1;
            }
            if (S.cur_chunk < 0) {
                S.cur_chunk = atomicAdd(a.chunk_counter, 1);
                a.item_first[item] = S.cur_chunk;
            }
            if (nrows + kTcBatch > S.cur_start + kCRows && S.next_chunk < 0)
                S.next_chunk = atomicAdd(a.chunk_counter, 1);
        }
        const PairRec* rec = S.rec[slot];
        const int cnt = (int)min((uint32_t)kTcBatch, range.y - (range.x + k * kTcBatch));
        uint32_t lm = 0u;   // this lane's non-zero weights (bit j = Gaussian j)
        if (__any_sync(0xffffffffu, !done)) {
            // Gaussians of the batch that can reach this warp's pixel block,
            // four at a time in list order: the four alphas are independent,
            // the transmittance recursion then takes them in order
            uint32_t rel = __ballot_sync(0xffffffffu, lane < cnt && ((rec[lane].mask >> warp) & 1u));
            while (rel != 0u && __any_sync(0xffffffffu, !done)) {
                int jj[4];
                float al[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    jj[q] = rel ? __ffs(rel) - 1 : -1;
                    rel &= rel - 1u;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jj[q] < 0 ? jj[0] : jj[q];
                    const float4 g = *reinterpret_cast<const float4*>(&rec[j].mx);
                    const float2 h = *reinterpret_cast<const float2*>(&rec[j].cc);
                    al[q] = alpha_at_nb(g.x, g.y, g.z, g.w, h.x, h.y, pxf, pyf);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (jj[q] >= 0 && al[q] > 0.f && !done) {
                        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al[q]));
                        if (Tn < kTransMin) {
                            done = true;
                        } else {
                            const float wv = __fmul_rn(al[q], T);
                            T = Tn;
                            lm |= 1u << jj[q];
                            const int o = jj[q] * kRowBytes + pix * 2;
                            const __nv_bfloat16 h1 = __float2bfloat16_rn(wv);
                            *reinterpret_cast<__nv_bfloat16*>(&S.stage[0][o]) = h1;
                            if (NT == 2)
                                *reinterpret_cast<__nv_bfloat16*>(&S.stage[NT - 1][o]) =
                                    __float2bfloat16_rn(wv - __bfloat162float(h1));
                        }
                    }
                }
            }
            const uint32_t mine = __reduce_or_sync(0xffffffffu, lm);
            if (lane == 0 && mine) atomicOr(&S.rowmask[buf], mine);
        }
        if (tid == 0) S.rowmask[buf ^ 1] = 0u;
        __syncthreads();
        const uint32_t rowmask = S.rowmask[buf];
        const int nnew = __popc(rowmask);
        const int cur = S.cur_chunk, nxt = S.next_chunk, cstart = S.cur_start;
        // the staging row of the i-th new Gaussian goes to tile row nrows + i
        // (chunk cur, or nxt past its 128 rows), 16 bytes per thread; the
        // staging row is cleared behind it
        const int per_term = nnew * 32;
        for (int e = tid; e < NT * per_term; e += 256) {
            const int t = e / per_term, rem = e - t * per_term;
            const int i = rem >> 5, c16 = rem & 31;
            const int j = (int)__fns(rowmask, 0u, i + 1);
            int local = nrows + i - cstart, ch = cur;
            if (local >= kCRows) {
                local -= kCRows;
                ch = nxt;
            }
            uint4* src = reinterpret_cast<uint4*>(&S.stage[t][j * kRowBytes + c16 * 16]);
            if (ch >= 0 && ch < a.cap) {
                uint8_t* dst = (t == 0 ? a.wg1 : a.wg2) + (size_t)ch * kChunkBytes + local * kRowBytes + c16 * 16;
                *reinterpret_cast<uint4*>(dst) = *src;
            }
            *src = make_uint4(0u, 0u, 0u, 0u);
        }
        if (tid < kTcBatch && ((rowmask >> tid) & 1u)) {
            int local = nrows + __popc(rowmask & lt_mask) - cstart, ch = cur;
            if (local >= kCRows) {
                local -= kCRows;
                ch = nxt;
            }
            if (ch >= 0 && ch < a.cap) a.chunk_gid[(size_t)ch * kCRows + local] = rec[tid].gid;
        }
        nrows += nnew;
        // no barrier here: the next batch's counting barrier orders these stores
    }
    // batches issued past an early stop still land: wait for them (bounded)
    for (uint32_t k = rcons; k < rissue; ++k)
        if (!mbar_wait(&S.rec_full[k % kRing], (k / kRing) & 1u)) break;
    __syncthreads();
    if (tid == 0) {
        const int cur = S.cur_chunk, cstart = S.cur_start, nxt = S.next_chunk;
        if (nrows > cstart + kCRows) {   // the last batch spilled into nxt
            finish_chunk(a, cur, kCRows, nxt);
            finish_chunk(a, nxt, nrows - cstart - kCRows, -1);
        } else {
            finish_chunk(a, cur, nrows - cstart, -1);
            finish_chunk(a, nxt, 0, -1);   // allocated, never used
        }
    }
}

// ------------------------------------------------------------ aggregation

struct AggArgs {
    int cap;
    const int* chunk_rows;
    const int* chunk_next;
    const int* item_first;
    const uint32_t* chunk_gid;
    int nitems, ntiles, TX, d;
    float* num;
    float* den;
    int* status;
    int store_mode;   // debug GEMM: num[gid * d + c] = accumulator (no den)
};

template <int NT>
struct AggSmem {
    static constexpr int kWS = NT == 1 ? 2 : 1;   // W stages (each NT x 64 KB)
    static constexpr int kFS = 2;                  // feature-block stages
    uint8_t W[kWS][NT][kChunkBytes];               // offset 0 (1024-aligned)
    uint8_t F[kFS][kFBlockBytes];
    float4 xpose[4][32 * 16];                      // epilogue: 32 rows x 64 columns per warp
    uint64_t w_full[kWS], w_empty[kWS];
    uint64_t f_full[kFS], f_empty[kFS];
    uint64_t t_full[kSlots], t_empty[kSlots];
    uint32_t tmem_base;
    int abort_flag;
};

template <int NT>
constexpr size_t agg_smem_bytes() {
    return sizeof(AggSmem<NT>) + 1024;   // + alignment slack
}

// The chunks a CTA aggregates: those of tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... in order, each tile's chunks back to back (so its feature blocks are
// still in L2 for the second chunk).  Every role walks the same sequence.
struct ChunkWalk {
    int item, c;
    __device__ ChunkWalk() : item((int)blockIdx.x - (int)gridDim.x), c(-1) {}
    // next non-empty chunk (its tile in item), or -1 at the end
    __device__ int next(const AggArgs& a) {
        for (;;) {
            if (c >= 0) c = a.chunk_next[c];
            while (c < 0) {
                item += gridDim.x;
                if (item >= a.nitems) return -1;
                c = a.item_first[item];
            }
            if (c >= a.cap) return -1;   // never with a complete weights pass
            if (a.chunk_rows[c] > 0) return c;
        }
    }
};

__device__ __forceinline__ bool agg_wait(volatile int* abort_flag, int* status, uint64_t* bar, uint32_t parity) {
    if (mbar_wait(bar, parity)) return true;
    *abort_flag = 1;
    atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
    return false;
}

template <int DB, int NT>
__global__ void __launch_bounds__(kAggThreads, 1)
    k_aggregate_tc(AggArgs a, const __grid_constant__ CUtensorMap wmap1, const __grid_constant__ CUtensorMap wmap2,
                   const __grid_constant__ CUtensorMap fmap1, const __grid_constant__ CUtensorMap fmap2) {
    using Sm = AggSmem<NT>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    Sm& S = *reinterpret_cast<Sm*>(smem_raw + pad);
    volatile int* abort_flag = &S.abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < Sm::kWS; ++s) {
            mbar_init(&S.w_full[s], 1);
            mbar_init(&S.w_empty[s], 1 + 4);   // MMA commit + 4 epilogue warps (den read)
        }
        for (int s = 0; s < Sm::kFS; ++s) {
            mbar_init(&S.f_full[s], 1);
            mbar_init(&S.f_empty[s], 1);
        }
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&S.t_full[s], 1);
            mbar_init(&S.t_empty[s], 4);
        }
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&S.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            uint32_t wc = 0, fc = 0;
            ChunkWalk walk;
            for (int c = walk.next(a); c >= 0 && !*abort_flag; c = walk.next(a)) {
                const int item = walk.item;
                const int v = item / a.ntiles, tile = item - v * a.ntiles;
                const int tx = tile % a.TX, ty = tile / a.TX;
                const uint32_t ws = wc % Sm::kWS;
                if (wc >= (uint32_t)Sm::kWS &&
                    !agg_wait(abort_flag, a.status, &S.w_empty[ws], ((wc / Sm::kWS) - 1) & 1u))
                    break;
                mbar_expect_tx(&S.w_full[ws], NT * kChunkBytes);
                for (int t = 0; t < NT; ++t)
                    for (int ka = 0; ka < 4; ++ka)
                        tma_load_2d(S.W[ws][t] + ka * kAtomBytes, t == 0 ? &wmap1 : &wmap2, &S.w_full[ws], ka * 64,
                                    c * kCRows);
                ++wc;
                bool ok = true;
                for (int b = 0; b < DB && ok; ++b)
                    for (int t = 0; t < NT; ++t) {
                        const uint32_t s = fc % Sm::kFS;
                        if (fc >= (uint32_t)Sm::kFS &&
                            !agg_wait(abort_flag, a.status, &S.f_empty[s], ((fc / Sm::kFS) - 1) & 1u)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&S.f_full[s], kFBlockBytes);
                        tma_load_4d(S.F[s], t == 0 ? &fmap1 : &fmap2, &S.f_full[s], 64 * b, tx * kTile, ty * kTile,
                                    v);
                        ++fc;
                    }
                if (!ok) break;
            }
            if (*abort_flag) {
                // let the copies already issued land (bounded)
                for (uint32_t u = (fc > (uint32_t)Sm::kFS ? fc - Sm::kFS : 0u); u < fc; ++u)
                    mbar_wait(&S.f_full[u % Sm::kFS], (u / Sm::kFS) & 1u);
                for (uint32_t u = (wc > (uint32_t)Sm::kWS ? wc - Sm::kWS : 0u); u < wc; ++u)
                    mbar_wait(&S.w_full[u % Sm::kWS], (u / Sm::kWS) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            uint32_t wc = 0, fc = 0, uc = 0;
            bool ok = true;
            ChunkWalk walk;
            for (int c = walk.next(a); c >= 0 && ok && !*abort_flag; c = walk.next(a)) {
                const uint32_t ws = wc % Sm::kWS;
                if (!agg_wait(abort_flag, a.status, &S.w_full[ws], (wc / Sm::kWS) & 1u)) break;
                tc_fence_after();
                for (int b = 0; b < DB && ok; ++b) {
                    const uint32_t slot = uc % kSlots;
                    if (uc >= (uint32_t)kSlots &&
                        !agg_wait(abort_flag, a.status, &S.t_empty[slot], ((uc / kSlots) - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = S.tmem_base + 64u * slot;
                    for (int t = 0; t < NT; ++t) {
                        const uint32_t s = fc % Sm::kFS;
                        if (!agg_wait(abort_flag, a.status, &S.f_full[s], (fc / Sm::kFS) & 1u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t f_base = saddr(S.F[s]);
                        // term 0 (F1): W1 F1 (+ W2 F1); term 1 (F2): W1 F2
#pragma unroll
                        for (int ks = 0; ks < 16; ++ks) {
                            const uint64_t bd = sw128_desc(f_base + ks * 2048, 1024, 1024);
                            const uint32_t koff = (ks >> 2) * kAtomBytes + (ks & 3) * 32;
                            const uint32_t acc = (ks > 0 || t > 0) ? 1u : 0u;
                            mma_bf16(dt, sw128_desc(saddr(S.W[ws][0]) + koff, 16, 1024), bd, kIdesc, acc);
                            if (NT == 2 && t == 0)
                                mma_bf16(dt, sw128_desc(saddr(S.W[ws][NT - 1]) + koff, 16, 1024), bd, kIdesc, 1u);
                        }
                        mma_commit(&S.f_empty[s]);
                        ++fc;
                    }
                    if (!ok) break;
                    mma_commit(&S.t_full[slot]);
                    ++uc;
                }
                if (!ok) break;
                mma_commit(&S.w_empty[ws]);
                ++wc;
            }
            if (*abort_flag && uc > 0)   // the MMAs issued complete in order (bounded)
                mbar_wait(&S.t_full[(uc - 1) % kSlots], ((uc - 1) / kSlots) & 1u);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = chunk rows
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const int d = a.d;
        uint32_t wc = 0, uc = 0;
        ChunkWalk walk;
        for (int c = walk.next(a); c >= 0 && !*abort_flag; c = walk.next(a)) {
            const int rows = a.chunk_rows[c];
            const bool valid = r < rows;
            const uint32_t g = valid ? a.chunk_gid[(size_t)c * kCRows + r] : 0u;
            const uint32_t ws = wc % Sm::kWS;
            if (!agg_wait(abort_flag, a.status, &S.w_full[ws], (wc / Sm::kWS) & 1u)) break;
            if (!a.store_mode && valid) {
                // den: the row's W terms summed over the 256 pixels
                float sden = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const uint8_t* row = S.W[ws][t] + r * 128;
#pragma unroll 2
                    for (int ka = 0; ka < 4; ++ka) {
#pragma unroll
                        for (int c16 = 0; c16 < 8; ++c16) {
                            const uint4 v4 = *reinterpret_cast<const uint4*>(row + ka * kAtomBytes + c16 * 16);
                            const uint32_t wv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                sden += __uint_as_float(wv[e] << 16);
                                sden += __uint_as_float(wv[e] & 0xffff0000u);
                            }
                        }
                    }
                }
                atomicAdd(a.den + g, sden);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.w_empty[ws]);
            ++wc;
            bool ok = true;
            for (int b = 0; b < DB; ++b) {
                const uint32_t slot = uc % kSlots;
                if (!agg_wait(abort_flag, a.status, &S.t_full[slot], (uc / kSlots) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                float v0[32], v1[32];
                const uint32_t taddr = S.tmem_base + ((uint32_t)(32 * q) << 16) + 64u * slot;
                tmem_ld32(taddr, v0);
                tmem_ld32(taddr + 32, v1);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.t_empty[slot]);
                ++uc;
                // this warp's 32 rows x 64 columns, row-major with the 16-byte
                // chunks XOR-swizzled by row (conflict-free both ways)
                float4* xp = S.xpose[q];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const float* src = c < 8 ? &v0[4 * c] : &v1[4 * (c - 8)];
                    xp[lane * 16 + (c ^ (lane & 7))] = make_float4(src[0], src[1], src[2], src[3]);
                }
                __syncwarp();
                // lane l: row 2i + l / 16, columns 4 (l % 16) .. + 3
                const int cc = lane & 15;
                const int lim = d - 64 * b;   // channels of this block inside d
#pragma unroll 4
                for (int i = 0; i < 16; ++i) {
                    const int rr = 2 * i + (lane >> 4);
                    const uint32_t gr = __shfl_sync(0xffffffffu, g, rr);
                    const float4 x = xp[rr * 16 + (cc ^ (rr & 7))];
                    if (32 * q + rr < rows && 4 * cc < lim) {
                        float* dst = a.num + (int64_t)gr * d + 64 * b + 4 * cc;
                        if (a.store_mode) {
                            dst[0] = x.x;
                            if (4 * cc + 1 < lim) dst[1] = x.y;
                            if (4 * cc + 2 < lim) dst[2] = x.z;
                            if (4 * cc + 3 < lim) dst[3] = x.w;
                        } else {
                            red_add_v4(dst, x.x, x.y, x.z, x.w);
                        }
                    }
                }
                __syncwarp();
            }
            if (!ok) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(S.tmem_base, 512);
}

// float32 features -> two bfloat16 arrays with f = hi + lo to 16 significant bits.
__global__ void k_split_f32(const float4* __restrict__ f, uint2* __restrict__ hi, uint2* __restrict__ lo,
                            int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = f[i];
        const __nv_bfloat16 a = __float2bfloat16_rn(x.x), b = __float2bfloat16_rn(x.y);
        const __nv_bfloat16 c = __float2bfloat16_rn(x.z), e = __float2bfloat16_rn(x.w);
        auto pk = [](__nv_bfloat16 l, __nv_bfloat16 h) {
            return (uint32_t)__bfloat16_as_ushort(l) | ((uint32_t)__bfloat16_as_ushort(h) << 16);
        };
        hi[i] = make_uint2(pk(a, b), pk(c, e));
        lo[i] = make_uint2(pk(__float2bfloat16_rn(x.x - __bfloat162float(a)), __float2bfloat16_rn(x.y - __bfloat162float(b))),
                           pk(__float2bfloat16_rn(x.z - __bfloat162float(c)), __float2bfloat16_rn(x.w - __bfloat162float(e))));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// bfloat16 tensor map, 128-byte swizzle, zero fill out of bounds.
ludvig_status encode_bf16(CUtensorMap* map, const void* base, cuuint32_t rank, const cuuint64_t* dims,
                          const cuuint64_t* strides, const cuuint32_t* box) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return LUDVIG_ERR_CUDA;
    }
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return LUDVIG_ERR_CUDA;
    }
    return LUDVIG_OK;
}

// Tensor map over features [nv, H, W, d] bfloat16: box of 64 channels x 16 x 16
// pixels of one view, zero fill outside the image and past d.
ludvig_status make_feature_map(CUtensorMap* map, const void* feats, int nv, int width, int height, int d) {
    cuuint64_t dims[4] = {(cuuint64_t)d, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)nv};
    cuuint64_t strides[3] = {(cuuint64_t)d * 2, (cuuint64_t)width * d * 2, (cuuint64_t)height * width * d * 2};
    cuuint32_t box[4] = {64, 16, 16, 1};
    return encode_bf16(map, feats, 4, dims, strides, box);
}

// Tensor map over chunk rows [cap * 128, 256] bfloat16: box of 64 pixels x 128
// rows (one K atom of a chunk).
ludvig_status make_w_map(CUtensorMap* map, const void* w, int64_t cap) {
    cuuint64_t dims[2] = {256, (cuuint64_t)cap * kCRows};
    cuuint64_t strides[1] = {(cuuint64_t)kRowBytes};
    cuuint32_t box[2] = {64, (cuuint32_t)kCRows};
    return encode_bf16(map, w, 2, dims, strides, box);
}

template <int DB, int NT>
ludvig_status launch_agg(const AggArgs& args, const CUtensorMap* maps, int grid, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        LV_CUDA(cudaFuncSetAttribute(k_aggregate_tc<DB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)agg_smem_bytes<NT>()));
        configured = true;
    }
    k_aggregate_tc<DB, NT><<<grid, kAggThreads, agg_smem_bytes<NT>(), st>>>(args, maps[0], maps[1], maps[2], maps[3]);
    LV_LAUNCH();
    return LUDVIG_OK;
}

template <int NT>
ludvig_status dispatch_agg(const AggArgs& args, const CUtensorMap* maps, int grid, cudaStream_t st) {
    switch ((args.d + 63) / 64) {
        case 1: return launch_agg<1, NT>(args, maps, grid, st);
        case 2: return launch_agg<2, NT>(args, maps, grid, st);
        case 3: return launch_agg<3, NT>(args, maps, grid, st);
        case 4: return launch_agg<4, NT>(args, maps, grid, st);
        case 5: return launch_agg<5, NT>(args, maps, grid, st);
        case 6: return launch_agg<6, NT>(args, maps, grid, st);
        case 7: return launch_agg<7, NT>(args, maps, grid, st);
        case 8: return launch_agg<8, NT>(args, maps, grid, st);
        default: set_error("tensor-core path needs 32 <= d <= 512"); return LUDVIG_ERR_INTERNAL;
    }
}

ludvig_status sm_count(int* sms) {
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    return LUDVIG_OK;
}

}  // namespace

// Tensor-core aggregation applies to d in [32, 512] with d % 8 == 0 (16-byte
// rows for TMA); bfloat16 features always, float32 unless disabled.
bool tc_supported(int dtype, int d) {
    return (dtype == LUDVIG_BF16 || dtype == LUDVIG_F32) && d >= 32 && d <= 512 && d % 8 == 0;
}

// Composite + tensor-core aggregation of one chunk of views (stage 6 of the
// uplift pipeline).  `status` receives LUDVIG_ERR_TIMEOUT if a wait expired;
// `*chunk_cap` (chunks of 128 weight rows kept in workspace) grows as needed.
ludvig_status composite_tc(const PairRec* pairs, const uint2* ranges, int nv, int width, int height,
                           const void* feats, int dtype, int d, float* num, float* den, Arena& ws, int* status,
                           int64_t* chunk_cap, cudaStream_t st) {
    const int NT = dtype == LUDVIG_F32 ? 2 : 1;
    int sms = 0;
    LV_TRY(sm_count(&sms));
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int nitems = nv * TX * TY;
    if (nitems == 0) return LUDVIG_OK;
    const void* f1 = feats;
    const void* f2 = feats;
    if (dtype == LUDVIG_F32) {
        // split the chunk's float32 features into two bfloat16 arrays
        const int64_t count = (int64_t)nv * width * height * d;
        void *hi, *lo;
        LV_TRY(ws.get("tc.f_hi", (size_t)count * 2, &hi));
        LV_TRY(ws.get("tc.f_lo", (size_t)count * 2, &lo));
        StageScope split_scope(LUDVIG_STAGE_SPLIT, st);
        k_split_f32<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(count / 4, 256))), 256,
                      0, st>>>(static_cast<const float4*>(feats), static_cast<uint2*>(hi), static_cast<uint2*>(lo),
                               count / 4);
        LV_LAUNCH();
        f1 = hi;
        f2 = lo;
    }
    int* counter;
    int* host;   // [0] chunks used, [1] status
    LV_TRY(ws.get("tc.counter", 1, &counter));
    {
        void* p;
        LV_TRY(ws.pinned("tc.host", 16, &p));
        host = static_cast<int*>(p);
    }
    int64_t cap = std::max<int64_t>(*chunk_cap, 3 * (int64_t)nitems);
    int count = 0;
    uint8_t *wg1 = nullptr, *wg2 = nullptr;
    uint32_t* cgid = nullptr;
    int *crows = nullptr, *cnext = nullptr, *ifirst = nullptr;
    LV_TRY(ws.get("tc.item_first", (size_t)nitems, &ifirst));
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (cap > 0x7fffffff / kCRows) {
            set_error("tile weights need %lld chunks of 128 rows", (long long)cap);
            return LUDVIG_ERR_UNSUPPORTED;
        }
        LV_TRY(ws.get("tc.w1", (size_t)cap * kChunkBytes, &wg1));
        if (NT == 2) LV_TRY(ws.get("tc.w2", (size_t)cap * kChunkBytes, &wg2));
        LV_TRY(ws.get("tc.chunk_gid", (size_t)cap * kCRows, &cgid));
        LV_TRY(ws.get("tc.chunk_rows", (size_t)cap, &crows));
        LV_TRY(ws.get("tc.chunk_next", (size_t)cap, &cnext));
        LV_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
        LV_CUDA(cudaMemsetAsync(ifirst, 0xff, sizeof(int) * (size_t)nitems, st));
        WeightsArgs w{};
        w.pairs = pairs;
        w.ranges = ranges;
        w.ntiles = TX * TY;
        w.TX = TX;
        w.width = width;
        w.height = height;
        w.wg1 = wg1;
        w.wg2 = NT == 2 ? wg2 : wg1;
        w.chunk_gid = cgid;
        w.chunk_rows = crows;
        w.chunk_next = cnext;
        w.item_first = ifirst;
        w.chunk_counter = counter;
        w.cap = (int)cap;
        w.status = status;
        const int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_WEIGHTS, st) : -1;
        if (NT == 2)
            k_weights<2><<<nitems, 256, 0, st>>>(w);
        else
            k_weights<1><<<nitems, 256, 0, st>>>(w);
        LV_LAUNCH();
        trace_end(tslot, st);
        LV_CUDA(cudaMemcpyAsync(host, counter, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaMemcpyAsync(host + 1, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        count = host[0];
        if (host[1] != 0) {
            set_error("tile weights: a bounded wait expired");
            return (ludvig_status)host[1];
        }
        if (count <= cap) break;
        // more chunks than kept: grow and run the weights again
        cap = (int64_t)count + count / 8 + 1;
    }
    if (count > cap) {
        set_error("tile weights exceed the chunk capacity");
        return LUDVIG_ERR_INTERNAL;
    }
    *chunk_cap = cap;
    if (count == 0) return LUDVIG_OK;
    CUtensorMap maps[4];
    LV_TRY(make_w_map(&maps[0], wg1, cap));
    LV_TRY(make_w_map(&maps[1], NT == 2 ? wg2 : wg1, cap));
    LV_TRY(make_feature_map(&maps[2], f1, nv, width, height, d));
    LV_TRY(make_feature_map(&maps[3], f2, nv, width, height, d));
    AggArgs g{};
    g.cap = (int)cap;
    g.chunk_rows = crows;
    g.chunk_next = cnext;
    g.item_first = ifirst;
    g.chunk_gid = cgid;
    g.nitems = nitems;
    g.ntiles = TX * TY;
    g.TX = TX;
    g.d = d;
    g.num = num;
    g.den = den;
    g.status = status;
    g.store_mode = 0;
    const int grid = std::min(sms, nitems);
    StageScope agg_scope(LUDVIG_STAGE_AGGREGATE, st);
    if (NT == 2) return dispatch_agg<2>(g, maps, grid, st);
    return dispatch_agg<1>(g, maps, grid, st);
}

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_debug_mma_bf16(const void* a, const void* f, int32_t d, float* out, void* stream) {
    LV_ARG(a != nullptr && f != nullptr && out != nullptr, "NULL argument");
    LV_ARG(d % 64 == 0 && d >= 64 && d <= 512, "d must be 64..512 in steps of 64");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // one chunk of 128 rows (row r -> output row r) over a single 16x16 tile
    struct Meta {
        int first, next, rows, status;
        uint32_t gid[kCRows];
    };
    static Meta* meta = nullptr;
    if (!meta) LV_CUDA(cudaMalloc(&meta, sizeof(Meta)));
    static Meta h{};
    h.first = 0;
    h.next = -1;
    h.rows = kCRows;
    h.status = 0;
    for (int r = 0; r < kCRows; ++r) h.gid[r] = (uint32_t)r;
    LV_CUDA(cudaMemcpyAsync(meta, &h, sizeof(Meta), cudaMemcpyHostToDevice, st));
    CUtensorMap maps[4];
    LV_TRY(make_w_map(&maps[0], a, 1));
    maps[1] = maps[0];
    LV_TRY(make_feature_map(&maps[2], f, 1, 16, 16, d));
    maps[3] = maps[2];
    AggArgs g{};
    g.cap = 1;
    g.chunk_rows = &meta->rows;
    g.chunk_next = &meta->next;
    g.item_first = &meta->first;
    g.chunk_gid = meta->gid;
    g.nitems = 1;
    g.ntiles = 1;
    g.TX = 1;
    g.d = d;
    g.num = out;
    g.den = nullptr;
    g.status = &meta->status;
    g.store_mode = 1;
    LV_TRY(dispatch_agg<1>(g, maps, 1, st));
    int hs = 0;
    LV_CUDA(cudaMemcpyAsync(&hs, &meta->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    if (hs != 0) {
        set_error("tensor-core kernel reported status %d", hs);
        return (ludvig_status)hs;
    }
    return LUDVIG_OK;
}
