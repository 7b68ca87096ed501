// Tensor-core aggregation of the uplift (Sec. 3.2, Eq. 3):
// num[i,:] += sum_p w_i(p) F[p,:] and den[i] += sum_p w_i(p) per 16x16 tile,
// as the dense product W_tile F_tile on the 5th-generation tensor cores, for
// bfloat16 features (NT = 1) and float32 features (NT = 2, float32-level
// accuracy).
//
// NT = 2: the float32 features are split into two bfloat16 terms F = F1 + F2
// in shared memory as they arrive, and the weights into w = W1 + W2; the product keeps
// W1 F1 + W2 F1 + W1 F2 (16 significant bits per operand, the dropped W2 F2 and
// the residuals are below 2^-16 relative).  den sums the same W terms, so each
// f_i stays a convex combination of the features.
//
// Two kernels per chunk of views:
//
//  k_weights (CUDA cores, one CTA of 8 warps per (view, tile), several CTAs
//  per SM): walks the tile's depth-ordered list in batches of 32 Gaussians
//  (float32 rules of Eq. 1: alpha, 1/255 skip, 1e-4 stop), one 8x4 pixel block
//  per warp.  Warp 0 gathers the batches' projected records (from the
//  depth-ordered record array, by the ranks the list holds) with cp.async
//  kRing - 1 batches ahead, and computes each entry's 8x4 block mask once its
//  record has landed (the next batch's masks after its own compositing of
//  the current one); only the batches the walk reaches are gathered.  The
//  batch's weights go to 32 staging rows in shared memory; the Gaussians with
//  a non-zero weight somewhere in the tile are then appended, as dense
//  bfloat16 rows of 256 pixels, to the tile's "chunks" of 128 rows in global
//  memory (chunk ids from an atomic counter; row count, Gaussian ids, den and
//  the tile's next chunk recorded per chunk, the first chunk per tile).  For
//  d <= 4 (k_weights<NT, true>) each new row is instead dotted with the
//  tile's features and added to num and den on the spot.
//
//  k_aggregate_tc (one persistent CTA per SM, warp-specialised, tiles taken
//  round-robin with each tile's chunks back to back).  Per chunk the K loop is
//  outermost: for each 64-pixel K atom, the atom of the W rows (16 KB per
//  term) and then one feature unit (64 pixels x 64 channels) per channel
//  block, all through rings of small stages so that many loads are in flight:
//    warp 0     TMA producer (128-byte swizzle; W K-major, features MN-major);
//    warps 10-17 (float32 features) turn each float32 unit into F1 | F2 in
//               place;
//    warp 1     MMA issuer: tcgen05.mma kind::f16, M = 128 rows, N = 128
//               channels (64 for an odd last block), 16 pixels per step; unit u
//               of the chunk accumulates over the 4 atoms in one 128-column
//               TMEM slot (of 4);
//    warps 2-9  epilogue, two warps per TMEM lane quarter (one per 64-column
//               half): den from the W atoms in shared memory, then each
//               finished slot read back (tcgen05.ld), one row per thread staged
//               in shared memory and added into num by the bulk-copy engine
//               (cp.reduce.async.bulk .add.f32, 256 B per row and block).
//  mbarriers hand every stage between the roles, so loads, conversion, MMAs
//  and the epilogue of neighbouring blocks and chunks overlap.
//
// Every mbarrier wait is bounded: on expiry the kernel records
// LUDVIG_ERR_TIMEOUT, stops taking work, waits (bounded) for what it issued,
// frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "spec.cuh"
#include "tc_ptx.cuh"
#include "uplift_int.cuh"

namespace ludvig {

bool option_count_normalise();
int option_agg_config();
int option_agg_sms();

namespace {

using namespace tc;

constexpr int kTcBatch = 32;                           // Gaussians composited per step
constexpr int kRing = 8;                               // list-record batches in flight
constexpr int kCRows = 128;                            // rows per chunk (MMA M)
constexpr int kRowBytes = 256 * 2;                     // one row: 256 pixels, bfloat16
constexpr uint32_t kChunkBytes = kCRows * kRowBytes;   // 64 KB per term
constexpr uint32_t kAtomBytes = kCRows * 128;          // 64-pixel K atom of a chunk: 16 KB
constexpr int kSlots = 4;                              // TMEM: 4 slots of 128 float32 columns

// kind::f16 instruction descriptor: D float32, A and B bfloat16, A K-major,
// B MN-major, M = 128, N = n.
constexpr uint32_t idesc_n(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// ------------------------------------------------------------ weights

struct WeightsArgs {
    const uint32_t* rank;   // list entries: depth rank within the view
    const PairRec* srec;    // [nv, npad] projected records in depth order
    int64_t npad;
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
    float* chunk_den;       // [cap][128][NT]: each row's den, the sum of its weight terms, in term 0's
                            // slot (term 1's: 0); rewritten on a re-run
    int count_den;          // chunk_den holds each row's count of non-zero weights instead
    // direct accumulation (k_weights<NT, true>, few channels): each new row's
    // sum_p w F[p, c] and its den go straight into the view's num and den
    // (atomic adds); no weight rows, chunks or plan are written
    int direct_d;           // channels, 1 .. kDirectMaxD
    int num_stride;         // floats per Gaussian in num
    const void* feats;      // [.., H, W, direct_d] float32 or bfloat16, views at views.fview
    int feat_bf16;
    AggViews views;
};

constexpr int kDirectMaxD = 4;

template <int NT>
struct WeightsSmemBase {
    alignas(16) PairRec rec[kRing][kTcBatch];
    alignas(16) uint8_t stage[NT][kTcBatch * kRowBytes];   // [term][j][256 pixels]
    uint32_t rowmask[2];
    int cur_chunk, cur_start, next_chunk;
};
template <int NT, bool DIRECT>
struct WeightsSmem : WeightsSmemBase<NT> {};
template <int NT>
struct WeightsSmem<NT, true> : WeightsSmemBase<NT> {
    alignas(16) float feat[kDirectMaxD][256];   // the tile's features by channel and pixel (0 off the image)
};

// A weight row's contribution to den, from its 256 bfloat16 values (8 per
// lane, packed in wv), summed over the warp: the sum of the term's values, or
// with count_den the number of non-zero weights (counted on term 0; a weight
// w > 0 is at least 1/255 * 1e-4, far above the smallest bfloat16).
__device__ __forceinline__ float lane_den(const uint32_t* wv, int count_den, int term) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (count_den)
            s += term == 0 ? (float)((wv[k] & 0xffffu) != 0u) + (float)((wv[k] >> 16) != 0u) : 0.f;
        else
            s += __uint_as_float(wv[k] << 16) + __uint_as_float(wv[k] & 0xffff0000u);
    }
    return s;
}

__device__ __forceinline__ float warp_sum(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__device__ __forceinline__ float row_den(const uint32_t* wv, int count_den, int term) {
    return warp_sum(lane_den(wv, count_den, term));
}

__device__ __forceinline__ void finish_chunk(const WeightsArgs& a, int c, int rows, int next) {
    if (c >= 0 && c < a.cap) {
        a.chunk_rows[c] = rows;
        a.chunk_next[c] = next;
    }
}

template <int NT, bool DIRECT>
__global__ void __launch_bounds__(256, 5) k_weights(const __grid_constant__ WeightsArgs a) {
    __shared__ WeightsSmem<NT, DIRECT> S;
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
        S.rowmask[0] = 0u;
        S.rowmask[1] = 0u;
        S.cur_chunk = -1;
        S.cur_start = 0;
        S.next_chunk = -1;
    }
    for (int e = tid; e < (int)(NT * kTcBatch * kRowBytes / 16); e += 256)
        reinterpret_cast<uint4*>(&S.stage[0][0])[e] = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (DIRECT) {
        // this thread's pixel's channels (zero off the image: no weight there)
        const bool in_img = px < a.width && py < a.height;
        const size_t pidx = ((size_t)a.views.fview[v] * a.height + (in_img ? py : 0)) * a.width + (in_img ? px : 0);
#pragma unroll
        for (int c = 0; c < kDirectMaxD; ++c) {
            float x = 0.f;
            if (in_img && c < a.direct_d)
                x = a.feat_bf16
                        ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.feats)[pidx * a.direct_d + c])
                        : static_cast<const float*>(a.feats)[pidx * a.direct_d + c];
            S.feat[c][pix] = x;
        }
    }
    __syncthreads();

    // batch k of the list goes to ring slot k % kRing.  Warp 0, lane j gathers
    // entry j of a batch (two 16-byte cp.async of its 32-byte record) and
    // commits one cp.async group per batch, empty past the list's end, so
    // that "at most kRing - 2 groups pending" always means "batch k landed".
    // The rank of the batch after next is loaded one iteration early, so the
    // gather does not wait on it.
    const PairRec* vrec = a.srec + (int64_t)v * a.npad;
    auto rank_of = [&](uint32_t k) -> uint32_t {
        const uint32_t e = range.x + k * kTcBatch + (uint32_t)lane;
        return (k < nb && e < range.y) ? a.rank[e] : 0xffffffffu;
    };
    auto issue_records = [&](uint32_t k, uint32_t rk) {
        if (warp == 0) {
            if (rk != 0xffffffffu) {
                PairRec* dst = &S.rec[k % kRing][lane];
                cp_async_16(dst, vrec + rk);
                cp_async_16(reinterpret_cast<uint8_t*>(dst) + 16, reinterpret_cast<const uint8_t*>(vrec + rk) + 16);
            }
            cp_async_commit();
        }
    };
    uint32_t next_rank = 0xffffffffu;   // warp 0: rank of batch k + kRing - 1 at iteration k
    // warp 0, lane j: entry j of batch k has landed; its block mask.  Batch 0's
    // is computed here, batch k + 1's after warp 0 has composited batch k (off
    // the path of the other warps, which are still compositing batch k)
    auto mask_batch = [&](uint32_t k) {
        cp_async_wait<kRing - 2>();
        if (k < nb && range.x + k * kTcBatch + (uint32_t)lane < range.y) {
            PairRec& r = S.rec[k % kRing][lane];
            r.mask = block_mask_fast(r.mx, r.my, r.ca, r.cb, r.cc, r.op, tx, ty);
        }
    };
    if (warp == 0) {
        for (uint32_t k = 0; k + 1 < (uint32_t)kRing; ++k) issue_records(k, rank_of(k));
        next_rank = rank_of(kRing - 1);
        mask_batch(0);
    }

    float T = 1.0f;
    bool done = !(px < a.width && py < a.height);
    int nrows = 0;   // rows of this tile written so far
    int buf = 0;
    for (uint32_t k = 0; k < nb; ++k, buf ^= 1) {
        const uint32_t slot = k % kRing;
        if (__syncthreads_count(!done) == 0) break;
        // every thread is past batch k-1: its slot takes batch k + kRing - 1
        if (warp == 0) {
            issue_records(k + kRing - 1, next_rank);
            next_rank = rank_of(k + kRing);
        }
        if (!DIRECT && tid == 0) {
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
        if (warp == 0) mask_batch(k + 1);   // (pending: batches k+1 .. k+kRing-1)
        if (tid == 0) S.rowmask[buf ^ 1] = 0u;
        __syncthreads();
        const uint32_t rowmask = S.rowmask[buf];
        const int nnew = __popc(rowmask);
        const int cur = S.cur_chunk, nxt = S.next_chunk, cstart = S.cur_start;
        // the staging row of the i-th new Gaussian (the i-th set bit j of the
        // row mask) goes to tile row nrows + i (chunk cur, or nxt past its 128
        // rows), 16 bytes per lane, one warp per row and term; the staging row
        // is cleared behind, the row's sum of each term (the bfloat16 values the
        // product uses) is kept for den, and the Gaussian id is recorded
        if constexpr (DIRECT) {
            // warp i % 8 takes row i: its weights w = W1 (+ W2), 8 pixels per
            // lane, dotted with the tile's channels; the staging row is cleared
            float* const vnum = a.views.num[v];
            float* const vden = a.views.den[v];
            uint32_t m = rowmask;
            for (int i = 0; m != 0u; ++i, m &= m - 1u) {
                if ((i & 7) != warp) continue;
                const int j = __ffs(m) - 1;
                float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float sden = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    uint4* src = reinterpret_cast<uint4*>(&S.stage[t][j * kRowBytes + lane * 16]);
                    const uint4 v4 = *src;
                    *src = make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t wv[4] = {v4.x, v4.y, v4.z, v4.w};
                    sden += lane_den(wv, a.count_den, t);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        w[2 * k] += __uint_as_float(wv[k] << 16);
                        w[2 * k + 1] += __uint_as_float(wv[k] & 0xffff0000u);
                    }
                }
                sden = warp_sum(sden);   // the row's den over both terms
                const uint32_t gid = rec[j].gid;
#pragma unroll
                for (int c = 0; c < kDirectMaxD; ++c) {
                    if (c >= a.direct_d) break;
                    const float4 f0 = *reinterpret_cast<const float4*>(&S.feat[c][lane * 8]);
                    const float4 f1 = *reinterpret_cast<const float4*>(&S.feat[c][lane * 8 + 4]);
                    float sc = w[0] * f0.x;
                    sc = fmaf(w[1], f0.y, sc);
                    sc = fmaf(w[2], f0.z, sc);
                    sc = fmaf(w[3], f0.w, sc);
                    sc = fmaf(w[4], f1.x, sc);
                    sc = fmaf(w[5], f1.y, sc);
                    sc = fmaf(w[6], f1.z, sc);
                    sc = fmaf(w[7], f1.w, sc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
                    if (lane == 0) atomicAdd(vnum + (size_t)gid * a.num_stride + c, sc);
                }
                if (lane == 0) atomicAdd(vden + gid, sden);
            }
        } else if constexpr (NT == 2) {
            // warp i % 8 takes row i, both terms
            uint32_t m = rowmask;
            for (int i = 0; m != 0u; ++i, m &= m - 1u) {
                if ((i & 7) != warp) continue;
                const int j = __ffs(m) - 1;
                int local = nrows + i - cstart, ch = cur;
                if (local >= kCRows) {
                    local -= kCRows;
                    ch = nxt;
                }
                const bool keep = ch >= 0 && ch < a.cap;
                float sden = 0.f;   // this lane's part of the row's den, both terms
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    uint4* src = reinterpret_cast<uint4*>(&S.stage[t][j * kRowBytes + lane * 16]);
                    const uint4 v4 = *src;
                    if (keep) {
                        uint8_t* dst = (t == 0 ? a.wg1 : a.wg2) + (size_t)ch * kChunkBytes + local * kRowBytes + lane * 16;
                        *reinterpret_cast<uint4*>(dst) = v4;
                    }
                    *src = make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t wv[4] = {v4.x, v4.y, v4.z, v4.w};
                    sden += lane_den(wv, a.count_den, t);
                }
                sden = warp_sum(sden);
                if (lane == 0 && keep) {
                    // the row's den in term 0's slot (the aggregation adds the slots)
                    a.chunk_den[((size_t)ch * kCRows + local) * NT] = sden;
                    a.chunk_den[((size_t)ch * kCRows + local) * NT + 1] = 0.f;
                    a.chunk_gid[(size_t)ch * kCRows + local] = rec[j].gid;
                }
            }
        } else {
            // warp w takes row w (row i of the 32 at most: warp i % 8 on pass i / 8)
            for (int e = tid; e < nnew * 32; e += 256) {
                const int i = e >> 5;
                const int j = (int)__fns(rowmask, 0u, i + 1);
                int local = nrows + i - cstart, ch = cur;
                if (local >= kCRows) {
                    local -= kCRows;
                    ch = nxt;
                }
                uint4* src = reinterpret_cast<uint4*>(&S.stage[0][j * kRowBytes + lane * 16]);
                const uint4 v4 = *src;
                if (ch >= 0 && ch < a.cap)
                    *reinterpret_cast<uint4*>(a.wg1 + (size_t)ch * kChunkBytes + local * kRowBytes + lane * 16) = v4;
                *src = make_uint4(0u, 0u, 0u, 0u);
                const uint32_t wv[4] = {v4.x, v4.y, v4.z, v4.w};
                const float sden = row_den(wv, a.count_den, 0);
                if (lane == 0 && ch >= 0 && ch < a.cap) a.chunk_den[(size_t)ch * kCRows + local] = sden;
            }
            if (tid < kTcBatch && ((rowmask >> tid) & 1u)) {
                int local = nrows + __popc(rowmask & lt_mask) - cstart, ch = cur;
                if (local >= kCRows) {
                    local -= kCRows;
                    ch = nxt;
                }
                if (ch >= 0 && ch < a.cap) a.chunk_gid[(size_t)ch * kCRows + local] = rec[tid].gid;
            }
        }
        nrows += nnew;
        // no barrier here: the next batch's counting barrier orders these stores
    }
    // gathers issued past an early stop still land before the CTA exits
    if (warp == 0) cp_async_wait<0>();
    __syncthreads();
    if (!DIRECT && tid == 0) {
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
    const float* chunk_den;   // [cap][128][NT]
    int nitems, ntiles, TX, d;
    int* status;
    int store_mode;          // debug GEMM: views.num[0][gid * d + c] = accumulator (no den)
    const int* chunk_count;  // chunks the weights pass used (may be null: known to fit)
    int* ovf;                // set to 2 when they exceeded cap (the launch then adds nothing)
    const uint32_t* plan_off;   // [nitems + 1]: the item's chunks are plan[plan_off[item] ..)
    const int2* plan;           // {chunk, rows} of every non-empty chunk, tile after tile
    const float* scales;        // FP8 codes: the scales by feature coordinate (x = decode(q) s_v)
    AggViews views;             // per view: feature coordinate and the num / den it adds into
};

// Feature units (16 KB): 128 channels of 64 pixels (NT = 1: one K atom, two
// 64-channel bfloat16 boxes of 8 KB) or of 32 pixels (NT = 2: half an atom,
// four 32-channel float32 boxes of 4 KB, turned in place into F1 (first 8 KB)
// and F2 (second 8 KB) by the converter warps).  The two 64-channel atoms of a
// term sit kBoxBytes apart (the MMA's N = 128).
// CF selects the float32 layout: 0 = seven feature stages and four epilogue
// warps, 1 = five stages and eight epilogue warps (more staged rows in flight).
// With NT = 1, CF = 2 takes FP8-E4M3 codes: each stage's codes (64 pixels x
// 128 channels, one 8 KB box in its second half) are decoded by 8 converter
// warps into the bfloat16 unit layout the MMA reads (x its view's scale,
// rounded to bfloat16), so the codes cross DRAM and the TMA unit at one byte
// per value.
template <int NT, int CF>
struct AggSmem {
    static constexpr int kWA = NT == 1 ? 4 : 2;              // W atom stages (NT x 16 KB each)
    static constexpr int kHalves = NT == 2 ? 2 : 1;           // feature units per K atom and channel group
    static constexpr int kUnitPx = 64 / kHalves;              // pixels per unit
    static constexpr uint32_t kBoxBytes = kUnitPx * 128u;     // one 128-byte-wide box (and one F1 atom)
    static constexpr uint32_t kFStage = 16384u;               // one feature unit
    static constexpr int kFS = (NT == 1 || CF == 1) ? 5 : 7;  // 80 KB or 112 KB of stages
    static constexpr int kEH = (NT == 1 || CF == 1) ? 2 : 1;  // epilogue warps per TMEM lane quarter
    static constexpr bool kF8 = NT == 1 && CF == 2;          // operands decoded from FP8 codes
    static constexpr int kConvWarps = (NT == 2 || kF8) ? 8 : 0;
    static constexpr int kConv0 = 2 + 4 * kEH;                // first converter warp
    static constexpr int kThreads = 32 * (kConv0 + kConvWarps);
    static constexpr int kPitch = 68;                         // staged row: 64 floats + 16 B pad
    uint8_t W[kWA][NT][kAtomBytes];                           // offset 0 (1024-aligned)
    uint8_t F[kFS][kFStage];
    float rows[4 * kEH][32 * kPitch];                         // epilogue: 32 rows x 64 columns per warp
    uint64_t w_full[kWA], w_empty[kWA];
    uint64_t f_full[kFS], f_conv[kFS], f_empty[kFS];
    uint64_t t_full[kSlots], t_empty[kSlots];
    static constexpr int kQ = 16;                             // chunk queue (producer -> other roles)
    static constexpr int kConsumers = 1 + 4 * kEH + kConvWarps;   // MMA thread + warps
    int4 q[kQ];                                               // chunk, tile, rows (chunk -1: end)
    uint64_t q_full[kQ], q_empty[kQ];
    uint32_t tmem_base;
    int abort_flag;
};

template <int NT, int CF>
constexpr size_t agg_smem_bytes() {
    return sizeof(AggSmem<NT, CF>) + 1024;   // + alignment slack
}
static_assert(agg_smem_bytes<1, 0>() <= 232448 && agg_smem_bytes<2, 0>() <= 232448 &&
                  agg_smem_bytes<2, 1>() <= 232448 && agg_smem_bytes<1, 2>() <= 232448,
              "shared memory");

// warp 0 producer, warp 1 MMA, then 4 kEH epilogue warps (8, or 4 for NT = 2
// with CF = 0) and, for NT = 2, 8 converter warps from kConv0
template <int NT, int CF>
constexpr int agg_threads() {
    return AggSmem<NT, CF>::kThreads;
}

// The chunks a CTA aggregates: those of tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... in order, each tile's chunks back to back (so its feature blocks are
// still in L2 for the second chunk).  A plan pass flattens every tile's chunk
// chain into consecutive {chunk, rows} entries first, so that the producer
// reads its sequence with independent loads it can issue ahead (following the
// chain would cost it a few dependent global loads per chunk), and hands it
// to the other roles through a queue in shared memory.

// Plan: non-empty chunks per item (count pass), then their entries (fill
// pass), one thread per item walking its chain.
__global__ void k_agg_plan(const int* __restrict__ item_first, const int* __restrict__ chunk_rows,
                           const int* __restrict__ chunk_next, int cap, int nitems, const uint32_t* __restrict__ off,
                           uint32_t* __restrict__ count, int2* __restrict__ plan) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nitems) {
        if (count && item == nitems) count[item] = 0u;
        return;
    }
    uint32_t k = off ? off[item] : 0u;
    for (int c = item_first[item]; c >= 0 && c < cap; c = chunk_next[c]) {
        const int rows = chunk_rows[c];
        if (rows <= 0) continue;
        if (plan) plan[k] = make_int2(c, rows);
        ++k;
    }
    if (count) count[item] = k;
}

__device__ __forceinline__ bool agg_wait(volatile int* abort_flag, int* status, uint64_t* bar, uint32_t parity);

// Next entry of the chunk queue for a consumer role (whole warp, or the MMA
// thread alone); false on a timed-out wait.  The entry's slot is released
// right away (one arrival per consumer warp).
template <class Sm>
__device__ __forceinline__ bool queue_next(Sm& S, volatile int* abort_flag, int* status, uint32_t& qc, int4& e,
                                           bool single) {
    const uint32_t slot = qc % Sm::kQ;
    if (!agg_wait(abort_flag, status, &S.q_full[slot], (qc / Sm::kQ) & 1u)) return false;
    e = S.q[slot];
    if (!single) __syncwarp();
    if (single || (threadIdx.x & 31) == 0) mbar_arrive(&S.q_empty[slot]);
    ++qc;
    return true;
}

__device__ __forceinline__ bool agg_wait(volatile int* abort_flag, int* status, uint64_t* bar, uint32_t parity) {
    if (mbar_wait(bar, parity)) return true;
    *abort_flag = 1;
    atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
    return false;
}

// float32 -> bfloat16 f1 = rn(x) and f2 = rn(x - f1) for 8 values (x - f1 is
// exact in float32), packed two per word in channel order.
__device__ __forceinline__ void split8(const float* x, uint4& f1, uint4& f2) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * k] - hf.x, x[2 * k + 1] - hf.y);
        h[k] = *reinterpret_cast<const uint32_t*>(&hb);
        l[k] = *reinterpret_cast<const uint32_t*>(&lb);
    }
    f1 = make_uint4(h[0], h[1], h[2], h[3]);
    f2 = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int DB, int NT, int CF>
__global__ void __launch_bounds__(agg_threads<NT, CF>(), 1)
    k_aggregate_tc(const __grid_constant__ AggArgs a, const __grid_constant__ CUtensorMap wmap1,
                   const __grid_constant__ CUtensorMap wmap2,
                   const __grid_constant__ CUtensorMap fmap) {
    using Sm = AggSmem<NT, CF>;
    // a weights pass that ran out of chunks left incomplete rows: the group is
    // redone once the workspace has grown, so nothing of it may be added now
    if (a.chunk_count && *a.chunk_count > a.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.ovf) atomicOr(a.ovf, 2);
        return;
    }
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    Sm& S = *reinterpret_cast<Sm*>(smem_raw + pad);
    volatile int* abort_flag = &S.abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < Sm::kWA; ++s) {
            mbar_init(&S.w_full[s], 1);
            mbar_init(&S.w_empty[s], 1);       // MMA commit
        }
        for (int s = 0; s < Sm::kFS; ++s) {
            mbar_init(&S.f_full[s], 1);
            mbar_init(&S.f_conv[s], 8);        // 8 converter warps (NT = 2)
            mbar_init(&S.f_empty[s], 1);
        }
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&S.t_full[s], 1);
            mbar_init(&S.t_empty[s], 4 * Sm::kEH);
        }
        for (int s = 0; s < Sm::kQ; ++s) {
            mbar_init(&S.q_full[s], 1);
            mbar_init(&S.q_empty[s], Sm::kConsumers);
        }
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&S.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    constexpr int U = (DB + 1) / 2;   // 128-channel units per chunk
    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: per chunk, K atom ka: W atom, then the U feature units
            uint32_t wc = 0, fc = 0, qc = 0;
            bool ok = true;
            // weight rows are read once and a tile's features by its chunks only:
            // first out of L2 after their last use, so that the num lines the
            // epilogue adds into stay there between tiles
            const uint64_t stream_policy = policy_evict_first(), keep_policy = policy_evict_normal();
            // plan entries: this item's [k, kend), the next item's range loaded one item ahead
            int item = blockIdx.x;
            uint32_t k = 0, kend = 0;
            if (item < a.nitems) {
                k = a.plan_off[item];
                kend = a.plan_off[item + 1];
            }
            int nitem = item + (int)gridDim.x;
            uint32_t nk = 0, nkend = 0;
            if (nitem < a.nitems) {
                nk = a.plan_off[nitem];
                nkend = a.plan_off[nitem + 1];
            }
            int2 e = k < kend ? a.plan[k] : make_int2(-1, 0);
            for (;;) {
                while (item < a.nitems && k >= kend) {   // next item with chunks
                    item = nitem;
                    k = nk;
                    kend = nkend;
                    nitem += (int)gridDim.x;
                    if (nitem < a.nitems) {
                        nk = a.plan_off[nitem];
                        nkend = a.plan_off[nitem + 1];
                    }
                    if (k < kend) e = a.plan[k];
                }
                const int c = (ok && !*abort_flag && item < a.nitems) ? e.x : -1;
                const int rows = e.y;
                const bool tile_last = k + 1 >= kend;
                if (c >= 0 && !tile_last) e = a.plan[k + 1];   // the next entry, ahead of its use
                // publish the chunk (or the end) to the other roles
                const uint32_t qs = qc % Sm::kQ;
                if (qc >= (uint32_t)Sm::kQ &&
                    !agg_wait(abort_flag, a.status, &S.q_empty[qs], ((qc / Sm::kQ) - 1) & 1u))
                    break;
                S.q[qs] = make_int4(c, c >= 0 ? item : -1, c >= 0 ? rows : 0, 0);
                mbar_arrive(&S.q_full[qs]);
                ++qc;
                if (c < 0) break;
                ++k;
                const int v = item / a.ntiles, tile = item - v * a.ntiles;
                const int tx = tile % a.TX, ty = tile / a.TX;
                const int fv = a.views.fview[v];   // the view's coordinate in the feature array
                const uint64_t fpolicy = tile_last ? stream_policy : keep_policy;
                for (int ka = 0; ka < 4 && ok; ++ka) {
                    const uint32_t ws = wc % Sm::kWA;
                    if (wc >= (uint32_t)Sm::kWA &&
                        !agg_wait(abort_flag, a.status, &S.w_empty[ws], ((wc / Sm::kWA) - 1) & 1u)) {
                        ok = false;
                        break;
                    }
                    // only the chunk's rows, in boxes of 32 (the rest of the atom is not read
                    // into any kept result)
                    const int nrb = (rows + 31) >> 5;
                    mbar_expect_tx(&S.w_full[ws], (uint32_t)(NT * nrb) * 4096u);
                    for (int rb = 0; rb < nrb; ++rb) {
                        tma_load_2d_hint(S.W[ws][0] + 4096 * rb, &wmap1, &S.w_full[ws], ka * 64, c * kCRows + 32 * rb,
                                         stream_policy);
                        if (NT == 2)
                            tma_load_2d_hint(S.W[ws][NT - 1] + 4096 * rb, &wmap2, &S.w_full[ws], ka * 64,
                                             c * kCRows + 32 * rb, stream_policy);
                    }
                    ++wc;
                    for (int un = 0; un < U && ok; ++un)
                    for (int hf = 0; hf < Sm::kHalves; ++hf) {
                        const uint32_t s = fc % Sm::kFS;
                        if (fc >= (uint32_t)Sm::kFS &&
                            !agg_wait(abort_flag, a.status, &S.f_empty[s], ((fc / Sm::kFS) - 1) & 1u)) {
                            ok = false;
                            break;
                        }
                        if constexpr (Sm::kF8) {
                            // 64 pixels x 128 codes, one box, into the stage's second half
                            mbar_expect_tx(&S.f_full[s], 8192u);
                            tma_load_4d_hint(S.F[s] + 8192, &fmap, &S.f_full[s], 128 * un, tx * kTile,
                                             ty * kTile + 4 * ka, fv, fpolicy);
                        } else {
                            mbar_expect_tx(&S.f_full[s], Sm::kFStage);
                            // kUnitPx pixels (kUnitPx / 16 rows of the tile) x 128 channels:
                            // boxes of 64 bfloat16 or 32 float32 channels
                            constexpr int kBoxes = 2 * NT, kBoxCh = 64 / NT;
#pragma unroll
                            for (int j = 0; j < kBoxes; ++j)
                                tma_load_4d_hint(S.F[s] + Sm::kBoxBytes * j, &fmap, &S.f_full[s],
                                                 128 * un + kBoxCh * j, tx * kTile,
                                                 ty * kTile + 4 * ka + (Sm::kUnitPx / 16) * hf, fv, fpolicy);
                        }
                        ++fc;
                    }
                }
            }
            if (*abort_flag) {
                // let the copies already issued land (bounded)
                for (uint32_t u = (fc > (uint32_t)Sm::kFS ? fc - Sm::kFS : 0u); u < fc; ++u)
                    mbar_wait(&S.f_full[u % Sm::kFS], (u / Sm::kFS) & 1u);
                for (uint32_t u = (wc > (uint32_t)Sm::kWA ? wc - Sm::kWA : 0u); u < wc; ++u)
                    mbar_wait(&S.w_full[u % Sm::kWA], (u / Sm::kWA) & 1u);
            }
        }
    } else if (Sm::kF8 && warp >= Sm::kConv0) {
        // ---- FP8 decoders: the stage's codes (row p = pixel, 128 bytes = 128
        // channels at 8 KB + 128 p, 16-byte chunks swizzled by p & 7) -> the
        // bfloat16 unit: 64-channel box h at 8 KB h, row p, 16-byte chunk c'
        // (8 channels) at ((c' ^ (p & 7)) << 4).  Warp cw owns rows 8 cw .. 8 cw
        // + 7; lane: row 8 cw + lane / 8 + 4 i, code chunk c = lane % 8
        // (channels 16 c ..); the codes of both rows are read before the warp
        // overwrites them (box 1 shares their bytes).
        const int cw = warp - Sm::kConv0, c = lane & 7;
        uint32_t fc = 0, qc = 0;
        bool ok = true;
        for (;;) {
            int4 e;
            if (!ok || *abort_flag || !queue_next(S, abort_flag, a.status, qc, e, false) || e.x < 0) break;
            const float sv = a.scales[a.views.fview[e.y / a.ntiles]];   // the chunk's view
            for (int un = 0; un < 4 * U; ++un) {
                const uint32_t s = fc % Sm::kFS;
                if (!agg_wait(abort_flag, a.status, &S.f_full[s], (fc / Sm::kFS) & 1u)) {
                    ok = false;
                    break;
                }
                uint8_t* base = S.F[s];
                uint4 code[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = 8 * cw + (lane >> 3) + 4 * i;
                    code[i] = *reinterpret_cast<const uint4*>(base + 8192 + p * 128 + ((c ^ (p & 7)) << 4));
                }
                __syncwarp();   // the warp's rows are read before any is overwritten
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = 8 * cw + (lane >> 3) + 4 * i;
                    const uint32_t w[4] = {code[i].x, code[i].y, code[i].z, code[i].w};
                    uint32_t o[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {   // codes 2k, 2k + 1 -> one word of two bfloat16
                        const uint32_t pair = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
                        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
                        const __nv_bfloat162 b = __floats2bfloat162_rn(f.x * sv, f.y * sv);
                        o[k] = *reinterpret_cast<const uint32_t*>(&b);
                    }
                    const int h = c >> 2, c0 = 2 * (c & 3);
                    *reinterpret_cast<uint4*>(base + 8192 * h + p * 128 + ((c0 ^ (p & 7)) << 4)) =
                        make_uint4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<uint4*>(base + 8192 * h + p * 128 + (((c0 + 1) ^ (p & 7)) << 4)) =
                        make_uint4(o[4], o[5], o[6], o[7]);
                }
                fence_proxy_async();   // generic writes, read by the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.f_conv[s]);
                ++fc;
            }
        }
    } else if (NT == 2 && warp >= Sm::kConv0) {
        // ---- converters: float32 unit (boxes j = 0..3 of 32 channels at 8 KB j)
        // -> F1 atoms h = 0, 1 (64 channels at 8 KB h) and F2 atoms (16 KB + 8 KB h).
        // Converter warp cw owns pixel rows 8 cw .. 8 cw + 7 of every region:
        // the bytes it reads are the bytes it writes, so the in-place rewrite
        // needs only a warp-level barrier.
        const int cw = warp - Sm::kConv0;
        uint32_t fc = 0, qc = 0;
        bool ok = true;
        for (;;) {
            int4 e;
            if (!ok || *abort_flag || !queue_next(S, abort_flag, a.status, qc, e, false) || e.x < 0) break;
            for (int un = 0; un < 4 * Sm::kHalves * U; ++un) {
                const uint32_t s = fc % Sm::kFS;
                if (!agg_wait(abort_flag, a.status, &S.f_full[s], (fc / Sm::kFS) & 1u)) {
                    ok = false;
                    break;
                }
                uint8_t* base = S.F[s];
                // item i: pixel row p, output chunk oc = channels 8 oc .. 8 oc + 7 of 128
                const int oc = lane & 15, box = oc >> 2, j0 = 2 * (oc & 3);
                float x[2][8];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = 4 * cw + 2 * i + (lane >> 4);
                    const uint8_t* row = base + box * 4096 + p * 128;
                    const float4 lo4 = *reinterpret_cast<const float4*>(row + ((j0 ^ (p & 7)) << 4));
                    const float4 hi4 = *reinterpret_cast<const float4*>(row + (((j0 + 1) ^ (p & 7)) << 4));
                    x[i][0] = lo4.x;
                    x[i][1] = lo4.y;
                    x[i][2] = lo4.z;
                    x[i][3] = lo4.w;
                    x[i][4] = hi4.x;
                    x[i][5] = hi4.y;
                    x[i][6] = hi4.z;
                    x[i][7] = hi4.w;
                }
                __syncwarp();   // the warp's rows are read before any is overwritten
                const int h = oc >> 3, cc = oc & 7;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int p = 4 * cw + 2 * i + (lane >> 4);
                    uint4 f1, f2;
                    split8(x[i], f1, f2);
                    const int o = 4096 * h + p * 128 + ((cc ^ (p & 7)) << 4);
                    *reinterpret_cast<uint4*>(base + o) = f1;
                    *reinterpret_cast<uint4*>(base + 8192 + o) = f2;
                }
                fence_proxy_async();   // generic writes, read by the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.f_conv[s]);
                ++fc;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: unit un of a chunk (128 channels; 64 for the last one
            // when DB is odd) accumulates over the 4 K atoms in TMEM slot
            // (units so far + un) % 4.  Descriptors advance by plain adds: the
            // start address is bits 0-13 (address / 16).
            constexpr uint32_t kIdFull = idesc_n(128), kIdLast = idesc_n(DB % 2 ? 64 : 128);
            const uint64_t w0 = sw128_desc(saddr(S.W[0][0]), 16, 1024);
            const uint64_t f0 = sw128_desc(saddr(S.F[0]), Sm::kBoxBytes, 1024);
            uint32_t wc = 0, fc = 0, ub = 0, qc = 0;
            bool ok = true;
            for (;;) {
                int4 e;
                if (!ok || *abort_flag || !queue_next(S, abort_flag, a.status, qc, e, true) || e.x < 0) break;
                for (int ka = 0; ka < 4 && ok; ++ka) {
                    const uint32_t ws = wc % Sm::kWA;
                    if (!agg_wait(abort_flag, a.status, &S.w_full[ws], (wc / Sm::kWA) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t wd1 = w0 + ((ws * NT * kAtomBytes) >> 4);
                    const uint64_t wd2 = wd1 + ((NT - 1) * kAtomBytes >> 4);
                    for (int un = 0; un < U && ok; ++un)
                    for (int hf = 0; hf < Sm::kHalves; ++hf) {
                        const uint32_t u = ub + un, slot = u % kSlots;
                        if (ka == 0 && hf == 0 && u >= (uint32_t)kSlots &&
                            !agg_wait(abort_flag, a.status, &S.t_empty[slot], ((u / kSlots) - 1) & 1u)) {
                            ok = false;
                            break;
                        }
                        const uint32_t s = fc % Sm::kFS;
                        if (!agg_wait(abort_flag, a.status, (NT == 2 || Sm::kF8) ? &S.f_conv[s] : &S.f_full[s],
                                      (fc / Sm::kFS) & 1u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = S.tmem_base + 128u * slot;
                        const uint64_t fd = f0 + ((s * Sm::kFStage) >> 4);
                        const uint32_t id = un == U - 1 ? kIdLast : kIdFull;
                        // W1 F1 (+ W2 F1 + W1 F2 for NT = 2), 16 pixels per step; the unit
                        // holds pixels kUnitPx hf .. of the atom
                        constexpr int kKS = Sm::kUnitPx / 16;
#pragma unroll
                        for (int ks = 0; ks < kKS; ++ks) {
                            const uint32_t ka16 = kKS * hf + ks;   // 16-pixel step within the W atom
                            mma_bf16(dt, wd1 + 2 * ka16, fd + 128 * ks, id, (ka > 0 || hf > 0 || ks > 0) ? 1u : 0u);
                            if (NT == 2) {
                                mma_bf16(dt, wd2 + 2 * ka16, fd + 128 * ks, id, 1u);
                                mma_bf16(dt, wd1 + 2 * ka16, fd + (8192 >> 4) + 128 * ks, id, 1u);
                            }
                        }
                        mma_commit(&S.f_empty[s]);
                        ++fc;
                        if (ka == 3 && hf == Sm::kHalves - 1) mma_commit(&S.t_full[slot]);
                    }
                    if (!ok) break;
                    mma_commit(&S.w_empty[ws]);
                    ++wc;
                }
                ub += U;
            }
            if (*abort_flag && fc > 0)   // the MMAs issued complete in order (bounded)
                mbar_wait(&S.f_empty[(fc - 1) % Sm::kFS], ((fc - 1) / Sm::kFS) & 1u);
        }
    } else if (warp >= 2 && warp < 2 + 4 * Sm::kEH) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = chunk rows;
        // with two warps per lane quarter (NT = 1) warps 2-5 take the first 64
        // columns of each unit and warps 6-9 the second 64
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int r = 32 * q + lane;
        const int d = a.d;
        float* st = &S.rows[warp - 2][lane * Sm::kPitch];
        const uint64_t num_policy = policy_evict_last();   // num lines recur in nearby tiles
        uint32_t ub = 0, qc = 0;
        bool ok = true;
        for (;;) {
            int4 e;
            if (!ok || *abort_flag || !queue_next(S, abort_flag, a.status, qc, e, false) || e.x < 0) break;
            const int c = e.x, rows = e.z;
            const bool valid = r < rows;
            const uint32_t g = valid ? a.chunk_gid[(size_t)c * kCRows + r] : 0u;
            const int cv = e.y / a.ntiles;   // the chunk's view: its num and den
            float* const num = a.views.num[cv];
            if (half == 0 && valid && !a.store_mode) {
                float sden = 0.f;
#pragma unroll
                for (int t = 0; t < NT; ++t) sden += a.chunk_den[((size_t)c * kCRows + r) * NT + t];
                atomicAdd(a.views.den[cv] + g, sden);
            }
            for (int un = 0; un < U; ++un) {
                const uint32_t u = ub + un, slot = u % kSlots;
                if (!agg_wait(abort_flag, a.status, &S.t_full[slot], (u / kSlots) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int hh = half; hh < 2; hh += Sm::kEH) {
                    const int b = 2 * un + hh;   // this warp's 64-channel block
                    const bool has = b < DB;
                    float v0[32], v1[32];
                    if (has) {
                        const uint32_t taddr = S.tmem_base + ((uint32_t)(32 * q) << 16) + 128u * slot + 64u * hh;
                        tmem_ld32(taddr, v0);
                        tmem_ld32(taddr + 32, v1);
                    }
                    if (hh + Sm::kEH >= 2) {   // this warp's last read of the slot
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S.t_empty[slot]);
                    }
                    if (!has) continue;
                    const int lim = min(64, d - 64 * b);   // channels of this block inside d
                    if (a.store_mode) {
                        if (valid) {
                            float* dst = num + (int64_t)g * d + 64 * b;
    #pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                if (i < lim) dst[i] = v0[i];
                                if (32 + i < lim) dst[32 + i] = v1[i];
                            }
                        }
                    } else {
                        // the row goes to shared memory (pitch 272 B: conflict-free) and the
                        // bulk-copy engine adds it into num[g, 64 b ..]
                        bulk_wait_read_all();   // the previous block's row has been read
    #pragma unroll
                        for (int c4 = 0; c4 < 16; ++c4) {
                            const float* src = c4 < 8 ? &v0[4 * c4] : &v1[4 * (c4 - 8)];
                            *reinterpret_cast<float4*>(st + 4 * c4) = make_float4(src[0], src[1], src[2], src[3]);
                        }
                        fence_proxy_async();   // generic writes, read by the bulk copy
                        if (valid && lim > 0) {
                            bulk_reduce_add_f32_hint(num + (int64_t)g * d + 64 * b, st, (uint32_t)lim * 4u,
                                                     num_policy);
                            bulk_commit();
                        }
                    }
                }
            }
            ub += U;
        }
    }
    bulk_wait_all();   // this thread's reductions into num are complete
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(S.tmem_base, 512);
}

// ------------------------------------------------------------ rendering (Eq. 4)
//
// F_hat[p, :] = sum_i w_i(p) f_i per 16x16 tile as the product
// F_hat_tile^T (128 channels x 256 pixels) = f_K^T (128 channels x K rows) W_K
// (K rows x 256 pixels) over the tile's weight rows K (its chunks): M = 128
// channels, N = 256 pixels, 16 rows per MMA, both operands MN-major in the
// 128-byte-swizzled layout (a W row segment of 64 pixels and an f row segment
// of 64 channels are each one 128-byte line).  float32 accuracy as in the
// aggregation: W = W1 + W2 and f = F1 + F2, products W1 F1 + W2 F1 + W1 F2.
//
// A plan pass first flattens every tile's chunk chain into its stages of 32
// weight rows ({first row, rows}, tile after tile), so that the kernel reads
// its work from indexed arrays instead of following the chain.
//
// One persistent CTA per SM takes the work units (view, tile, 128-channel
// block) blockIdx.x, blockIdx.x + gridDim.x, ...; the units of one tile are
// adjacent, so neighbouring CTAs read its weight rows at the same time (once
// from DRAM).  Stages flow through a ring of 4; each slot carries the stage's
// unit, rows and first/last flags in shared memory, so only the producer
// reads the plan:
//   warp 0      producer: the stage's info and Gaussian ids into shared
//               memory, then its rows of W1 and W2 by TMA (4 boxes of 64
//               pixels each);
//   warps 6-13  converters: each owns 4 rows of every stage, copies their f
//               segments (128 channels of the unit's block) with 16-byte
//               cp.async two stages ahead, 32 channels per 128-byte line, and
//               turns the float32 lines into F1 | F2 in place (rows past the
//               chunk and channels past d become zero); they also zero the W
//               lines of rows past the chunk;
//   warp 1      TMEM allocation and MMA issue, into one of two 256-column
//               accumulators (unit by unit, alternating);
//   warps 2-5   epilogue: TMEM lanes = channels, columns = pixels; 32 pixels
//               at a time are staged [pixel][channel] in shared memory and
//               written by one TMA store of 16 KB (many small stores from few
//               warps would be limited by requests in flight, not bandwidth);
//               the accumulator is released for the unit after next.
// Units of tiles without rows write zeros.  Bounded waits as in the aggregation.
struct RenderTcArgs {
    const uint32_t* stage_start;              // [nitems + 1]: the item's stages in `stages`
    const uint2* stages;                      // {first weight row, rows (1..32)}
    const uint32_t* chunk_gid;
    int ntiles, TX, width, height, d, nblk;   // nblk: 128-channel blocks
    int nwork;                                // (view, tile) items x nblk
    const float* f;                           // [n, d]
    float* out;                               // chunk's first view, [nv, H, W, d]
    int* status;
};

// Plan: stages per item (count pass), then the stages themselves (fill pass),
// one thread per item walking its chain.
__global__ void k_render_plan(const int* __restrict__ item_first, const int* __restrict__ chunk_rows,
                              const int* __restrict__ chunk_next, int cap, int nitems,
                              const uint32_t* __restrict__ start, uint32_t* __restrict__ count,
                              uint2* __restrict__ stages) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= nitems) {
        if (count && item == nitems) count[item] = 0u;
        return;
    }
    uint32_t k = start ? start[item] : 0u;
    for (int c = item_first[item]; c >= 0 && c < cap; c = chunk_next[c]) {
        const int rows = chunk_rows[c];
        for (int r = 0; r < rows; r += 32) {
            if (stages) stages[k] = make_uint2((uint32_t)(c * kCRows + r), (uint32_t)min(32, rows - r));
            ++k;
        }
    }
    if (count) count[item] = k;
}

constexpr int kRS = 4;                         // ring of stages of 32 weight rows
constexpr int kLook = 2;                       // stages of f rows in flight ahead of the one converted
constexpr int kRenderThreads = 448;            // 14 warps
constexpr uint32_t kRBox = 32 * 128;           // one box: 32 rows x 128 bytes
constexpr int kFirst = 1, kLast = 2, kEnd = 4; // stage flags

struct RenderSmem {
    uint8_t W[kRS][2][4 * kRBox];              // [stage][term][box of 64 pixels], offset 0 (1024-aligned)
    uint8_t F[kRS][4 * kRBox];                 // float32 boxes of 32 channels, then F1 (2 boxes) | F2 (2 boxes)
    float O[2][32 * 128];                      // output staging: 32 pixels x 128 channels, two buffers
    int4 info[kRS];                            // unit, rows, channels of the block, flags
    uint32_t gid[kRS][32];                     // the stage's Gaussian ids
    uint64_t meta[kRS], full[kRS], ready[kRS], empty[kRS];
    uint64_t t_full[2], t_empty[2];
    uint32_t tmem_base;
    int abort_flag;
    int epi_go;
};

constexpr size_t render_smem_bytes() { return sizeof(RenderSmem) + 1024; }
static_assert(render_smem_bytes() <= 232448, "shared memory");

// kind::f16 instruction descriptor: D float32, A and B bfloat16, both MN-major,
// M = 128, N = 256.
constexpr uint32_t kIdRender =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

// Bounded wait taken by every lane of a warp, with a warp-uniform outcome.
__device__ __forceinline__ bool warp_wait(volatile int* abort_flag, int* status, uint64_t* bar, uint32_t parity) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, parity));
    if (!ok && (threadIdx.x & 31) == 0) {
        *abort_flag = 1;
        atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
    }
    return ok;
}

__device__ __forceinline__ bool warp_aborted(volatile int* abort_flag) {
    return __shfl_sync(0xffffffffu, *abort_flag, 0) != 0;
}

__global__ void __launch_bounds__(kRenderThreads, 1)
    k_render_tc(RenderTcArgs a, const __grid_constant__ CUtensorMap wmap1, const __grid_constant__ CUtensorMap wmap2,
                const __grid_constant__ CUtensorMap omap) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    RenderSmem& S = *reinterpret_cast<RenderSmem*>(smem_raw + pad);
    volatile int* abort_flag = &S.abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < kRS; ++s) {
            mbar_init(&S.meta[s], 1);      // producer: info and ids written
            mbar_init(&S.full[s], 1);      // producer's arrival with the W bytes
            mbar_init(&S.ready[s], 8);     // the 8 converter warps
            mbar_init(&S.empty[s], 1);     // MMA commit
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&S.t_full[k], 1);    // MMA commit
            mbar_init(&S.t_empty[k], 4);   // the 4 epilogue warps
        }
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&S.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        // ---- producer (whole warp): per stage the info and the 32 Gaussian ids in
        // shared memory (meta), then the W rows by TMA (full).  The plan is read 32
        // stages per load, the next stage's ids one stage ahead.
        uint32_t it = 0;
        bool ok = true;
        for (int u = blockIdx.x; ok; u += gridDim.x) {
            const bool end = u >= a.nwork;
            const int item = end ? 0 : u / a.nblk, cb = end ? 0 : u - item * a.nblk;
            const int dv = min(128, a.d - 128 * cb);   // channels of the block inside d (a multiple of 8)
            const uint32_t k0 = end ? 0u : a.stage_start[item], k1 = end ? 1u : a.stage_start[item + 1];
            for (uint32_t kb = k0; kb < k1 && ok; kb += 32) {
                const uint2 rec = (!end && kb + lane < k1) ? a.stages[kb + lane] : make_uint2(0u, 0u);
                const int m = (int)min(32u, k1 - kb);
                // (shuffles outside any lane-dependent branch: every lane takes part)
                const uint32_t row00 = __shfl_sync(0xffffffffu, rec.x, 0);
                const int valid0 = (int)__shfl_sync(0xffffffffu, rec.y, 0);
                uint32_t gid = lane < valid0 ? a.chunk_gid[row00 + lane] : 0u;
                for (int j = 0; j < m; ++j, ++it) {
                    const uint32_t row0 = __shfl_sync(0xffffffffu, rec.x, j);
                    const int valid = (int)__shfl_sync(0xffffffffu, rec.y, j);
                    const int jn = j + 1 < m ? j + 1 : j;
                    const uint32_t row0n = __shfl_sync(0xffffffffu, rec.x, jn);
                    const int validn = (int)__shfl_sync(0xffffffffu, rec.y, jn);
                    const uint32_t gidn = (j + 1 < m && lane < validn) ? a.chunk_gid[row0n + lane] : 0u;
                    const uint32_t s = it % kRS;
                    if (warp_aborted(abort_flag) ||
                        (it >= (uint32_t)kRS && !warp_wait(abort_flag, a.status, &S.empty[s], ((it / kRS) - 1) & 1u))) {
                        ok = false;
                        break;
                    }
                    S.gid[s][lane] = lane < valid ? gid : 0u;
                    if (lane == 0) {
                        const int flags = end ? kEnd : ((kb + j == k0 ? kFirst : 0) | (kb + j + 1 == k1 ? kLast : 0));
                        S.info[s] = make_int4(u, valid, dv, flags);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        mbar_arrive(&S.meta[s]);
                        if (end) {
                            mbar_arrive(&S.full[s]);
                        } else {
                            mbar_expect_tx(&S.full[s], 2u * 4u * kRBox);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                tma_load_2d(S.W[s][0] + kRBox * q, &wmap1, &S.full[s], 64 * q, (int)row0);
                                tma_load_2d(S.W[s][1] + kRBox * q, &wmap2, &S.full[s], 64 * q, (int)row0);
                            }
                        }
                    }
                    gid = gidn;
                }
            }
            if (end) break;
        }
        if (lane == 0 && *abort_flag)   // let the copies already issued land (bounded)
            for (uint32_t k = (it > (uint32_t)kRS ? it - kRS : 0u); k < it; ++k)
                mbar_wait(&S.full[k % kRS], (k / kRS) & 1u);
    } else if (warp >= 6) {
        // ---- converters: warp cw owns rows 4 cw .. 4 cw + 3 of every stage; lane:
        // row p = 4 cw + lane / 8, o = lane % 8.  The warp copies its rows' f
        // segments itself (cp.async, kLook stages ahead: lane o copies channels
        // 4 (o + 8 m) .. + 3, m = 0..3, into float32 box m), then turns its
        // rows' float32 lines into F1 | F2 in place: chunks of 8 channels o and
        // 8 + o.  Every line a warp reads or writes belongs to its own rows, so
        // warp barriers order the copies, reads and writes.
        const int cw = warp - 6, p = 4 * cw + (lane >> 3), oc = lane & 7;
        uint32_t end_it = 0xffffffffu;   // stage index of the end record, once seen
        bool ok = true;
        // copies of stage k (after its info and ids are published); one cp.async group per stage
        auto issue = [&](uint32_t k) {
            if (k <= end_it && ok) {
                const uint32_t sk = k % kRS;
                if (warp_aborted(abort_flag) || !warp_wait(abort_flag, a.status, &S.meta[sk], (k / kRS) & 1u)) {
                    ok = false;
                } else {
                    const int4 inf = S.info[sk];
                    if (inf.w & kEnd) {
                        end_it = k;
                    } else if (p < inf.y) {
                        const int cbk = inf.x - (inf.x / a.nblk) * a.nblk;
                        const float* src = a.f + (size_t)S.gid[sk][p] * a.d + 128 * cbk + 4 * oc;
                        uint8_t* dst = S.F[sk] + p * 128 + oc * 16;
#pragma unroll
                        for (int mq = 0; mq < 4; ++mq)
                            if (4 * (oc + 8 * mq) < inf.z) cp_async_16(dst + kRBox * mq, src + 32 * mq);
                    }
                }
            }
            cp_async_commit();
        };
        for (uint32_t k = 0; k < (uint32_t)kLook; ++k) issue(k);
        for (uint32_t it = 0; ok; ++it) {
            issue(it + kLook);
            if (!ok) break;
            cp_async_wait<kLook>();   // this thread's copies of stage it have landed
            __syncwarp();             // and the warp's (its rows only)
            const uint32_t s = it % kRS;
            const int4 inf = S.info[s];
            if (!(inf.w & kEnd)) {
                const int valid = inf.y, dv = inf.z;
                uint8_t* base = S.F[s];
                float x[2][8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 64 * h + 8 * oc;   // first channel of the chunk
                    const uint8_t* line = base + kRBox * (c >> 5) + p * 128 + (c & 31) * 4;
                    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
                    if (p < valid && c < dv) {
                        lo = *reinterpret_cast<const float4*>(line);
                        hi = *reinterpret_cast<const float4*>(line + 16);
                    }
                    x[h][0] = lo.x;
                    x[h][1] = lo.y;
                    x[h][2] = lo.z;
                    x[h][3] = lo.w;
                    x[h][4] = hi.x;
                    x[h][5] = hi.y;
                    x[h][6] = hi.z;
                    x[h][7] = hi.w;
                }
                __syncwarp();   // the warp's lines are read before any is overwritten
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint4 f1, f2;
                    split8(x[h], f1, f2);
                    const int o = kRBox * h + p * 128 + ((oc ^ (p & 7)) << 4);
                    *reinterpret_cast<uint4*>(base + o) = f1;
                    *reinterpret_cast<uint4*>(base + 2 * kRBox + o) = f2;
                }
                if (valid < 32) {
                    // rows past the chunk: zero the W lines that the copy brought in
                    if (!warp_wait(abort_flag, a.status, &S.full[s], (it / kRS) & 1u)) break;
                    const int nz = (32 - valid) * 64;   // 16-byte pieces: rows x 2 terms x 4 boxes x 8
                    for (int e = 32 * cw + lane; e < nz; e += 256) {
                        const int row = valid + (e >> 6), rem = e & 63;
                        *reinterpret_cast<uint4*>(S.W[s][rem >> 5] + kRBox * ((rem >> 3) & 3) + row * 128 +
                                                  (rem & 7) * 16) = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
                fence_proxy_async();   // generic writes, read by the tensor core
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.ready[s]);
            if (inf.w & kEnd) break;
        }
        cp_async_wait<0>();   // no copy of this thread is left in flight
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: descriptors advance by plain adds (start address / 16
            // in bits 0-13); a 16-row step is 2048 bytes
            const uint64_t wd0 = sw128_desc(saddr(S.W[0][0]), kRBox, 1024);
            const uint64_t fd0 = sw128_desc(saddr(S.F[0]), kRBox, 1024);
            uint32_t it = 0, ks = 0;   // stages, units with stages
            bool ok = true;
            for (;; ++it) {
                const uint32_t s = it % kRS;
                if (*abort_flag || !agg_wait(abort_flag, a.status, &S.ready[s], (it / kRS) & 1u)) {
                    ok = false;
                    break;
                }
                const int4 inf = S.info[s];
                if (inf.w & kEnd) break;
                if (!agg_wait(abort_flag, a.status, &S.full[s], (it / kRS) & 1u)) {
                    ok = false;
                    break;
                }
                const uint32_t slot = ks & 1u;
                if ((inf.w & kFirst) && ks >= 2u &&
                    !agg_wait(abort_flag, a.status, &S.t_empty[slot], ((ks >> 1) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = S.tmem_base + 256u * slot;
                const uint64_t w1 = wd0 + ((s * sizeof(S.W[0])) >> 4), w2 = w1 + ((4 * kRBox) >> 4);
                const uint64_t f1 = fd0 + ((s * sizeof(S.F[0])) >> 4), f2 = f1 + ((2 * kRBox) >> 4);
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint32_t o = 128u * kk;
                    mma_bf16(dt, f1 + o, w1 + o, kIdRender, ((inf.w & kFirst) && kk == 0) ? 0u : 1u);
                    mma_bf16(dt, f1 + o, w2 + o, kIdRender, 1u);
                    mma_bf16(dt, f2 + o, w1 + o, kIdRender, 1u);
                }
                mma_commit(&S.empty[s]);
                if (inf.w & kLast) {
                    mma_commit(&S.t_full[slot]);
                    ++ks;
                }
            }
            if (!ok && it > 0)   // the MMAs issued complete in order (bounded)
                mbar_wait(&S.empty[(it - 1) % kRS], ((it - 1) / kRS) & 1u);
        }
    } else {
        // ---- epilogue (warps 2-5): warp w reads TMEM lanes 32 (w % 4) .. + 31 =
        // channels; 32 pixels at a time go to a staging buffer [pixel][128
        // channels] and out by one TMA store (2 tile rows x 16 pixels x 128
        // channels; the store leaves out what lies outside the image or past d).
        // Warp 2 lane 0 leads: it waits for the accumulator, issues the stores and
        // tracks their reads of the two staging buffers.
        const int qq = warp & 3;
        const bool lead = warp == 2 && lane == 0;
        uint32_t ks = 0;
        int u = blockIdx.x;
        bool has = false;
        if (u < a.nwork) {
            const int item = u / a.nblk;
            has = a.stage_start[item + 1] > a.stage_start[item];
        }
        for (; u < a.nwork; u += gridDim.x) {
            const int item = u / a.nblk, cb = u - item * a.nblk;
            bool has_next = false;   // the next unit's stage count, loaded ahead
            if (u + (int)gridDim.x < a.nwork) {
                const int itn = (u + (int)gridDim.x) / a.nblk;
                has_next = a.stage_start[itn + 1] > a.stage_start[itn];
            }
            const int v = item / a.ntiles, tile = item - v * a.ntiles;
            const int tx = tile % a.TX, ty = tile / a.TX;
            const uint32_t slot = ks & 1u;
            if (warp == 2) {
                bool go = true;
                if (has) go = warp_wait(abort_flag, a.status, &S.t_full[slot], (ks >> 1) & 1u);
                if (lane == 0) S.epi_go = go && !*abort_flag;
            }
            named_sync(1, 128);
            if (!S.epi_go) break;
            tc_fence_after();
            for (int gq = 0; gq < 8; ++gq) {   // pixels 32 gq .. 32 gq + 31: tile rows 2 gq, 2 gq + 1
                const int b = gq & 1;
                float val[32];
                if (has) {
                    tmem_ld32(S.tmem_base + ((uint32_t)(32 * qq) << 16) + 256u * slot + 32u * gq, val);
                    if (gq == 7) {   // the accumulator is free for the unit after next
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S.t_empty[slot]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) val[i] = 0.f;
                }
                if (lead) bulk_wait_read_1();   // the store of buffer b two rounds ago has read it
                named_sync(1, 128);
                float* ob = S.O[b] + 32 * qq + lane;
#pragma unroll
                for (int i = 0; i < 32; ++i) ob[128 * i] = val[i];
                fence_proxy_async();   // generic writes, read by the TMA store
                named_sync(1, 128);
                if (lead && ty * kTile + 2 * gq < a.height) {   // (no store for a box wholly below the image)
                    tma_store_4d(&omap, S.O[b], 128 * cb, tx * kTile, ty * kTile + 2 * gq, v);
                    bulk_commit();
                }
            }
            if (has) ++ks;
            has = has_next;
        }
        if (lead) bulk_wait_all();   // the stores are complete
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(S.tmem_base, 512);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    // looked up once per process (a function-local static is initialised by one thread)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
        return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }();
    return fn;
}

// Tensor map with 128-byte swizzle and zero fill out of bounds.
ludvig_status encode(CUtensorMap* map, CUtensorMapDataType type, const void* base, cuuint32_t rank,
                     const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box,
                     CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return LUDVIG_ERR_CUDA;
    }
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, type, rank, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return LUDVIG_ERR_CUDA;
    }
    return LUDVIG_OK;
}

// Tensor map over features [nv, H, W, d]: 64 (bfloat16) or 32 (float32)
// pixels of one view per box, 64 bfloat16 channels or 32 float32 channels (128-byte
// rows either way), zero fill outside the image and past d.
ludvig_status make_feature_map(CUtensorMap* map, const void* feats, int dtype, int nv, int width, int height,
                               int d) {
    const cuuint64_t es = dtype == LUDVIG_F32 ? 4 : (dtype == kDtypeE4M3 ? 1 : 2);
    cuuint64_t dims[4] = {(cuuint64_t)d, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)nv};
    cuuint64_t strides[3] = {(cuuint64_t)d * es, (cuuint64_t)width * d * es, (cuuint64_t)height * width * d * es};
    cuuint32_t box[4] = {(cuuint32_t)(128 / es), 16, dtype == LUDVIG_F32 ? 2u : 4u, 1};
    const CUtensorMapDataType t = dtype == LUDVIG_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : dtype == kDtypeE4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                        : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    return encode(map, t, feats, 4, dims, strides, box);
}

// Tensor map over rendered maps [nv, H, W, d] float32 for TMA stores: box of
// 128 channels x 16 pixels x 2 rows of one view, no swizzle.
ludvig_status make_out_map(CUtensorMap* map, float* out, int nv, int width, int height, int d) {
    cuuint64_t dims[4] = {(cuuint64_t)d, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)nv};
    cuuint64_t strides[3] = {(cuuint64_t)d * 4, (cuuint64_t)width * d * 4, (cuuint64_t)height * width * d * 4};
    cuuint32_t box[4] = {128, 16, 2, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, out, 4, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

// Tensor map over chunk rows [cap * 128, 256] bfloat16: box of 64 pixels x 32
// rows (a quarter of one K atom of a chunk).
ludvig_status make_w_map(CUtensorMap* map, const void* w, int64_t cap) {
    cuuint64_t dims[2] = {256, (cuuint64_t)cap * kCRows};
    cuuint64_t strides[1] = {(cuuint64_t)kRowBytes};
    cuuint32_t box[2] = {64, 32};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w, 2, dims, strides, box);
}

template <int DB, int NT, int CF>
ludvig_status launch_agg(const AggArgs& args, const CUtensorMap* maps, int grid, cudaStream_t st) {
    // set once per process; a function-local static is initialised by one thread
    static const cudaError_t configured = cudaFuncSetAttribute(
        k_aggregate_tc<DB, NT, CF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)agg_smem_bytes<NT, CF>());
    LV_CUDA(configured);
    k_aggregate_tc<DB, NT, CF>
        <<<grid, agg_threads<NT, CF>(), agg_smem_bytes<NT, CF>(), st>>>(args, maps[0], maps[1], maps[2]);
    LV_LAUNCH();
    return LUDVIG_OK;
}

template <int NT, int CF>
ludvig_status dispatch_agg_cf(const AggArgs& args, const CUtensorMap* maps, int grid, cudaStream_t st) {
    switch ((args.d + 63) / 64) {
        case 1: return launch_agg<1, NT, CF>(args, maps, grid, st);
        case 2: return launch_agg<2, NT, CF>(args, maps, grid, st);
        case 3: return launch_agg<3, NT, CF>(args, maps, grid, st);
        case 4: return launch_agg<4, NT, CF>(args, maps, grid, st);
        case 5: return launch_agg<5, NT, CF>(args, maps, grid, st);
        case 6: return launch_agg<6, NT, CF>(args, maps, grid, st);
        case 7: return launch_agg<7, NT, CF>(args, maps, grid, st);
        case 8: return launch_agg<8, NT, CF>(args, maps, grid, st);
        default: set_error("tensor-core path needs 32 <= d <= 512"); return LUDVIG_ERR_INTERNAL;
    }
}

template <int NT>
ludvig_status dispatch_agg(const AggArgs& args, const CUtensorMap* maps, int grid, cudaStream_t st) {
    if (NT == 2 && option_agg_config() == 1) return dispatch_agg_cf<2, 1>(args, maps, grid, st);
    return dispatch_agg_cf<NT, 0>(args, maps, grid, st);
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

// workspace names of the two buffer sets of the weight rows
const char* const kWsW1[2] = {"tc.w1.0", "tc.w1.1"};
const char* const kWsW2[2] = {"tc.w2.0", "tc.w2.1"};
const char* const kWsGid[2] = {"tc.chunk_gid.0", "tc.chunk_gid.1"};
const char* const kWsRows[2] = {"tc.chunk_rows.0", "tc.chunk_rows.1"};
const char* const kWsNext[2] = {"tc.chunk_next.0", "tc.chunk_next.1"};
const char* const kWsDen[2] = {"tc.chunk_den.0", "tc.chunk_den.1"};
const char* const kWsFirst[2] = {"tc.item_first.0", "tc.item_first.1"};
const char* const kWsCounter[2] = {"tc.counter.0", "tc.counter.1"};
const char* const kWsPlanOff[2] = {"tc.plan_off.0", "tc.plan_off.1"};
const char* const kWsPlan[2] = {"tc.plan.0", "tc.plan.1"};

ludvig_status tc_reserve(Arena& ws, int NT, int nitems, int64_t cap) {
    cap = std::max<int64_t>(cap, 3 * (int64_t)nitems);
    for (int p = 0; p < 2; ++p) {
        void* q;
        LV_TRY(ws.get(kWsCounter[p], sizeof(int), &q));
        LV_TRY(ws.get(kWsFirst[p], sizeof(int) * (size_t)nitems, &q));
        LV_TRY(ws.get(kWsW1[p], (size_t)cap * kChunkBytes, &q));
        if (NT == 2) LV_TRY(ws.get(kWsW2[p], (size_t)cap * kChunkBytes, &q));
        LV_TRY(ws.get(kWsGid[p], sizeof(uint32_t) * (size_t)cap * kCRows, &q));
        LV_TRY(ws.get(kWsRows[p], sizeof(int) * (size_t)cap, &q));
        LV_TRY(ws.get(kWsNext[p], sizeof(int) * (size_t)cap, &q));
        LV_TRY(ws.get(kWsDen[p], sizeof(float) * (size_t)cap * kCRows * NT, &q));
        LV_TRY(ws.get(kWsPlanOff[p], sizeof(uint32_t) * ((size_t)nitems + 1), &q));
        LV_TRY(ws.get(kWsPlan[p], sizeof(int2) * (size_t)cap, &q));
    }
    return LUDVIG_OK;
}

ludvig_status tc_weights(const GroupLists& L, int nv, int width, int height, int NT, Arena& ws, int parity,
                         int* status, int64_t* chunk_cap, bool checked, cudaStream_t st, TileWeights* tw) {
    const int p = parity & 1;
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int nitems = nv * TX * TY;
    TileWeights t;
    LV_TRY(ws.get(kWsCounter[p], 1, &t.counter));
    LV_TRY(ws.get(kWsFirst[p], (size_t)nitems, &t.ifirst));
    int* host = nullptr;   // [0] chunks used, [1] status
    if (checked) {
        void* hp;
        LV_TRY(ws.pinned("tc.host", 16, &hp));
        host = static_cast<int*>(hp);
    }
    int64_t cap = std::max<int64_t>(*chunk_cap, 3 * (int64_t)nitems);
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (cap > 0x7fffffff / kCRows) {
            set_error("tile weights need %lld chunks of 128 rows", (long long)cap);
            return LUDVIG_ERR_UNSUPPORTED;
        }
        LV_TRY(ws.get(kWsW1[p], (size_t)cap * kChunkBytes, &t.wg1));
        if (NT == 2) LV_TRY(ws.get(kWsW2[p], (size_t)cap * kChunkBytes, &t.wg2));
        LV_TRY(ws.get(kWsGid[p], (size_t)cap * kCRows, &t.cgid));
        LV_TRY(ws.get(kWsRows[p], (size_t)cap, &t.crows));
        LV_TRY(ws.get(kWsNext[p], (size_t)cap, &t.cnext));
        LV_TRY(ws.get(kWsDen[p], (size_t)cap * kCRows * NT, &t.cden));
        LV_CUDA(cudaMemsetAsync(t.counter, 0, sizeof(int), st));
        LV_CUDA(cudaMemsetAsync(t.ifirst, 0xff, sizeof(int) * (size_t)nitems, st));
        WeightsArgs w{};
        w.rank = L.rank;
        w.srec = L.srec;
        w.npad = L.npad;
        w.ranges = L.ranges;
        w.ntiles = TX * TY;
        w.TX = TX;
        w.width = width;
        w.height = height;
        w.wg1 = t.wg1;
        w.wg2 = NT == 2 ? t.wg2 : t.wg1;
        w.chunk_gid = t.cgid;
        w.chunk_rows = t.crows;
        w.chunk_next = t.cnext;
        w.item_first = t.ifirst;
        w.chunk_counter = t.counter;
        w.cap = (int)cap;
        w.chunk_den = t.cden;
        w.count_den = option_count_normalise() ? 1 : 0;
        const int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_WEIGHTS, st) : -1;
        if (NT == 2)
            k_weights<2, false><<<nitems, 256, 0, st>>>(w);
        else
            k_weights<1, false><<<nitems, 256, 0, st>>>(w);
        LV_LAUNCH();
        trace_end(tslot, st);
        if (!checked) break;
        LV_CUDA(cudaMemcpyAsync(host, t.counter, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaMemcpyAsync(host + 1, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        t.count = host[0];
        if (host[1] != 0) {
            set_error("tile weights: a bounded wait expired");
            return (ludvig_status)host[1];
        }
        if (t.count <= cap) break;
        // more chunks than kept: grow and run the weights again
        cap = (int64_t)t.count + t.count / 8 + 1;
    }
    if (checked && t.count > cap) {
        set_error("tile weights exceed the chunk capacity");
        return LUDVIG_ERR_INTERNAL;
    }
    // the aggregation's plan: every tile's non-empty chunks, flattened
    LV_TRY(ws.get(kWsPlanOff[p], (size_t)nitems + 1, &t.plan_off));
    LV_TRY(ws.get(kWsPlan[p], (size_t)cap, &t.plan));
    {
        const int pb = 256, pg = (nitems + 1 + pb - 1) / pb;
        k_agg_plan<<<pg, pb, 0, st>>>(t.ifirst, t.crows, t.cnext, (int)cap, nitems, nullptr, t.plan_off, nullptr);
        LV_LAUNCH();
        LV_TRY(scan_exclusive_u32(t.plan_off, t.plan_off, (int64_t)nitems + 1, nullptr, ws, st));
        k_agg_plan<<<pg, pb, 0, st>>>(t.ifirst, t.crows, t.cnext, (int)cap, nitems, t.plan_off, nullptr, t.plan);
        LV_LAUNCH();
    }
    t.cap = cap;
    *chunk_cap = cap;
    *tw = t;
    return LUDVIG_OK;
}

// The weights pass with direct accumulation for d <= kDirectMaxD channels:
// num (row stride num_stride) and den of each view take every row's
// contribution as the row is made, so no weight rows, chunk plan or
// aggregation launch exist for the group.  The chunk counter stays 0.
bool tc_direct_supported(int d) { return d >= 1 && d <= kDirectMaxD; }

ludvig_status tc_weights_direct(const GroupLists& L, int nv, int width, int height, int NT, int d, int num_stride,
                                const void* feats, int feat_dtype, const AggViews& av, Arena& ws, int parity,
                                int* status, bool checked, cudaStream_t st, int** counter) {
    if (!tc_direct_supported(d) || nv < 1 || nv > kMaxGroupViews) {
        set_error("direct accumulation takes 1 to %d channels and 1 to %d views", kDirectMaxD, kMaxGroupViews);
        return LUDVIG_ERR_INTERNAL;
    }
    const int p = parity & 1;
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int nitems = nv * TX * TY;
    int* cnt;
    LV_TRY(ws.get(kWsCounter[p], 1, &cnt));
    LV_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), st));
    WeightsArgs w{};
    w.rank = L.rank;
    w.srec = L.srec;
    w.npad = L.npad;
    w.ranges = L.ranges;
    w.ntiles = TX * TY;
    w.TX = TX;
    w.width = width;
    w.height = height;
    w.chunk_counter = cnt;
    w.count_den = option_count_normalise() ? 1 : 0;
    w.direct_d = d;
    w.num_stride = num_stride;
    w.feats = feats;
    w.feat_bf16 = feat_dtype == LUDVIG_BF16 ? 1 : 0;
    w.views = av;
    const int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_WEIGHTS, st) : -1;
    if (NT == 2)
        k_weights<2, true><<<nitems, 256, 0, st>>>(w);
    else
        k_weights<1, true><<<nitems, 256, 0, st>>>(w);
    LV_LAUNCH();
    trace_end(tslot, st);
    if (checked) {
        void* hp;
        LV_TRY(ws.pinned("tc.host", 16, &hp));
        int* host = static_cast<int*>(hp);
        LV_CUDA(cudaMemcpyAsync(host + 1, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        if (host[1] != 0) {
            set_error("tile weights: a bounded wait expired");
            return (ludvig_status)host[1];
        }
    }
    if (counter) *counter = cnt;
    return LUDVIG_OK;
}

ludvig_status tc_aggregate(const TileWeights& t, int nv, int width, int height, const void* feats, int fextent,
                           int dtype, int d, const AggViews& av, int* status, int* ovf, cudaStream_t st,
                           const float* scales) {
    const int NT = dtype == LUDVIG_F32 ? 2 : 1;
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int nitems = nv * TX * TY;
    if (nitems == 0 || t.count == 0) return LUDVIG_OK;
    int sms = 0;
    LV_TRY(sm_count(&sms));
    CUtensorMap maps[3];
    LV_TRY(make_w_map(&maps[0], t.wg1, t.cap));
    LV_TRY(make_w_map(&maps[1], NT == 2 ? t.wg2 : t.wg1, t.cap));
    LV_TRY(make_feature_map(&maps[2], feats, dtype, fextent, width, height, d));
    AggArgs g{};
    g.cap = (int)t.cap;
    g.chunk_rows = t.crows;
    g.chunk_next = t.cnext;
    g.item_first = t.ifirst;
    g.chunk_gid = t.cgid;
    g.chunk_den = t.cden;
    g.nitems = nitems;
    g.ntiles = TX * TY;
    g.TX = TX;
    g.d = d;
    g.status = status;
    g.store_mode = 0;
    g.chunk_count = t.count >= 0 ? nullptr : t.counter;   // a checked run already fits
    g.ovf = ovf;
    g.plan_off = t.plan_off;
    g.plan = t.plan;
    g.scales = scales;
    g.views = av;
    const int cap_sms = option_agg_sms();
    const int grid = std::min(cap_sms > 0 ? std::min(cap_sms, sms) : sms, nitems);
    StageScope agg_scope(LUDVIG_STAGE_AGGREGATE, st);
    if (dtype == kDtypeE4M3) return dispatch_agg_cf<1, 2>(g, maps, grid, st);
    if (NT == 2) return dispatch_agg<2>(g, maps, grid, st);
    return dispatch_agg<1>(g, maps, grid, st);
}

// Rendering F_hat = W f of a group on the tensor cores (Eq. 4): the weight
// rows of k_weights (float32 split in two bfloat16 terms), then the
// persistent k_render_tc over the (view, tile, 128-channel block) units.
ludvig_status tc_render(const TileWeights& t, Arena& ws, int nv, int width, int height, const float* f, int d,
                        float* out, int* status, cudaStream_t st) {
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int nitems = nv * TX * TY;
    if (nitems == 0) return LUDVIG_OK;
    if (t.count < 0) {
        set_error("render needs a checked weights pass");
        return LUDVIG_ERR_INTERNAL;
    }
    // plan: stages of every item (a chunk has at most 4 stages of 32 rows)
    uint32_t* start;
    uint2* stages;
    LV_TRY(ws.get("render.stage_start", (size_t)nitems + 1, &start));
    LV_TRY(ws.get("render.stages", (size_t)std::max(1, 4 * t.count), &stages));
    const int pb = 256, pg = (nitems + 1 + pb - 1) / pb;
    k_render_plan<<<pg, pb, 0, st>>>(t.ifirst, t.crows, t.cnext, (int)t.cap, nitems, nullptr, start, nullptr);
    LV_LAUNCH();
    LV_TRY(scan_exclusive_u32(start, start, (int64_t)nitems + 1, nullptr, ws, st));
    k_render_plan<<<pg, pb, 0, st>>>(t.ifirst, t.crows, t.cnext, (int)t.cap, nitems, start, nullptr, stages);
    LV_LAUNCH();
    CUtensorMap maps[3];
    LV_TRY(make_w_map(&maps[0], t.wg1, t.cap));
    LV_TRY(make_w_map(&maps[1], t.wg2, t.cap));
    LV_TRY(make_out_map(&maps[2], out, nv, width, height, d));
    RenderTcArgs r{};
    r.stage_start = start;
    r.stages = stages;
    r.chunk_gid = t.cgid;
    r.ntiles = TX * TY;
    r.TX = TX;
    r.width = width;
    r.height = height;
    r.d = d;
    r.nblk = (d + 127) / 128;
    r.nwork = nitems * r.nblk;
    r.f = f;
    r.out = out;
    r.status = status;
    // set once per process; a function-local static is initialised by one thread
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_render_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)render_smem_bytes());
    LV_CUDA(configured);
    int sms = 0;
    LV_TRY(sm_count(&sms));
    const int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_RENDER_PRODUCT, st) : -1;
    k_render_tc<<<std::min(sms, r.nwork), kRenderThreads, render_smem_bytes(), st>>>(r, maps[0], maps[1], maps[2]);
    LV_LAUNCH();
    trace_end(tslot, st);
    return LUDVIG_OK;
}

}  // namespace ludvig

using namespace ludvig;

namespace ludvig {
namespace {
// Failure-detection check: a bounded wait on an mbarrier that nothing arrives
// on expires, records LUDVIG_ERR_TIMEOUT and returns (the kernels' pattern).
__global__ void k_wait_timeout(long long budget, int* status, long long* waited) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long t0 = clock64();
    const bool ok = mbar_wait_for(&bar, 0u, budget);
    *waited = clock64() - t0;
    *status = ok ? (int)LUDVIG_OK : (int)LUDVIG_ERR_TIMEOUT;
    mbar_arrive(&bar);   // complete the phase so that nothing is left pending
}

// The same wait reporting into a status word the way the tensor-core kernels
// do (only an expiry writes it).
__global__ void k_wait_timeout_status(long long budget, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait_for(&bar, 0u, budget)) atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
    mbar_arrive(&bar);
}
}  // namespace

ludvig_status tc_wait_into_status(int64_t cycles, int* status, cudaStream_t st) {
    k_wait_timeout_status<<<1, 32, 0, st>>>((long long)cycles, status);
    LV_LAUNCH();
    return LUDVIG_OK;
}
}  // namespace ludvig

extern "C" ludvig_status ludvig_debug_wait_timeout(int64_t cycles, int64_t* waited, void* stream) {
    LV_ARG(cycles >= 0 && cycles <= 4000000000ll, "cycles must be in [0, 4e9]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct Out {
        int status;
        int pad;
        long long waited;
    };
    Out* d = nullptr;
    LV_CUDA(cudaMalloc(&d, sizeof(Out)));
    k_wait_timeout<<<1, 32, 0, st>>>((long long)cycles, &d->status, &d->waited);
    LV_LAUNCH();
    Out h{};
    const cudaError_t e1 = cudaMemcpyAsync(&h, d, sizeof(Out), cudaMemcpyDeviceToHost, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(d);
    LV_CUDA(e1);
    LV_CUDA(e2);
    if (waited) *waited = h.waited;
    if (h.status != LUDVIG_OK) set_error("bounded wait expired after %lld cycles", h.waited);
    return (ludvig_status)h.status;
}

extern "C" ludvig_status ludvig_debug_mma_bf16(const void* a, const void* f, int32_t d, float* out, void* stream) {
    LV_ARG(a != nullptr && f != nullptr && out != nullptr, "NULL argument");
    LV_ARG(d % 64 == 0 && d >= 64 && d <= 512, "d must be 64..512 in steps of 64");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // one chunk of 128 rows (row r -> output row r) over a single 16x16 tile
    struct Meta {
        int first, next, rows, status;
        uint32_t gid[kCRows];
        uint32_t off[2];
        int2 plan[1];
    };
    static Meta* meta = nullptr;
    if (!meta) LV_CUDA(cudaMalloc(&meta, sizeof(Meta)));
    static Meta h{};
    h.first = 0;
    h.next = -1;
    h.rows = kCRows;
    h.status = 0;
    for (int r = 0; r < kCRows; ++r) h.gid[r] = (uint32_t)r;
    h.off[0] = 0u;
    h.off[1] = 1u;
    h.plan[0] = make_int2(0, kCRows);
    LV_CUDA(cudaMemcpyAsync(meta, &h, sizeof(Meta), cudaMemcpyHostToDevice, st));
    CUtensorMap maps[3];
    LV_TRY(make_w_map(&maps[0], a, 1));
    maps[1] = maps[0];
    LV_TRY(make_feature_map(&maps[2], f, LUDVIG_BF16, 1, 16, 16, d));
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
    g.views.fview[0] = 0;
    g.views.num[0] = out;
    g.views.den[0] = nullptr;
    g.status = &meta->status;
    g.store_mode = 1;
    g.chunk_count = nullptr;
    g.ovf = nullptr;
    g.plan_off = meta->off;
    g.plan = meta->plan;
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
