// Tensor-core aggregation of the uplift (Sec. 3.2, Eq. 3):
// num[i,:] += sum_p w_i(p) F[p,:] per 16x16 tile as the dense product
// W_tile^T F_tile on the 5th-generation tensor cores, for bfloat16 features
// (NT = 1) and float32 features (NT = 2, float32-level accuracy).
//
// NT = 2: the float32 features are split beforehand into two bfloat16 arrays
// F = F1 + F2 (k_split_f32) and the weights into w = W1 + W2; the product keeps
// W1 F1 + W2 F1 + W1 F2 (16 significant bits per operand, the dropped W2 F2 and
// the residuals are below 2^-16 relative).  beta sums the same W terms, so each
// f_i stays a convex combination of the features.
//
// One persistent CTA per SM (8 warps = 256 pixels) takes (view, tile) items
// from an atomic counter.  For each item it
//   * walks the tile's depth-ordered list in batches of 32 Gaussians (float32
//     rules of Eq. 1: alpha, 1/255 skip, 1e-4 stop), one 8x4 pixel block per
//     warp, with the next batch's records and culling constants prefetched;
//   * appends every Gaussian with a non-zero weight in the tile as a row of a
//     128 x 256 W tile per term in shared memory (K-major, 128-byte swizzle);
//   * when the tile cannot take another batch (or the list ends) thread 0
//     streams the feature tile through a TMA ring (256 pixels x 64 channels
//     per stage, MN-major 128-byte swizzle, zero fill past the image and past
//     d) and issues tcgen05.mma (kind::f16, M = 128, N = 64, K = 16) into a
//     128 x 64*DB float32 accumulator in tensor memory;
//   * all warps read the accumulator back (tcgen05.ld) and add each row into
//     num with vector reductions.
// Every mbarrier wait is bounded: on expiry the kernel records
// LUDVIG_ERR_TIMEOUT, drains what it issued (bounded), frees tensor memory and
// returns.
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

constexpr int kTcThreads = 256;
constexpr int kTcRows = 128;                       // MMA M: Gaussians per W tile
constexpr int kTcBatch = 32;                       // Gaussians composited per step
constexpr uint32_t kWBytes = kTcRows * 256 * 2;    // 64 KB per bfloat16 term
constexpr uint32_t kFBlockBytes = 256 * 64 * 2;    // 32 KB: 256 pixels x 64 channels

template <int NT>
struct TcSmem {
    static constexpr int kStages = NT == 1 ? 4 : 2;
    uint8_t W[NT][kWBytes];                        // offset 0 (1024-aligned)
    uint8_t F[kStages][kFBlockBytes];              // 1024-aligned stages
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t mma_done;
    float4 ra[2][kTcBatch];                        // [buffer][j]
    float2 rb[2][kTcBatch];
    float4 rr[2][kTcBatch];                        // culling constants: thr, 1/a, 1/c, possible
    uint32_t gid[2][kTcBatch];
    uint32_t row_gid[kTcRows];
    uint32_t rowmask[2];
    uint32_t tmem_base;
    int item;
    int abort_flag;
};

template <int NT>
constexpr size_t tc_smem_bytes() {
    return sizeof(TcSmem<NT>) + 1024;   // + alignment slack
}

// kind::f16 instruction descriptor: D float32, A and B bfloat16, A K-major,
// B MN-major, M = 128, N = 64.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((64u >> 3) << 17) |
                            ((128u >> 4) << 24);

// Byte offset of element (row r, pixel k) in the K-major 128-byte-swizzled
// W tile: four 64-pixel atoms of 128 rows x 128 bytes, 16-byte chunks XORed
// with the row index mod 8.
__device__ __forceinline__ uint32_t w_offset(int r, int k) {
    const int ka = k >> 6, kk = k & 63;
    return (uint32_t)(ka * (kTcRows * 128) + r * 128 + ((((kk >> 3) ^ (r & 7))) << 4) + ((kk & 7) << 1));
}

struct TcArgs {
    const float4* rec_a;
    const float2* rec_b;
    int64_t n;
    const uint2* ranges;
    const uint32_t* list;
    int ntiles, TX, width, height, d, nitems;
    float* num;
    float* den;
    int* counter;     // work-queue head (zeroed before launch)
    int* status;      // LUDVIG_OK or LUDVIG_ERR_TIMEOUT
    int store_mode;   // debug GEMM: plain stores of the accumulator, no list
};

template <int NT>
__device__ __forceinline__ void fail(TcSmem<NT>& S, int* status) {
    S.abort_flag = 1;
    atomicExch(status, (int)LUDVIG_ERR_TIMEOUT);
}

// TMA loads + MMA issue for one W tile (thread 0 only).  `fcount` counts the
// feature blocks loaded so far (ring position); false on a timed-out wait.
template <int DB, int NT>
__device__ bool issue_tile(TcSmem<NT>& S, const CUtensorMap* f1, const CUtensorMap* f2, uint32_t& fcount, int tx,
                           int ty, int v) {
    constexpr int kS = TcSmem<NT>::kStages;
    constexpr int kLoads = DB * NT;   // F1 block cb, then F2 block cb (NT = 2)
    auto issue = [&](int l) -> bool {
        const uint32_t k = fcount + l, s = k % kS;
        if (k >= (uint32_t)kS && !mbar_wait(&S.empty[s], ((k / kS) - 1) & 1u)) return false;
        mbar_expect_tx(&S.full[s], kFBlockBytes);
        const int cb = l / NT, term = l % NT;
        tma_load_4d(S.F[s], term == 0 ? f1 : f2, &S.full[s], 64 * cb, tx * kTile, ty * kTile, v);
        return true;
    };
    for (int l = 0; l < kLoads && l < kS; ++l)
        if (!issue(l)) return false;
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    for (int l = 0; l < kLoads; ++l) {
        const uint32_t k = fcount + l, s = k % kS;
        const int cb = l / NT, term = l % NT;
        if (!mbar_wait(&S.full[s], (k / kS) & 1u)) return false;
        tc_fence_after();
        const uint32_t f_base = saddr(S.F[s]);
        // term 0 (F1): W1 F1 (+ W2 F1); term 1 (F2): W1 F2
#pragma unroll
        for (int ks = 0; ks < 16; ++ks) {
            const uint64_t bd = sw128_desc(f_base + ks * 2048, 1024, 1024);
            const uint32_t koff = (ks >> 2) * (kTcRows * 128) + (ks & 3) * 32;
            const uint32_t acc = (ks > 0 || term > 0) ? 1u : 0u;
            mma_bf16(tmem + 64 * cb, sw128_desc(saddr(S.W[0]) + koff, 16, 1024), bd, kIdesc, acc);
            if (NT == 2 && term == 0)
                mma_bf16(tmem + 64 * cb, sw128_desc(saddr(S.W[NT - 1]) + koff, 16, 1024), bd, kIdesc, 1u);
        }
        mma_commit(&S.empty[s]);
        // refill the stage of the previous load (its MMAs are queued ahead)
        if (l >= 1 && l - 1 + kS < kLoads)
            if (!issue(l - 1 + kS)) return false;
    }
    mma_commit(&S.mma_done);
    fcount += kLoads;
    return true;
}

// Flush of the W tile rows [0, nrows): MMA over every channel block, then the
// accumulator rows are added into num (or stored, in debug mode).  All threads.
template <int DB, int NT>
__device__ __noinline__ void flush_tile(TcSmem<NT>& S, const TcArgs& a, const CUtensorMap* f1,
                                        const CUtensorMap* f2, int nrows, uint32_t& fcount, uint32_t& mma_phase,
                                        int tx, int ty, int v) {
    fence_proxy_async();   // W written with generic stores, read by the tensor core
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0 && !issue_tile<DB, NT>(S, f1, f2, fcount, tx, ty, v)) fail(S, a.status);
    __syncthreads();
    if (S.abort_flag) return;
    if (!mbar_wait(&S.mma_done, mma_phase)) fail(S, a.status);
    mma_phase ^= 1u;
    __syncthreads();
    if (S.abort_flag) return;
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    const int units = 2 * DB, u0 = half ? units / 2 : 0, u1 = half ? units : units / 2;
    const int r = 32 * q + lane;
    const bool valid = r < nrows;
    const uint32_t g = valid ? S.row_gid[r] : 0u;
    const int d = a.d;
    for (int u = u0; u < u1; ++u) {
        float val[32];
        tmem_ld32(S.tmem_base + ((uint32_t)(32 * q) << 16) + 32 * u, val);
        if (valid) {
            float* dst = a.num + (int64_t)g * d + 32 * u;
            if (a.store_mode) {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (32 * u + i < d) dst[i] = val[i];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (32 * u + 4 * i < d)
                        red_add_v4(dst + 4 * i, val[4 * i], val[4 * i + 1], val[4 * i + 2], val[4 * i + 3]);
            }
        }
    }
    if (!a.store_mode && tid < nrows) {
        // beta partial of row tid: the sum of its W terms over the 256 pixels
        float sden = 0.f;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint8_t* row = S.W[t] + tid * 128;
#pragma unroll 4
            for (int ka = 0; ka < 4; ++ka) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 v4 = *reinterpret_cast<const uint4*>(row + ka * (kTcRows * 128) + c * 16);
                    const uint32_t wv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        sden += __uint_as_float(wv[e] << 16);
                        sden += __uint_as_float(wv[e] & 0xffff0000u);
                    }
                }
            }
        }
        atomicAdd(a.den + S.row_gid[tid], sden);
    }
    tc_fence_before();
    __syncthreads();
    // the MMA has read the W tiles: clear them for the next rows
    for (int t = 0; t < NT; ++t) {
        uint4* w4 = reinterpret_cast<uint4*>(S.W[t]);
        for (int e = tid; e < (int)(kWBytes / 16); e += kTcThreads) w4[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
}

template <int DB, int NT>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_composite_tc(TcArgs a, const __grid_constant__ CUtensorMap fmap1, const __grid_constant__ CUtensorMap fmap2) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    TcSmem<NT>& S = *reinterpret_cast<TcSmem<NT>*>(smem_raw + pad);
    constexpr int kS = TcSmem<NT>::kStages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;

    if (tid == 0) {
        for (int s = 0; s < kS; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.mma_done, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&S.tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    uint32_t fcount = 0, mma_phase = 0;
    for (int t = 0; t < NT; ++t) {
        uint4* w4 = reinterpret_cast<uint4*>(S.W[t]);
        for (int e = tid; e < (int)(kWBytes / 16); e += kTcThreads) w4[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();

    if (a.store_mode) {
        // debug GEMM: W rows come from a.list reinterpreted as bf16 [128][256]
        const __nv_bfloat16* Ain = reinterpret_cast<const __nv_bfloat16*>(a.list);
        for (int e = tid; e < kTcRows * 256; e += kTcThreads) {
            const int r = e >> 8, k = e & 255;
            *reinterpret_cast<__nv_bfloat16*>(S.W[0] + w_offset(r, k)) = Ain[e];
        }
        if (tid < kTcRows) S.row_gid[tid] = tid;
        flush_tile<DB, NT>(S, a, &fmap1, &fmap2, kTcRows, fcount, mma_phase, 0, 0, 0);
    } else {
        // warp w covers the 8x4 pixel block ((w & 1) * 8, (w >> 1) * 4) of the tile
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
            if (tid < kTcBatch && range.x + tid < range.y) {
                const uint32_t g0 = a.list[range.x + tid];
                const float4 ra = rec_a[g0];
                const float2 rb = rec_b[g0];
                const Reach R = reach_prep(ra.z, ra.w, rb.x, rb.y);
                S.gid[0][tid] = g0;
                S.ra[0][tid] = ra;
                S.rb[0][tid] = rb;
                S.rr[0][tid] = make_float4(R.thr, R.inv_ca, R.inv_cc, R.possible ? 1.f : 0.f);
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
            for (uint32_t b0 = range.x; b0 < range.y; b0 += kTcBatch, buf ^= 1) {
                if (__syncthreads_count(!done) == 0) break;
                // room for up to 32 new rows, before any weight is live in registers
                if (nrows + kTcBatch > kTcRows) {
                    flush_tile<DB, NT>(S, a, &fmap1, &fmap2, nrows, fcount, mma_phase, tx, ty, v);
                    nrows = 0;
                    if (S.abort_flag) break;
                }
                const int cnt = (int)min((uint32_t)kTcBatch, range.y - b0);
                // prefetch the next batch's records (stored at the end of this batch)
                const uint32_t nb0 = b0 + kTcBatch;
                const bool pf = tid < kTcBatch && nb0 + tid < range.y;
                uint32_t pg = 0;
                float4 pra = make_float4(0.f, 0.f, 0.f, 0.f);
                float2 prb = make_float2(0.f, 0.f);
                if (pf) {
                    pg = a.list[nb0 + tid];
                    pra = rec_a[pg];
                    prb = rec_b[pg];
                }
                // Gaussians of the batch that can reach this warp's pixel block
                const bool warp_active = __any_sync(0xffffffffu, !done);
                uint32_t lm = 0u;   // this lane's non-zero weights (bit j = Gaussian j)
                float w[kTcBatch];
#pragma unroll
                for (int j = 0; j < kTcBatch; ++j) w[j] = 0.f;
                if (warp_active) {
                    bool rr = false;
                    if (lane < cnt) {
                        const float4 ra = S.ra[buf][lane];
                        const float2 rb = S.rb[buf][lane];
                        const float4 c4 = S.rr[buf][lane];
                        Reach R;
                        R.thr = c4.x;
                        R.inv_ca = c4.y;
                        R.inv_cc = c4.z;
                        R.possible = c4.w != 0.f;
                        R.cb2 = __fmul_rn(2.0f, ra.w);
                        rr = reaches_rect(R, ra.x, ra.y, ra.z, ra.w, rb.x, bxa, bxa + 7.0f, bya, bya + 3.0f);
                    }
                    const uint32_t rel = __ballot_sync(0xffffffffu, rr);
                    // alphas first (independent chains), then the transmittance recursion
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        if ((rel >> j) & 1u) {
                            const float4 ra = S.ra[buf][j];
                            const float2 rb = S.rb[buf][j];
                            w[j] = alpha_at(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, pxf, pyf);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        const float al = w[j];
                        w[j] = 0.f;
                        if (al > 0.f && !done) {
                            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
                            if (Tn < kTransMin) {
                                done = true;
                            } else {
                                w[j] = __fmul_rn(al, T);
                                T = Tn;
                                lm |= 1u << j;
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
                if (lm) {
                    // only non-zero weights are written: the W tiles are cleared after each flush
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        if ((lm >> j) & 1u) {
                            const int slot = nrows + __popc(rowmask & ((1u << j) - 1u));
                            const uint32_t o = w_offset(slot, pix);
                            const __nv_bfloat16 h1 = __float2bfloat16_rn(w[j]);
                            *reinterpret_cast<__nv_bfloat16*>(S.W[0] + o) = h1;
                            if (NT == 2)
                                *reinterpret_cast<__nv_bfloat16*>(S.W[NT - 1] + o) =
                                    __float2bfloat16_rn(w[j] - __bfloat162float(h1));
                        }
                    }
                }
                if (tid < kTcBatch && ((rowmask >> tid) & 1u))
                    S.row_gid[nrows + __popc(rowmask & lt_mask)] = S.gid[buf][tid];
                nrows += nnew;
                if (pf) {
                    const Reach R = reach_prep(pra.z, pra.w, prb.x, prb.y);
                    S.gid[buf ^ 1][tid] = pg;
                    S.ra[buf ^ 1][tid] = pra;
                    S.rb[buf ^ 1][tid] = prb;
                    S.rr[buf ^ 1][tid] = make_float4(R.thr, R.inv_ca, R.inv_cc, R.possible ? 1.f : 0.f);
                }
                // no barrier here: the next batch's counting barrier orders these stores
            }
            if (S.abort_flag) break;
            if (nrows > 0) flush_tile<DB, NT>(S, a, &fmap1, &fmap2, nrows, fcount, mma_phase, tx, ty, v);
            if (S.abort_flag) break;
            __syncthreads();   // every thread has read S.item before thread 0 takes the next one
        }
    }
    __syncthreads();
    if (S.abort_flag && tid == 0) mbar_wait(&S.mma_done, mma_phase);   // drain (bounded)
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

// Tensor map over features [nv, H, W, d] bfloat16: box of 64 channels x 16 x 16
// pixels of one view, 128-byte swizzle, zero fill outside the image and past d.
ludvig_status make_feature_map(CUtensorMap* map, const void* feats, int nv, int width, int height, int d) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return LUDVIG_ERR_CUDA;
    }
    cuuint64_t dims[4] = {(cuuint64_t)d, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)nv};
    cuuint64_t strides[3] = {(cuuint64_t)d * 2, (cuuint64_t)width * d * 2, (cuuint64_t)height * width * d * 2};
    cuuint32_t box[4] = {64, 16, 16, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(feats), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return LUDVIG_ERR_CUDA;
    }
    return LUDVIG_OK;
}

template <int DB, int NT>
ludvig_status launch_tc(const TcArgs& args, const CUtensorMap& m1, const CUtensorMap& m2, int grid, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        LV_CUDA(cudaFuncSetAttribute(k_composite_tc<DB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes<NT>()));
        configured = true;
    }
    k_composite_tc<DB, NT><<<grid, kTcThreads, tc_smem_bytes<NT>(), st>>>(args, m1, m2);
    LV_LAUNCH();
    return LUDVIG_OK;
}

template <int NT>
ludvig_status dispatch_tc(const TcArgs& args, const CUtensorMap& m1, const CUtensorMap& m2, int grid,
                          cudaStream_t st) {
    switch ((args.d + 63) / 64) {
        case 1: return launch_tc<1, NT>(args, m1, m2, grid, st);
        case 2: return launch_tc<2, NT>(args, m1, m2, grid, st);
        case 3: return launch_tc<3, NT>(args, m1, m2, grid, st);
        case 4: return launch_tc<4, NT>(args, m1, m2, grid, st);
        case 5: return launch_tc<5, NT>(args, m1, m2, grid, st);
        case 6: return launch_tc<6, NT>(args, m1, m2, grid, st);
        case 7: return launch_tc<7, NT>(args, m1, m2, grid, st);
        case 8: return launch_tc<8, NT>(args, m1, m2, grid, st);
        default: set_error("tensor-core path needs 32 <= d <= 512"); return LUDVIG_ERR_INTERNAL;
    }
}

}  // namespace

// Tensor-core aggregation applies to d in [32, 512] with d % 8 == 0 (16-byte
// rows for TMA); bfloat16 features always, float32 unless disabled.
bool tc_supported(int dtype, int d) {
    return (dtype == LUDVIG_BF16 || dtype == LUDVIG_F32) && d >= 32 && d <= 512 && d % 8 == 0;
}

// Composite + tensor-core aggregation of one chunk of views (stage 6 of the
// uplift pipeline).  `status` receives LUDVIG_ERR_TIMEOUT if a wait expired.
ludvig_status composite_tc(const float4* rec_a, const float2* rec_b, int64_t n, const uint2* ranges,
                           const uint32_t* list, int nv, int width, int height, const void* feats, int dtype, int d,
                           float* num, float* den, Arena& ws, int* status, cudaStream_t st) {
    CUtensorMap m1, m2;
    const void* f1 = feats;
    const void* f2 = feats;
    int dev = 0, sms = 148;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dtype == LUDVIG_F32) {
        // split the chunk's float32 features into two bfloat16 arrays
        const int64_t count = (int64_t)nv * width * height * d;
        void *hi, *lo;
        LV_TRY(ws.get("tc.f_hi", (size_t)count * 2, &hi));
        LV_TRY(ws.get("tc.f_lo", (size_t)count * 2, &lo));
        k_split_f32<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(count / 4, 256))), 256,
                      0, st>>>(static_cast<const float4*>(feats), static_cast<uint2*>(hi), static_cast<uint2*>(lo),
                               count / 4);
        LV_LAUNCH();
        f1 = hi;
        f2 = lo;
    }
    LV_TRY(make_feature_map(&m1, f1, nv, width, height, d));
    LV_TRY(make_feature_map(&m2, f2, nv, width, height, d));
    int* counter;
    LV_TRY(ws.get("tc.counter", 1, &counter));
    LV_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    TcArgs a;
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
    a.num = num;
    a.den = den;
    a.counter = counter;
    a.status = status;
    a.store_mode = 0;
    const int grid = std::min(sms, a.nitems);
    if (dtype == LUDVIG_F32) return dispatch_tc<2>(a, m1, m2, grid, st);
    return dispatch_tc<1>(a, m1, m2, grid, st);
}

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_debug_mma_bf16(const void* a, const void* f, int32_t d, float* out, void* stream) {
    LV_ARG(a != nullptr && f != nullptr && out != nullptr, "NULL argument");
    LV_ARG(d % 64 == 0 && d >= 64 && d <= 512, "d must be 64..512 in steps of 64");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUtensorMap map;
    LV_TRY(make_feature_map(&map, f, 1, 16, 16, d));
    static int* status = nullptr;
    if (!status) LV_CUDA(cudaMalloc(&status, sizeof(int)));
    LV_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    TcArgs args{};
    args.list = static_cast<const uint32_t*>(a);
    args.d = d;
    args.num = out;
    args.status = status;
    args.store_mode = 1;
    LV_TRY(dispatch_tc<1>(args, map, map, 1, st));
    int h = 0;
    LV_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        set_error("tensor-core kernel reported status %d", h);
        return (ludvig_status)h;
    }
    return LUDVIG_OK;
}
