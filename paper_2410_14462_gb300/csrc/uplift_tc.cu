// Tensor-core aggregation for bfloat16 features (the precision form of the
// uplift, Sec. 3.2 Eq. 3): num[i,:] += sum_p w_i(p) F[p,:] computed per 16x16
// tile as the dense product W_tile^T F_tile on the 5th-generation tensor cores.
//
// One persistent CTA per SM (8 warps = 256 pixels) takes (view, tile) items
// from an atomic counter and, for each item:
//   * walks the tile's depth-ordered list in batches of 32 Gaussians (the same
//     float32 rules as the CUDA-core path: alpha, 1/255 skip, 1e-4 stop);
//   * appends every Gaussian with a non-zero weight in the tile as one row of
//     a 128 x 256 bfloat16 W tile in shared memory (K-major, 128-byte
//     swizzle); beta_i sums the same bfloat16-rounded weights, so each f_i stays
//     a convex combination of the features;
//   * when the W tile is full (or the list ends) one thread streams the tile's
//     features channel block by channel block (256 pixels x 64 channels, TMA,
//     4-stage ring, MN-major 128-byte swizzle) and issues tcgen05.mma
//     (kind::f16, M=128, N=64, K=16) into a 128 x D float32 accumulator in
//     tensor memory;
//   * all warps read the accumulator back (tcgen05.ld) and add each Gaussian's
//     row into num with vector reductions.
// Every mbarrier wait is bounded; on expiry the kernel records
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
constexpr int kTcStages = 4;                       // feature channel-block ring
constexpr int kTcBatch = 32;                       // Gaussians composited per step
constexpr uint32_t kWBytes = kTcRows * 256 * 2;    // 64 KB
constexpr uint32_t kFBlockBytes = 256 * 64 * 2;    // 32 KB: 256 pixels x 64 channels

struct TcSmem {
    uint8_t W[kWBytes];                            // offset 0 (1024-aligned)
    uint8_t F[kTcStages][kFBlockBytes];            // 1024-aligned stages
    uint64_t full[kTcStages];
    uint64_t empty[kTcStages];
    uint64_t mma_done;
    float4 ra[kTcBatch];
    float2 rb[kTcBatch];
    uint32_t gid[kTcBatch];
    uint32_t row_gid[kTcRows];
    float row_den[kTcRows];
    float denpart[8][kTcBatch];
    uint32_t rowmask;
    uint32_t tmem_base;
    int item;
    int abort_flag;
};

constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;   // + alignment slack

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

// Producer + MMA issue for one W tile (thread 0 only).  Returns false on a
// timed-out wait.
template <int DB>
__device__ bool issue_tile(TcSmem& S, const CUtensorMap* fmap, uint32_t& fcount, int tx, int ty, int v) {
    const uint32_t w_base = saddr(S.W);
    const uint32_t tmem = S.tmem_base;
    auto issue = [&](int cb) -> bool {
        const uint32_t k = fcount + cb, s = k % kTcStages;
        if (k >= (uint32_t)kTcStages && !mbar_wait(&S.empty[s], ((k / kTcStages) - 1) & 1u)) return false;
        mbar_expect_tx(&S.full[s], kFBlockBytes);
        tma_load_4d(S.F[s], fmap, &S.full[s], 64 * cb, tx * kTile, ty * kTile, v);
        return true;
    };
    for (int cb = 0; cb < DB && cb < kTcStages; ++cb)
        if (!issue(cb)) return false;
    tc_fence_after();
    for (int cb = 0; cb < DB; ++cb) {
        const uint32_t k = fcount + cb, s = k % kTcStages;
        if (!mbar_wait(&S.full[s], (k / kTcStages) & 1u)) return false;
        tc_fence_after();
        const uint32_t f_base = saddr(S.F[s]);
#pragma unroll
        for (int ks = 0; ks < 16; ++ks) {
            const uint64_t ad = sw128_desc(w_base + (ks >> 2) * (kTcRows * 128) + (ks & 3) * 32, 16, 1024);
            const uint64_t bd = sw128_desc(f_base + ks * 2048, 1024, 1024);
            mma_bf16(tmem + 64 * cb, ad, bd, kIdesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&S.empty[s]);
        // refill the stage of the previous block (its MMAs are queued ahead)
        if (cb >= 1 && cb - 1 + kTcStages < DB)
            if (!issue(cb - 1 + kTcStages)) return false;
    }
    mma_commit(&S.mma_done);
    fcount += DB;
    return true;
}

// Flush of the W tile: MMA over all channel blocks, then read back the
// accumulator rows [0, nrows) and add them into num (or store them in debug
// mode).  Called by all threads.
template <int DB>
__device__ void flush_tile(TcSmem& S, const TcArgs& a, const CUtensorMap* fmap, int nrows, uint32_t& fcount,
                           uint32_t& mma_phase, int tx, int ty, int v) {
    fence_proxy_async();   // W written with generic stores, read by the tensor core
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        if (!issue_tile<DB>(S, fmap, fcount, tx, ty, v)) {
            S.abort_flag = 1;
            atomicExch(a.status, (int)LUDVIG_ERR_TIMEOUT);
        }
    }
    __syncthreads();
    if (S.abort_flag) return;
    if (!mbar_wait(&S.mma_done, mma_phase)) {
        S.abort_flag = 1;
        atomicExch(a.status, (int)LUDVIG_ERR_TIMEOUT);
    }
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
                for (int i = 0; i < 32; ++i) dst[i] = val[i];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) red_add_v4(dst + 4 * i, val[4 * i], val[4 * i + 1], val[4 * i + 2], val[4 * i + 3]);
            }
        }
    }
    if (!a.store_mode && tid < nrows) atomicAdd(a.den + S.row_gid[tid], S.row_den[tid]);
    tc_fence_before();
    __syncthreads();
}

template <int DB>
__global__ void __launch_bounds__(kTcThreads, 1) k_composite_tc(TcArgs a, const __grid_constant__ CUtensorMap fmap) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t pad = (1024u - (saddr(smem_raw) & 1023u)) & 1023u;
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw + pad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;

    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
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

    if (a.store_mode) {
        // debug GEMM: W rows come from a.num's companion buffer a.list (bf16 [128][256])
        const __nv_bfloat16* Ain = reinterpret_cast<const __nv_bfloat16*>(a.list);
        for (int e = tid; e < kTcRows * 256; e += kTcThreads) {
            const int r = e >> 8, k = e & 255;
            *reinterpret_cast<__nv_bfloat16*>(S.W + w_offset(r, k)) = Ain[e];
        }
        if (tid < kTcRows) S.row_gid[tid] = tid;
        flush_tile<DB>(S, a, &fmap, kTcRows, fcount, mma_phase, 0, 0, 0);
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
            float T = 1.0f;
            bool done = !inside;
            int nrows = 0;
            for (uint32_t b0 = range.x; b0 < range.y; b0 += kTcBatch) {
                if (__syncthreads_count(!done) == 0) break;
                const int cnt = (int)min((uint32_t)kTcBatch, range.y - b0);
                if (tid < cnt) {
                    const uint32_t g = a.list[b0 + tid];
                    S.gid[tid] = g;
                    S.ra[tid] = rec_a[g];
                    S.rb[tid] = rec_b[g];
                }
                if (tid == 0) S.rowmask = 0u;
                __syncthreads();
                uint32_t rel;
                {
                    bool rr = false;
                    if (lane < cnt) {
                        const float4 ra = S.ra[lane];
                        const float2 rb = S.rb[lane];
                        rr = reaches_rect(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, bxa, bxa + 7.0f, bya, bya + 3.0f);
                    }
                    rel = __ballot_sync(0xffffffffu, rr);
                    if (!__any_sync(0xffffffffu, !done)) rel = 0u;
                }
                float w[kTcBatch];
#pragma unroll
                for (int j = 0; j < kTcBatch; ++j) {
                    w[j] = 0.f;
                    if (((rel >> j) & 1u) && !done) {
                        const float4 ra = S.ra[j];
                        const float2 rb = S.rb[j];
                        const float al = alpha_at(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, pxf, pyf);
                        if (al > 0.f) {
                            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
                            if (Tn < kTransMin) {
                                done = true;
                            } else {
                                w[j] = __bfloat162float(__float2bfloat16_rn(__fmul_rn(al, T)));
                                T = Tn;
                            }
                        }
                    }
                }
                // Gaussians with a non-zero weight somewhere in the tile, and their
                // per-warp weight sums (beta uses the same rounded weights)
                uint32_t mine = 0u;
#pragma unroll
                for (int j = 0; j < kTcBatch; ++j) {
                    const uint32_t m = __ballot_sync(0xffffffffu, w[j] != 0.f);
                    float sj = 0.f;
                    if (m) {
                        mine |= 1u << j;
                        sj = w[j];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
                    }
                    if (lane == 0) S.denpart[warp][j] = sj;
                }
                if (lane == 0 && mine) atomicOr(&S.rowmask, mine);
                __syncthreads();
                const uint32_t rowmask = S.rowmask;
                const int nnew = __popc(rowmask);
                if (nnew) {
                    if (nrows + nnew > kTcRows) {
                        flush_tile<DB>(S, a, &fmap, nrows, fcount, mma_phase, tx, ty, v);
                        nrows = 0;
                        if (S.abort_flag) break;
                    }
#pragma unroll
                    for (int j = 0; j < kTcBatch; ++j) {
                        if ((rowmask >> j) & 1u) {
                            const int slot = nrows + __popc(rowmask & ((1u << j) - 1u));
                            *reinterpret_cast<__nv_bfloat16*>(S.W + w_offset(slot, pix)) = __float2bfloat16_rn(w[j]);
                        }
                    }
                    if (tid < kTcBatch && ((rowmask >> tid) & 1u)) {
                        const int slot = nrows + __popc(rowmask & lt_mask);
                        float s = 0.f;
#pragma unroll
                        for (int wi = 0; wi < 8; ++wi) s += S.denpart[wi][tid];
                        S.row_gid[slot] = S.gid[tid];
                        S.row_den[slot] = s;
                    }
                    nrows += nnew;
                }
                __syncthreads();
            }
            if (S.abort_flag) break;
            if (nrows > 0) flush_tile<DB>(S, a, &fmap, nrows, fcount, mma_phase, tx, ty, v);
            if (S.abort_flag) break;
            __syncthreads();   // every thread has read S.item before thread 0 takes the next one
        }
    }
    __syncthreads();
    if (S.abort_flag && tid == 0) {
        // drain: wait (bounded) for whatever was committed last
        mbar_wait(&S.mma_done, mma_phase);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(S.tmem_base, 512);
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
// pixels of one view, 128-byte swizzle, zero fill outside the image.
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

template <int DB>
ludvig_status launch_tc(const TcArgs& args, const CUtensorMap& map, int grid, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        LV_CUDA(cudaFuncSetAttribute(k_composite_tc<DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmemBytes));
        configured = true;
    }
    k_composite_tc<DB><<<grid, kTcThreads, kTcSmemBytes, st>>>(args, map);
    LV_LAUNCH();
    return LUDVIG_OK;
}

ludvig_status dispatch_tc(const TcArgs& args, const CUtensorMap& map, int grid, cudaStream_t st) {
    switch (args.d / 64) {
        case 1: return launch_tc<1>(args, map, grid, st);
        case 2: return launch_tc<2>(args, map, grid, st);
        case 3: return launch_tc<3>(args, map, grid, st);
        case 4: return launch_tc<4>(args, map, grid, st);
        case 5: return launch_tc<5>(args, map, grid, st);
        case 6: return launch_tc<6>(args, map, grid, st);
        case 7: return launch_tc<7>(args, map, grid, st);
        case 8: return launch_tc<8>(args, map, grid, st);
        default: set_error("tensor-core path needs d = 64..512 in steps of 64"); return LUDVIG_ERR_INTERNAL;
    }
}

}  // namespace

bool tc_supported(int dtype, int d) { return dtype == LUDVIG_BF16 && d % 64 == 0 && d >= 64 && d <= 512; }

// Composite + tensor-core aggregation of one chunk of views (stage 6 of the
// uplift pipeline).  `status` receives LUDVIG_ERR_TIMEOUT if a wait expired.
ludvig_status composite_tc(const float4* rec_a, const float2* rec_b, int64_t n, const uint2* ranges,
                           const uint32_t* list, int nv, int width, int height, const void* feats, int d,
                           float* num, float* den, Arena& ws, int* status, cudaStream_t st) {
    CUtensorMap map;
    LV_TRY(make_feature_map(&map, feats, nv, width, height, d));
    int* counter;
    LV_TRY(ws.get("tc.counter", 1, &counter));
    LV_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    int dev = 0, sms = 148;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
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
    return dispatch_tc(a, map, std::min(sms, a.nitems), st);
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
    LV_TRY(dispatch_tc(args, map, 1, st));
    int h = 0;
    LV_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        set_error("tensor-core kernel reported status %d", h);
        return (ludvig_status)h;
    }
    return LUDVIG_OK;
}
