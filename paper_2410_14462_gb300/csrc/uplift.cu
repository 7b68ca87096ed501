// Uplifting of 2D feature maps onto a Gaussian Splatting scene
// (Sec. 3.2, Eq. 3 / Eq. 5): f_i = sum_{v,p} w_i(v,p) F_v[p] / sum_{v,p} w_i(v,p)
// with w the alpha-blending weights of Sec. 3.1 (Eq. 1).
//
// Pipeline per group of up to kMaxViews views (all stages are batched over the
// group's views):
//   1. project     one thread per (view, Gaussian): EWA footprint, depth key,
//                  tile rectangle, number of tiles reached
//   2. depth sort  stable radix sort of (depth bits, index) per view
//   3. bin         the projected records rewritten in depth order (32 bytes
//                  each), exclusive scan of the tiles reached, then one
//                  (view*tiles + tile, depth rank) pair per reached tile
//   4. tile sort   stable radix sort of the pairs by (view, tile): every
//                  tile's list stays in (depth, index) order
//   5. ranges      [start, end) of every (view, tile) list
//   6. composite + aggregate: on the tensor cores (uplift_tc.cu: weight rows
//                  of every tile, gathering the walked records by rank, then
//                  W^T F by tcgen05) for d < 32 (features zero-padded to 32
//                  channels) and for 32 <= d <= 512 with d % 8 == 0; otherwise
//                  here on CUDA cores, one CTA (256 threads = 16x16 pixels) per
//                  (view, tile) over list records with their 8x4 block masks:
//                  walk the list in batches of 32 Gaussians,
//                  form w = alpha T per pixel, keep the non-zero weights of
//                  the tile in a shared-memory sparse store grouped by
//                  Gaussian, then multiply the store with the tile's feature
//                  rows (staged in shared memory by channel chunks) and add
//                  every Gaussian's partial sum into num / den with vector
//                  reductions.
//   7. normalise   f = num / den (den > 0), beta = den.
//
// The uplift entry points do not wait on the host.  The pair count and the
// weight-chunk count of a group are checked on the device against the
// workspace's capacities (a group that does not fit adds nothing and is
// redone by ludvig_sync once the workspace has grown; capacities come from
// earlier calls, or from a first group that runs checked).  Stages 1-5 and the
// weights of a group run on the scene's front stream, its aggregation on the
// aggregation stream, with two buffer sets for the weight rows, so the front
// end of group g + 1 overlaps the aggregation of group g.
//
// Rendering (Eq. 4, F_hat = W f) runs stages 1-5 unchanged and replaces
// stage 6 by the transposed product: every pixel's sum of w_i(p) f_i over its
// contributors, written to the view's feature map.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "spec.cuh"
#include "uplift_int.cuh"

namespace ludvig {

constexpr int kMaxViews = kMaxGroupViews;

bool option_f32_tensor_cores();
bool option_count_normalise();
int64_t option_group_bytes();

// Per-view cameras and scenes of a group (kernel parameters, read in place).
struct CamBatch {
    Cam cam[kMaxViews];
};
struct SceneBatch {
    const float4* geo[kMaxViews];
    const float4* cov_a[kMaxViews];
    const float2* cov_b[kMaxViews];
    int64_t n[kMaxViews];
};
// Per-view coordinates in a feature array (kernel parameter).
struct FViews {
    int f[kMaxViews];
};

// Whether a request's aggregation runs on the tensor cores (else CUDA cores).
bool use_tensor_cores(int dtype, int d) {
    if (!tc_supported(dtype, d)) return false;
    return dtype == LUDVIG_BF16 || option_f32_tensor_cores();
}

namespace {

// ------------------------------------------------------------ scene setup
// scales: linear standard deviations, or (log_scales) their logarithms,
// exponentiated here with CUDA's expf.
__global__ void k_scene_init(const float* __restrict__ means, const float* __restrict__ scales,
                             const float* __restrict__ quats, const float* __restrict__ opac,
                             int64_t n, int log_scales, float4* __restrict__ geo, float4* __restrict__ cov_a,
                             float2* __restrict__ cov_b, float* __restrict__ means_copy) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    if (log_scales) {
        s[0] = expf(s[0]);
        s[1] = expf(s[1]);
        s[2] = expf(s[2]);
    }
    const float q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
    float S[6];
    covariance3d(s, q, S);
    geo[i] = make_float4(m[0], m[1], m[2], opac[i]);
    cov_a[i] = make_float4(S[0], S[1], S[2], S[3]);
    cov_b[i] = make_float2(S[4], S[5]);
    means_copy[3 * i] = m[0];
    means_copy[3 * i + 1] = m[1];
    means_copy[3 * i + 2] = m[2];
}

// ------------------------------------------------------------ 1. project

// One projected Gaussian of one view, as k_project writes it: mean, conic,
// opacity and the tile rectangle (x0 | y0 << 16, x1 | y1 << 16) in 32 bytes.
struct __align__(16) ProjRec {
    float4 a;      // mx, my, conic a, conic b
    float2 b;      // conic c, opacity
    uint2 rect;
};
static_assert(sizeof(ProjRec) == 32, "ProjRec is 32 bytes");

// View v projects the sb.n[v] Gaussians of its own scene; the records of the
// group have a stride of n (the largest scene) per view.
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ SceneBatch sb, int64_t n, int64_t npad,
                          int nv, const __grid_constant__ CamBatch cb, int width, int height,
                          ProjRec* __restrict__ prec, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                          uint32_t* __restrict__ ntile, float* __restrict__ dbg_rec,
                          int32_t* __restrict__ dbg_rect, int prune) {
    // every block is full and lies in one view: npad is a multiple of the
    // block size.  The view's camera and scene go to shared memory once.
    __shared__ Cam cam;
    __shared__ const float4* s_geo;
    __shared__ const float4* s_cov_a;
    __shared__ const float2* s_cov_b;
    __shared__ int64_t s_n;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = (int)((int64_t)blockIdx.x * blockDim.x / npad);
    if (threadIdx.x < 16) reinterpret_cast<float*>(&cam)[threadIdx.x] = reinterpret_cast<const float*>(&cb.cam[v])[threadIdx.x];
    if (threadIdx.x == 0) {
        s_geo = sb.geo[v];
        s_cov_a = sb.cov_a[v];
        s_cov_b = sb.cov_b[v];
        s_n = sb.n[v];
    }
    __syncthreads();
    const int64_t i = idx - (int64_t)v * npad;
    const bool real = i < s_n;
    Projected P{};
    float op = 0.f;
    if (real) {
        const float4 g = s_geo[i];
        const float4 ca = s_cov_a[i];
        const float2 cbv = s_cov_b[i];
        const float m[3] = {g.x, g.y, g.z};
        const float S6[6] = {ca.x, ca.y, ca.z, ca.w, cbv.x, cbv.y};
        P = project_gaussian(m, S6, cam, width, height);
        op = g.w;
        const int64_t o = (int64_t)v * n + i;
        ProjRec pr;
        pr.a = make_float4(P.mx, P.my, P.ca, P.cb);
        pr.b = make_float2(P.cc, g.w);
        pr.rect = P.visible ? make_uint2((uint32_t)P.x0 | ((uint32_t)P.y0 << 16),
                                         (uint32_t)P.x1 | ((uint32_t)P.y1 << 16))
                            : make_uint2(0u, 0u);
        prec[o] = pr;
    }
    const bool vis = real && P.visible;
    const uint32_t area = vis ? (uint32_t)((P.x1 - P.x0) * (P.y1 - P.y0)) : 0u;
    uint32_t count = area;
    if (prune && vis) {
        // only tiles that the alpha >= 1/255 ellipse can reach, row by row
        const EllipseX E = ellipse_prep(reach_prep(P.ca, P.cb, P.cc, op), P.ca, P.cb, P.cc);
        count = 0;
        for (int ty = P.y0; ty < P.y1; ++ty) {
            int c0, c1;
            tile_row_range(E, P.mx, P.my, ty, P.x0, P.x1, c0, c1);
            count += (uint32_t)(c1 - c0);
        }
    }
    keys[idx] = count ? __float_as_uint(P.z) : 0xffffffffu;
    vals[idx] = (uint32_t)i;
    ntile[idx] = count;
    if (dbg_rec && v == 0 && real) {
        float* r = dbg_rec + 8 * i;
        r[0] = P.visible ? P.mx : 0.f;
        r[1] = P.visible ? P.my : 0.f;
        r[2] = P.visible ? P.z : 0.f;
        r[3] = P.visible ? P.ca : 0.f;
        r[4] = P.visible ? P.cb : 0.f;
        r[5] = P.visible ? P.cc : 0.f;
        r[6] = P.visible ? op : 0.f;
        r[7] = P.visible ? P.radius : 0.f;
        int32_t* q = dbg_rect + 4 * i;
        q[0] = P.visible ? P.x0 : 0;
        q[1] = P.visible ? P.y0 : 0;
        q[2] = P.visible ? P.x1 : 0;
        q[3] = P.visible ? P.y1 : 0;
    }
}

// ------------------------------------------------------------ 3. bin
// Largest pair count a group may have: positions are 32-bit and the sort pads
// to whole blocks.
constexpr int64_t kMaxPairs = 0x7fffffff - 2 * (int64_t)kRadixTile;

// Whether `np` pairs fit buffers of `cap` entries (cap a multiple of the sort block).
__device__ __forceinline__ bool pairs_fit(uint64_t np, uint64_t cap) {
    return np <= (uint64_t)kMaxPairs && (np + kRadixTile - 1) / kRadixTile * kRadixTile <= cap;
}

// The projected records in depth order, one per (view, rank): mean, conic,
// opacity and index in a 32-byte record (its mask word unused) plus the tile
// rectangle, and the number of tiles each reaches (0 for the culled ones,
// whose records are never read).  A record is gathered in one 32-byte sector.
__global__ void k_sorted_records(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                                 const uint32_t* __restrict__ ntile, const ProjRec* __restrict__ prec, int64_t n,
                                 int64_t npad, int64_t total, uint32_t* __restrict__ cnt, PairRec* __restrict__ srec,
                                 uint2* __restrict__ srect) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    if (skeys[idx] == 0xffffffffu) {
        cnt[idx] = 0u;
        return;
    }
    const int64_t v = idx / npad;
    const uint32_t i = svals[idx];
    const ProjRec pr = prec[v * n + i];
    const float4 ra = pr.a;
    const float2 rb = pr.b;
    cnt[idx] = ntile[v * npad + i];
    PairRec r;
    r.mx = ra.x;
    r.my = ra.y;
    r.ca = ra.z;
    r.cb = ra.w;
    r.cc = rb.x;
    r.op = rb.y;
    r.gid = i;
    r.mask = 0u;
    srec[idx] = r;
    srect[idx] = pr.rect;
}

// One (view * tiles + tile, rank) pair per tile a Gaussian reaches, written in
// depth order at the Gaussian's scanned offset.  Nothing is written when the
// group's pairs do not fit the buffers (the overflow word is set instead).
// Keys are 32-bit, or 16-bit when every (view, tile) key and the sentinel fit.
//
// The pairs of a warp's 32 consecutive Gaussians occupy one contiguous range
// (the offsets are an exclusive scan of the counts).  The warp fills that
// range window by window: each lane puts its pairs that fall in the window
// into shared memory (re-walking its tile rows from the first for a later
// window), then the warp copies the window out with consecutive lanes on
// consecutive entries, so the stores coalesce instead of scattering one
// 2- or 4-byte store per pair over the Gaussians' separate runs.
constexpr int kEmitThreads = 128;
constexpr int kEmitWin = 1024;   // pairs per warp and window

template <class KeyT>
__global__ void __launch_bounds__(kEmitThreads)
k_emit_pairs(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ off, const PairRec* __restrict__ srec,
             const uint2* __restrict__ srect, int64_t npad, int64_t total, int TX, int ntiles, int prune,
             const uint64_t* __restrict__ np_dev, uint64_t cap, int* ovf, uint32_t sentinel,
             KeyT* __restrict__ pkey, uint32_t* __restrict__ pval) {
    __shared__ KeyT s_key[kEmitThreads / 32][kEmitWin];
    __shared__ uint32_t s_val[kEmitThreads / 32][kEmitWin];
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (idx - lane >= total) return;   // (whole warp)
    if (!pairs_fit(*np_dev, cap)) {
        if (idx == 0 && ovf) atomicOr(ovf, 1);
        return;
    }
    const bool in = idx < total;
    const uint32_t c = in ? cnt[idx] : 0u;
    const uint32_t o = in ? off[idx] : 0u;
    const uint32_t wbase = __shfl_sync(0xffffffffu, o, 0);           // lane 0 is in range
    const uint32_t wend = __reduce_max_sync(0xffffffffu, in ? o + c : 0u);
    if (wend <= wbase) return;
    int64_t v = 0;
    uint32_t rank = 0;
    PairRec r{};
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    EllipseX E{};
    E.state = 2;   // unpruned: every tile of the rectangle
    if (c > 0) {
        v = idx / npad;
        rank = (uint32_t)(idx - v * npad);
        r = srec[idx];
        const uint2 rt = srect[idx];
        x0 = rt.x & 0xffff;
        y0 = rt.x >> 16;
        x1 = rt.y & 0xffff;
        y1 = rt.y >> 16;
        if (prune) E = ellipse_prep(reach_prep(r.ca, r.cb, r.cc, r.op), r.ca, r.cb, r.cc);
    }
    const uint32_t base = (uint32_t)(v * ntiles);
    const uint32_t end = o + c;   // never write past the counted slots
    KeyT* sk = s_key[warp];
    uint32_t* sv = s_val[warp];
    for (uint32_t win = wbase; win < wend; win += kEmitWin) {
        const uint32_t wlim = min(win + (uint32_t)kEmitWin, wend);
        if (c > 0 && o < wlim && end > win) {
            uint32_t p = o;
            for (int ty = y0; ty < y1 && p < end && p < wlim; ++ty) {
                int c0, c1;
                tile_row_range(E, r.mx, r.my, ty, x0, x1, c0, c1);
                if (p + (uint32_t)(c1 - c0) <= win) {   // the whole row lies before the window
                    p += (uint32_t)(c1 - c0);
                    continue;
                }
                for (int tx = c0; tx < c1 && p < end && p < wlim; ++tx, ++p)
                    if (p >= win) {
                        sk[p - win] = (KeyT)(base + (uint32_t)(ty * TX + tx));
                        sv[p - win] = rank;
                    }
            }
            // unreachable when the count and this walk agree; keeps the keys defined
            for (p = max(p, win); p < end && p < wlim; ++p) {
                sk[p - win] = (KeyT)sentinel;
                sv[p - win] = 0u;
            }
        }
        __syncwarp();
        for (uint32_t j = lane; j < wlim - win; j += 32) {
            pkey[win + j] = sk[j];
            pval[win + j] = sv[j];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ 5. ranges
// Each thread takes 8 consecutive sorted keys (one or two 16-byte loads) and
// marks where a key's run starts and ends; the neighbours across its group
// come from two scalar loads.  The key buffer starts on a 16-byte boundary.
template <class KeyT>
__global__ void k_ranges(const KeyT* __restrict__ pkey, const uint64_t* __restrict__ np_dev, uint64_t cap,
                         uint32_t nkeys, uint2* __restrict__ ranges) {
    constexpr int kV = 8;
    const uint64_t np = *np_dev;
    if (!pairs_fit(np, cap)) return;
    const int64_t P = (int64_t)np;
    const int64_t ngroups = (P + kV - 1) / kV;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = g * kV;
        uint32_t k[kV];
        if (j0 + kV <= P) {
            if constexpr (sizeof(KeyT) == 2) {
                const uint4 q = *reinterpret_cast<const uint4*>(pkey + j0);
                const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    k[2 * i] = w[i] & 0xffffu;
                    k[2 * i + 1] = w[i] >> 16;
                }
            } else {
                const uint4 a = *reinterpret_cast<const uint4*>(pkey + j0);
                const uint4 b = *reinterpret_cast<const uint4*>(pkey + j0 + 4);
                k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
                k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kV; ++i) k[i] = j0 + i < P ? (uint32_t)pkey[j0 + i] : 0xffffffffu;
        }
        const uint32_t prev = j0 > 0 ? (uint32_t)pkey[j0 - 1] : 0xffffffffu;
        const uint32_t next = j0 + kV < P ? (uint32_t)pkey[j0 + kV] : 0xffffffffu;
#pragma unroll
        for (int i = 0; i < kV; ++i) {
            const int64_t j = j0 + i;
            const uint32_t kk = k[i];
            if (j >= P || kk >= nkeys) continue;
            const uint32_t before = i > 0 ? k[i - 1] : prev;
            const uint32_t after = i + 1 < kV ? k[i + 1] : next;
            if (j == 0 || before != kk) ranges[kk].x = (uint32_t)j;
            if (j == P - 1 || after != kk) ranges[kk].y = (uint32_t)(j + 1);
        }
    }
}

// The sorted lists as the CUDA-core compositing kernels stream them: one
// 32-byte record per entry, in list order, with the entry's 8x4 block mask.
// (The tensor-core weights kernel gathers the depth-ordered records itself.)
__global__ void k_pair_records(const uint32_t* __restrict__ pkey, const uint32_t* __restrict__ pval,
                               const uint64_t* __restrict__ np_dev, uint64_t cap, int ntiles, int TX, int64_t npad,
                               const PairRec* __restrict__ srec, PairRec* __restrict__ out) {
    const uint64_t np = *np_dev;
    if (!pairs_fit(np, cap)) return;
    const int64_t P = (int64_t)np;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = pkey[j];
        const uint32_t v = key / (uint32_t)ntiles, tile = key - v * (uint32_t)ntiles;
        const int tx = (int)(tile % (uint32_t)TX), ty = (int)(tile / (uint32_t)TX);
        PairRec r = srec[(int64_t)v * npad + pval[j]];
        r.mask = block_mask_fast(r.mx, r.my, r.ca, r.cb, r.cc, r.op, tx, ty);
        out[j] = r;
    }
}

// ------------------------------------------------------------ 6. composite + aggregate
constexpr int kBatch = 32;        // Gaussians composited per step
constexpr int kStoreCap = 12288;  // non-zero weights kept per flush
constexpr int kRowCap = 1024;     // Gaussians kept per flush
constexpr int kChunk = 32;        // channels per aggregation chunk (vector path)

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

struct CompositeArgs {
    const PairRec* pairs;   // list records in list order
    const uint2* ranges;
    int ntiles, TX, width, height;
    const void* feats;      // chunk's first view
    int d;
    float* num;
    float* den;
    float* dbg_t;           // [H*W] view 0 only, or null
    int32_t* dbg_cnt;
    int count_den;          // den += the number of non-zero weights instead of their sum
};

struct CompositeSmem {
    float4 ra[kBatch];
    float2 rb[kBatch];
    uint32_t gid[kBatch];
    uint32_t bmask[kBatch];
    uint32_t wcnt[8][kBatch];
    uint32_t rtot[kBatch];
    uint32_t rbase[kBatch];
    uint32_t row_gid[kRowCap];
    uint32_t row_start[kRowCap];
    uint32_t row_cnt[kRowCap];
    float store_w[kStoreCap];
    uint8_t store_p[kStoreCap];
    int nstore, nrows;
    alignas(16) float F[256 * kChunk];
};

template <class TIn, bool kVec>
__device__ void flush_store(CompositeSmem& sm, const CompositeArgs& a, const TIn* __restrict__ fv,
                            int tx, int ty) {
    __syncthreads();
    const int R = sm.nrows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (R > 0) {
        // beta_i partial: sum of the Gaussian's stored weights
        for (int r = warp; r < R; r += 8) {
            const uint32_t st = sm.row_start[r], c = sm.row_cnt[r];
            float s = 0.f;
            for (uint32_t k = lane; k < c; k += 32) s += a.count_den ? 1.f : sm.store_w[st + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) atomicAdd(a.den + sm.row_gid[r], s);
        }
        const int d = a.d;
        constexpr int cw = kVec ? kChunk : 8;   // channels per chunk
        for (int c0 = 0; c0 < d; c0 += cw) {
            const int dcw = min(cw, d - c0);
            // stage F[tile pixels][c0 : c0+dcw) (zeros outside the image)
            for (int idx = tid; idx < 256 * cw; idx += 256) {
                const int p = idx / cw, c = idx % cw;
                const int px = tx * kTile + (p & 15), py = ty * kTile + (p >> 4);
                float val = 0.f;
                if (c < dcw && px < a.width && py < a.height)
                    val = to_f32(fv[((int64_t)py * a.width + px) * d + c0 + c]);
                sm.F[p * kChunk + c] = val;
            }
            __syncthreads();
            if (kVec) {
                const int q = lane & 7;
                for (int r = warp * 4 + (lane >> 3); r < R; r += 32) {
                    const uint32_t st = sm.row_start[r], c = sm.row_cnt[r];
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (uint32_t k = 0; k < c; ++k) {
                        const int p = sm.store_p[st + k];
                        const float w = sm.store_w[st + k];
                        const float4 f = *reinterpret_cast<const float4*>(&sm.F[p * kChunk + 4 * q]);
                        acc.x = fmaf(w, f.x, acc.x);
                        acc.y = fmaf(w, f.y, acc.y);
                        acc.z = fmaf(w, f.z, acc.z);
                        acc.w = fmaf(w, f.w, acc.w);
                    }
                    if (4 * q < dcw) red_add_v4(a.num + (int64_t)sm.row_gid[r] * d + c0 + 4 * q, acc);
                }
            } else {
                const int q = lane & 7;
                for (int r = warp * 4 + (lane >> 3); r < R; r += 32) {
                    const uint32_t st = sm.row_start[r], c = sm.row_cnt[r];
                    float acc = 0.f;
                    for (uint32_t k = 0; k < c; ++k)
                        acc = fmaf(sm.store_w[st + k], sm.F[sm.store_p[st + k] * kChunk + q], acc);
                    if (q < dcw) atomicAdd(a.num + (int64_t)sm.row_gid[r] * d + c0 + q, acc);
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        sm.nstore = 0;
        sm.nrows = 0;
    }
    __syncthreads();
}

template <class TIn, bool kVec>
__global__ void __launch_bounds__(256, 2) k_composite(CompositeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CompositeSmem& sm = *reinterpret_cast<CompositeSmem*>(smem_raw);
    const int item = blockIdx.x;
    const int v = item / a.ntiles, tile = item - v * a.ntiles;
    const int tx = tile % a.TX, ty = tile / a.TX;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    // warp w covers the 8x4 pixel block ((w & 1) * 8, (w >> 1) * 4) of the tile
    const int bx = (warp & 1) * 8, by = (warp >> 1) * 4;
    const int lx = bx + (lane & 7), ly = by + (lane >> 3);
    const int pix = ly * kTile + lx;   // tile-local pixel index
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < a.width && py < a.height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 range = a.ranges[item];
    const TIn* fv = reinterpret_cast<const TIn*>(a.feats) + (int64_t)v * a.height * a.width * a.d;
    if (tid == 0) {
        sm.nstore = 0;
        sm.nrows = 0;
    }
    // records of the next batch, loaded one batch ahead
    PairRec nxt{};
    if (tid < kBatch && range.x + tid < range.y) nxt = a.pairs[range.x + tid];
    float T = 1.0f;
    bool done = !inside;
    int ncontrib = 0;
    __syncthreads();
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        if (__syncthreads_count(!done) == 0) break;
        const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
        if (sm.nstore + kBatch * 256 > kStoreCap || sm.nrows + kBatch > kRowCap)
            flush_store<TIn, kVec>(sm, a, fv, tx, ty);
        if (tid < cnt) {
            sm.gid[tid] = nxt.gid;
            sm.bmask[tid] = nxt.mask;
            sm.ra[tid] = make_float4(nxt.mx, nxt.my, nxt.ca, nxt.cb);
            sm.rb[tid] = make_float2(nxt.cc, nxt.op);
        }
        if (tid < kBatch && b0 + kBatch + tid < range.y) nxt = a.pairs[b0 + kBatch + tid];
        __syncthreads();
        // Gaussians of the batch that can reach this warp's pixel block
        uint32_t rel = __ballot_sync(0xffffffffu, lane < cnt && ((sm.bmask[lane] >> warp) & 1u));
        if (!__any_sync(0xffffffffu, !done)) rel = 0u;
        // alphas of the batch first (independent chains the scheduler can
        // overlap), then the sequential transmittance recursion
        float w[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            w[j] = 0.f;
            if ((rel >> j) & 1u) {
                const float4 ra = sm.ra[j];
                const float2 rb = sm.rb[j];
                w[j] = alpha_at(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, pxf, pyf);
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const float al = w[j];
            w[j] = 0.f;
            if (al > 0.f && !done) {
                const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
                if (Tn < kTransMin) {
                    done = true;
                } else {
                    w[j] = __fmul_rn(al, T);
                    T = Tn;
                    ++ncontrib;
                }
            }
        }
        // per-warp counts of non-zero weights of every Gaussian of the batch
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const uint32_t m = __ballot_sync(0xffffffffu, w[j] != 0.f);
            if (lane == 0) sm.wcnt[warp][j] = __popc(m);
        }
        __syncthreads();
        if (tid < kBatch) {
            uint32_t t = 0;
#pragma unroll
            for (int wi = 0; wi < 8; ++wi) {
                const uint32_t c = sm.wcnt[wi][tid];
                sm.wcnt[wi][tid] = t;
                t += c;
            }
            sm.rtot[tid] = t;
        }
        __syncthreads();
        if (warp == 0) {
            const int ns = sm.nstore, nr = sm.nrows;
            const uint32_t t = lane < cnt ? sm.rtot[lane] : 0u;
            uint32_t incl = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const uint32_t start = (uint32_t)ns + incl - t;
            sm.rbase[lane] = start;
            const uint32_t nzm = __ballot_sync(0xffffffffu, t > 0);
            if (t > 0) {
                const int slot = nr + __popc(nzm & lt_mask);
                sm.row_gid[slot] = sm.gid[lane];
                sm.row_start[slot] = start;
                sm.row_cnt[slot] = t;
            }
            __syncwarp();
            if (lane == 31) {
                sm.nstore = ns + (int)incl;
                sm.nrows = nr + __popc(nzm);
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const uint32_t m = __ballot_sync(0xffffffffu, w[j] != 0.f);
            if (w[j] != 0.f) {
                const uint32_t pos = sm.rbase[j] + sm.wcnt[warp][j] + __popc(m & lt_mask);
                sm.store_w[pos] = w[j];
                sm.store_p[pos] = (uint8_t)pix;
            }
        }
        __syncthreads();
    }
    flush_store<TIn, kVec>(sm, a, fv, tx, ty);
    if (a.dbg_t && v == 0 && inside) {
        a.dbg_t[(int64_t)py * a.width + px] = T;
        a.dbg_cnt[(int64_t)py * a.width + px] = ncontrib;
    }
}

// ------------------------------------------------------------ 6'. render (Eq. 4)
struct RenderArgs {
    const PairRec* pairs;   // list records in list order
    const uint2* ranges;
    int ntiles, TX, width, height;
    const float* f;         // [n, d]
    int d;
    float* out;             // chunk's first view, [H, W, d]
};

// CUDA-core rendering: one CTA per (view, tile) and DC channels (blockIdx.y),
// one thread per pixel.  Walks the tile's list in batches of 32 Gaussians with
// the compositing rules of k_composite and adds w f_i (the batch's DC-channel
// feature slices staged in shared memory) into per-pixel registers in list
// order; every pixel of the image is written (zero without contributors).
template <int DC>
__global__ void __launch_bounds__(256) k_render_cc(RenderArgs a) {
    __shared__ float4 ra[kBatch];
    __shared__ float2 rb[kBatch];
    __shared__ uint32_t bmask[kBatch];
    __shared__ uint32_t gid[kBatch];
    __shared__ float fs[kBatch][DC];
    const int item = blockIdx.x, c0 = blockIdx.y * DC;
    const int v = item / a.ntiles, tile = item - v * a.ntiles;
    const int tx = tile % a.TX, ty = tile / a.TX;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp w covers the 8x4 pixel block ((w & 1) * 8, (w >> 1) * 4) of the tile
    const int lx = (warp & 1) * 8 + (lane & 7), ly = (warp >> 1) * 4 + (lane >> 3);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < a.width && py < a.height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 range = a.ranges[item];
    const int d = a.d;
    float acc[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) acc[c] = 0.f;
    float T = 1.0f;
    bool done = !inside;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        // every thread is done with the previous batch's shared memory
        if (__syncthreads_count(!done) == 0) break;
        const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
        if (tid < cnt) {
            const PairRec r = a.pairs[b0 + tid];
            ra[tid] = make_float4(r.mx, r.my, r.ca, r.cb);
            rb[tid] = make_float2(r.cc, r.op);
            bmask[tid] = r.mask;
            gid[tid] = r.gid;
        }
        __syncthreads();
        for (int e = tid; e < cnt * DC; e += 256) {
            const int j = e / DC, c = e - j * DC;
            fs[j][c] = c0 + c < d ? a.f[(int64_t)gid[j] * d + c0 + c] : 0.f;
        }
        __syncthreads();
        uint32_t rel = __ballot_sync(0xffffffffu, lane < cnt && ((bmask[lane] >> warp) & 1u));
        if (!__any_sync(0xffffffffu, !done)) rel = 0u;
        float w[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            w[j] = 0.f;
            if ((rel >> j) & 1u) {
                const float4 g = ra[j];
                const float2 h = rb[j];
                w[j] = alpha_at(g.x, g.y, g.z, g.w, h.x, h.y, pxf, pyf);
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            const float al = w[j];
            w[j] = 0.f;
            if (al > 0.f && !done) {
                const float Tn = __fmul_rn(T, __fsub_rn(1.0f, al));
                if (Tn < kTransMin) {
                    done = true;
                } else {
                    w[j] = __fmul_rn(al, T);
                    T = Tn;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
            if (w[j] != 0.f) {
#pragma unroll
                for (int c = 0; c < DC; ++c) acc[c] = fmaf(w[j], fs[j][c], acc[c]);
            }
        }
    }
    if (inside) {
        float* o = a.out + (((int64_t)v * a.height + py) * a.width + px) * d + c0;
#pragma unroll
        for (int c = 0; c < DC; ++c)
            if (c0 + c < d) o[c] = acc[c];
    }
}

// ------------------------------------------------------------ 7. normalise
// `skip` (device, may be null): when non-zero, nothing is written (an
// asynchronous uplift whose sums are still incomplete).
__global__ void k_normalise(const float* num, const float* __restrict__ den, float* out, float* beta,
                            int64_t n, int d, const int* __restrict__ skip) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * d) return;
    if (skip && *skip) return;
    const int64_t i = idx / d;
    const float b = den[i];
    out[idx] = b > 0.f ? num[idx] / b : 0.f;
    if (beta && idx % d == 0) beta[i] = b;
}

// Same, one warp per Gaussian (d >= 32), float4 accesses when vec4 (d % 4 == 0
// and 16-byte aligned rows).
__global__ void k_normalise_rows(const float* num, const float* __restrict__ den, float* out, float* beta,
                                 int64_t n, int d, int vec4, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        const float b = den[i];
        const float* src = num + i * d;
        float* dst = out + i * d;
        if (vec4) {
            for (int c = 4 * lane; c < d; c += 128) {
                const float4 x = *reinterpret_cast<const float4*>(src + c);
                *reinterpret_cast<float4*>(dst + c) =
                    b > 0.f ? make_float4(x.x / b, x.y / b, x.z / b, x.w / b) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int c = lane; c < d; c += 32) dst[c] = b > 0.f ? src[c] / b : 0.f;
        }
        if (beta && lane == 0) beta[i] = b;
    }
}

unsigned grid_for(int64_t work, int threads) { return (unsigned)ceil_div(work, threads); }

// Grid of the grid-stride kernels over a group's pairs (their count is on the device).
constexpr unsigned kPairGrid = 152 * 16;

struct ChunkDebug {
    float* rec = nullptr;
    int32_t* rect = nullptr;
    bool stop_after_project = false;
    int64_t* ranges64 = nullptr;   // [ntiles*2]
    int32_t* list = nullptr;
    int64_t list_cap = 0;
    int64_t* list_total = nullptr;  // host
    bool stop_after_sort = false;
    bool unpruned = false;          // lists by the tile-rectangle rule alone
    float* t_final = nullptr;
    int32_t* n_contrib = nullptr;
};

__global__ void k_export_ranges(const uint2* __restrict__ r, int64_t nt, int64_t* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    out[2 * t] = r[t].x;
    out[2 * t + 1] = r[t].y;
}

__global__ void k_debug_fill(float* __restrict__ t, int32_t* __restrict__ c, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        t[i] = 1.0f;
        c[i] = 0;
    }
}

// The list entries as Gaussian indices (the lists hold depth ranks).
__global__ void k_export_list(const uint32_t* __restrict__ pkey, const uint32_t* __restrict__ pval, int64_t P,
                              int ntiles, int64_t npad, const PairRec* __restrict__ srec, int32_t* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const int64_t v = pkey[j] / (uint32_t)ntiles;
    out[j] = (int32_t)srec[v * npad + pval[j]].gid;
}

size_t composite_smem() { return sizeof(CompositeSmem); }

template <class TIn, bool kVec>
ludvig_status launch_composite(const CompositeArgs& args, int64_t nitems, cudaStream_t st) {
    // set once per process; a function-local static is initialised by one thread
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_composite<TIn, kVec>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)composite_smem());
    LV_CUDA(configured);
    k_composite<TIn, kVec><<<(unsigned)nitems, 256, composite_smem(), st>>>(args);
    LV_LAUNCH();
    return LUDVIG_OK;
}

template <int DC>
ludvig_status launch_render_cc(const RenderArgs& args, int64_t nitems, cudaStream_t st) {
    const dim3 grid((unsigned)nitems, (unsigned)ceil_div(args.d, DC));
    StageScope scope(LUDVIG_STAGE_RENDER_PRODUCT, st);
    k_render_cc<DC><<<grid, 256, 0, st>>>(args);
    LV_LAUNCH();
    return LUDVIG_OK;
}

// Few channels (d < 32): the tensor-core path with the features zero-padded
// to kPadD channels.  The CUDA-core composite spends its time walking each
// tile's list once per pixel and reducing per Gaussian; the weight-row walk
// of the tensor-core path does the same walk faster, and the padded
// contraction costs little next to it.  The padded features of up to
// kMaxViews views live in the workspace, the padded numerator [n, kPadD]
// too; its first d columns are added to num at the end (the zero channels
// contribute nothing, den is the same sum of weights).
constexpr int kPadD = 32;

// One thread per 16-byte group of a padded pixel (8 bfloat16 or 4 float
// channels): one vector store each, loads only for the channels below d.
// Padded view v (group order) comes from view coordinate fv.f[v] of src.
template <class T>
__global__ void k_pad_features(const T* __restrict__ src, const __grid_constant__ FViews fv, int64_t view_px,
                               int64_t npx, int d, T* __restrict__ dst) {
    constexpr int kPer = 16 / (int)sizeof(T);
    constexpr int kGroups = kPadD / kPer;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npx * kGroups) return;
    const int64_t p = e / kGroups;
    const int64_t v = p / view_px;
    const T* sp = src + ((int64_t)fv.f[v] * view_px + (p - v * view_px)) * d;
    const int c0 = (int)(e - p * kGroups) * kPer;
    T vals[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) vals[k] = c0 + k < d ? sp[c0 + k] : T(0.f);
    uint4 packed;
    memcpy(&packed, vals, sizeof(packed));
    reinterpret_cast<uint4*>(dst)[e] = packed;
}

__global__ void k_add_columns(const float* __restrict__ wide, int64_t n, int d, float* __restrict__ num) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    const int64_t i = e / d;
    num[e] += wide[i * kPadD + (e - i * d)];
}

bool use_padded(int dtype, int d) { return d < kPadD && use_tensor_cores(dtype, kPadD); }

// FP8-E4M3 features (codes q, per-view scales s): x = decode(q) s_v rounded
// to bfloat16 for the tensor-core path (the E4M3 value is exact in half
// precision; the bfloat16 rounding adds at most 2^-9 relative to an FP8
// quantisation error of up to 2^-4).  Thread t converts elements 4t .. 4t+3
// of the group (one 4-byte load, one 8-byte store, when the codes and the
// output are aligned for them; else element by element); the scalar tail
// covers a total that is not a multiple of 4.
__device__ __forceinline__ __nv_bfloat16 dequant_e4m3(uint32_t code, float s) {
    const __half h(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3));
    return __float2bfloat16_rn(__half2float(h) * s);
}

__global__ void k_dequant_e4m3(const uint8_t* __restrict__ q, const float* __restrict__ s, int64_t view_elems,
                               int64_t total, __nv_bfloat16* __restrict__ out) {
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e0 >= total) return;
    const bool aligned = ((reinterpret_cast<uintptr_t>(q) & 3) | (reinterpret_cast<uintptr_t>(out) & 7)) == 0;
    if (aligned && e0 + 4 <= total) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(q + e0);
        __nv_bfloat16 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = dequant_e4m3((w >> (8 * k)) & 0xffu, s[(e0 + k) / view_elems]);
        uint2 v;
        memcpy(&v, o, sizeof(v));
        *reinterpret_cast<uint2*>(out + e0) = v;
    } else {
        for (int64_t e = e0; e < total && e < e0 + 4; ++e) out[e] = dequant_e4m3(q[e], s[e / view_elems]);
    }
}

// ---------------------------------------------------------------- front end

// The lists of a group of views after stages 1-5.
struct FrontEnd {
    GroupLists L{};
    const uint32_t* spk = nullptr;   // sorted pair keys (view * tiles + tile)
    const uint64_t* np = nullptr;    // device: the group's pair count
    int64_t cap = 0;                 // capacity of the pair buffers
    int64_t P = -1;                  // pair count, when read back (checked runs)
    bool too_many = false;           // checked runs: more pairs than one group may hold
};

// The views v0 .. v0 + nv - 1 of one scene as a group: feature coordinates
// v0 .. v0 + nv - 1, sums into num / den.
GroupViews scene_group(const ludvig_scene* s, const ludvig_camera* cams, int v0, int nv, float* num, float* den) {
    GroupViews g;
    g.nmax = s->n;
    g.v.resize((size_t)nv);
    for (int k = 0; k < nv; ++k) g.v[(size_t)k] = ViewRef{s, cams[v0 + k], v0 + k, num, den};
    return g;
}

// Whether the group's views read consecutive feature coordinates and add into
// the same num / den (a group of one scene's call).
bool single_call(const GroupViews& g) {
    for (size_t k = 1; k < g.v.size(); ++k)
        if (g.v[k].fview != g.v[0].fview + (int)k || g.v[k].num != g.v[0].num || g.v[k].den != g.v[0].den ||
            g.v[k].scene != g.v[0].scene)
            return false;
    return true;
}

// The per-view Gaussian scratch of a group of nv views of up to n Gaussians
// (about 120 bytes per view and Gaussian).
struct FrontBufs {
    ProjRec* prec;
    uint2* srect;
    uint32_t *keys, *vals, *keys2, *vals2, *ntile, *cnt, *off;
    PairRec* srec;
    uint64_t* total;
};

ludvig_status front_buffers(Arena& ws, int nv, int64_t n, FrontBufs* b) {
    const int64_t nG = (int64_t)nv * round_up(std::max<int64_t>(n, 1), kRadixTile);
    LV_TRY(ws.get("up.prec", (size_t)nv * n, &b->prec));
    LV_TRY(ws.get("up.keys", (size_t)nG, &b->keys));
    LV_TRY(ws.get("up.vals", (size_t)nG, &b->vals));
    LV_TRY(ws.get("up.keys2", (size_t)nG, &b->keys2));
    LV_TRY(ws.get("up.vals2", (size_t)nG, &b->vals2));
    LV_TRY(ws.get("up.ntile", (size_t)nG, &b->ntile));
    LV_TRY(ws.get("up.cnt", (size_t)nG, &b->cnt));
    LV_TRY(ws.get("up.off", (size_t)nG, &b->off));
    LV_TRY(ws.get("up.srec", (size_t)nG, &b->srec));
    LV_TRY(ws.get("up.srect", (size_t)nG, &b->srect));
    LV_TRY(ws.get("up.total", 1, &b->total));
    return LUDVIG_OK;
}

// Stages 1-5 of a group on `st`, in the workspace of `ctx` (the scene of a
// one-scene call, or a batch's context).  checked: the pair count is read
// back (synchronises `st`) and the pair buffers grow to fit it.  Otherwise
// nothing waits: the buffers keep ctx's pair capacity, and a group that
// needs more sets *ovf, writes no pairs (all lists empty) and is redone later.
ludvig_status front_end(ludvig_scene* ctx, const GroupViews& g, int width, int height, bool checked,
                        int* ovf, const ChunkDebug* dbg, cudaStream_t st, FrontEnd* fe, bool keys16_ok = false) {
    ludvig_scene* s = ctx;
    Arena& ws = s->ws;
    const int nv = (int)g.v.size();
    const int64_t n = g.nmax;
    const int64_t npad = round_up(std::max<int64_t>(n, 1), kRadixTile);
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int ntiles = TX * TY;
    const int64_t nG = (int64_t)nv * npad;
    const int prune = (dbg && dbg->unpruned) ? 0 : 1;

    FrontBufs b;
    LV_TRY(front_buffers(ws, nv, n, &b));
    ProjRec* prec = b.prec;
    uint2* srect = b.srect;
    uint32_t *keys = b.keys, *vals = b.vals, *keys2 = b.keys2, *vals2 = b.vals2, *ntile = b.ntile, *cnt = b.cnt,
             *off = b.off;
    PairRec* srec = b.srec;
    uint64_t* total_d = b.total;

    if (nv < 1 || nv > kMaxViews) {
        set_error("a group holds 1 to %d views, not %d", kMaxViews, nv);
        return LUDVIG_ERR_INTERNAL;
    }
    CamBatch cb;
    SceneBatch sb;
    for (int v = 0; v < nv; ++v) {
        const ludvig_camera& c = g.v[(size_t)v].cam;
        for (int k = 0; k < 9; ++k) cb.cam[v].R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) cb.cam[v].t[k] = c.t[k];
        cb.cam[v].fx = c.fx;
        cb.cam[v].fy = c.fy;
        cb.cam[v].cx = c.cx;
        cb.cam[v].cy = c.cy;
        const ludvig_scene* vs = g.v[(size_t)v].scene;
        sb.geo[v] = vs->geo;
        sb.cov_a[v] = vs->cov_a;
        sb.cov_b[v] = vs->cov_b;
        sb.n[v] = vs->n;
    }
    int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_PROJECT, st) : -1;
    k_project<<<grid_for(nG, 256), 256, 0, st>>>(sb, n, npad, nv, cb, width, height, prec, keys,
                                                  vals, ntile, dbg ? dbg->rec : nullptr, dbg ? dbg->rect : nullptr,
                                                  prune);
    LV_LAUNCH();
    trace_end(tslot, st);
    if (dbg && dbg->stop_after_project) return LUDVIG_OK;

    uint32_t *sk = keys, *sv = vals;
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_DEPTH_SORT, st) : -1;
    // (a packed batch's context sorts in one kernel per pass: fewer launches for
    // many groups; a single call takes the faster reduce-then-scan passes)
    if (s->onesweep)
        LV_TRY(radix_sort_onesweep(&sk, &sv, keys2, vals2, nv, npad, nullptr, 32, s->dstat, ws, st));
    else
        LV_TRY(radix_sort_pairs(&sk, &sv, keys2, vals2, nv, npad, 32, ws, st));
    trace_end(tslot, st);
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_BIN, st) : -1;
    k_sorted_records<<<grid_for(nG, 256), 256, 0, st>>>(sk, sv, ntile, prec, n, npad, nG, cnt, srec,
                                                        srect);
    LV_LAUNCH();
    LV_TRY(scan_exclusive_u32(cnt, off, nG, total_d, ws, st));
    int64_t P = -1;
    if (checked) {
        void* h;
        LV_TRY(ws.pinned("up.total_h", 16, &h));
        LV_CUDA(cudaMemcpyAsync(h, total_d, 8, cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        P = (int64_t)*static_cast<uint64_t*>(h);
        if (P > kMaxPairs) {
            trace_end(tslot, st);
            fe->too_many = true;
            return LUDVIG_OK;
        }
        const int64_t need = round_up(std::max<int64_t>(P, 1), kRadixTile);
        if (s->pair_cap < need) s->pair_cap = round_up(need + need / 8, kRadixTile);
    }
    const int64_t cap = std::max<int64_t>(s->pair_cap, kRadixTile);
    const uint32_t sentinel = (uint32_t)nv * (uint32_t)ntiles;
    uint32_t *pk, *pv, *pk2, *pv2;
    LV_TRY(ws.get("up.pk", (size_t)cap, &pk));
    LV_TRY(ws.get("up.pv", (size_t)cap, &pv));
    LV_TRY(ws.get("up.pk2", (size_t)cap, &pk2));
    LV_TRY(ws.get("up.pv2", (size_t)cap, &pv2));
    // 16-bit keys when the caller reads only the ranks and lists afterwards
    // (the tensor-core path) and every key and the sentinel fit
    const bool k16 = keys16_ok && !s->onesweep && sentinel < 0xffffu && !dbg;
    if (k16)
        k_emit_pairs<uint16_t><<<grid_for(nG, kEmitThreads), kEmitThreads, 0, st>>>(cnt, off, srec, srect, npad, nG, TX, ntiles, prune,
                                                                  total_d, (uint64_t)cap, ovf, sentinel,
                                                                  reinterpret_cast<uint16_t*>(pk), pv);
    else
        k_emit_pairs<uint32_t><<<grid_for(nG, kEmitThreads), kEmitThreads, 0, st>>>(cnt, off, srec, srect, npad, nG, TX, ntiles, prune,
                                                                  total_d, (uint64_t)cap, ovf, sentinel, pk, pv);
    LV_LAUNCH();
    trace_end(tslot, st);
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_TILE_SORT, st) : -1;
    int nbits = 1;
    while (((uint32_t)1 << nbits) <= sentinel) ++nbits;
    uint32_t *spk = pk, *spv = pv;
    uint16_t* spk16 = reinterpret_cast<uint16_t*>(pk);
    if (k16)
        LV_TRY(radix_sort_pairs_len16(&spk16, &spv, reinterpret_cast<uint16_t*>(pk2), pv2, 1, cap, total_d, nbits, ws,
                                      st));
    else if (s->onesweep)
        LV_TRY(radix_sort_onesweep(&spk, &spv, pk2, pv2, 1, cap, total_d, nbits, s->dstat, ws, st));
    else
        LV_TRY(radix_sort_pairs_len(&spk, &spv, pk2, pv2, 1, cap, total_d, nbits, ws, st));
    uint2* ranges;
    LV_TRY(ws.get("up.ranges", (size_t)nv * ntiles, &ranges));
    LV_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)nv * ntiles, st));
    if (k16)
        k_ranges<uint16_t><<<kPairGrid, 256, 0, st>>>(spk16, total_d, (uint64_t)cap, sentinel, ranges);
    else
        k_ranges<uint32_t><<<kPairGrid, 256, 0, st>>>(spk, total_d, (uint64_t)cap, sentinel, ranges);
    LV_LAUNCH();
    trace_end(tslot, st);
    if (dbg && dbg->ranges64) {
        k_export_ranges<<<grid_for(ntiles, 256), 256, 0, st>>>(ranges, ntiles, dbg->ranges64);
        LV_LAUNCH();
        *dbg->list_total = P;
        if (P <= dbg->list_cap && P > 0) {
            k_export_list<<<grid_for(P, 256), 256, 0, st>>>(spk, spv, P, ntiles, npad, srec, dbg->list);
            LV_LAUNCH();
        }
    }
    fe->L = GroupLists{ranges, spv, srec, npad};
    fe->spk = k16 ? nullptr : spk;   // (16-bit keys: only the ranks and lists are read afterwards)
    fe->np = total_d;
    fe->cap = cap;
    fe->P = P;
    return LUDVIG_OK;
}

// CUDA-core stage 6 of a group (k_composite): the list records with their
// block masks, then the per-tile composite with its shared-memory weight store.
ludvig_status composite_cc(ludvig_scene* s, const FrontEnd& fe, int nv, int width, int height, const void* feats,
                           int dtype, int d, float* num, float* den, const ChunkDebug* dbg, cudaStream_t st) {
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int ntiles = TX * TY;
    PairRec* pairs;
    LV_TRY(s->ws.get("up.pairs", (size_t)fe.cap, &pairs));
    StageScope scope(LUDVIG_STAGE_COMPOSITE, st);
    k_pair_records<<<kPairGrid, 256, 0, st>>>(fe.spk, fe.L.rank, fe.np, (uint64_t)fe.cap, ntiles, TX, fe.L.npad,
                                              fe.L.srec, pairs);
    LV_LAUNCH();
    CompositeArgs args;
    args.pairs = pairs;
    args.ranges = fe.L.ranges;
    args.ntiles = ntiles;
    args.TX = TX;
    args.width = width;
    args.height = height;
    args.feats = feats;
    args.d = d;
    args.num = num;
    args.den = den;
    args.dbg_t = dbg ? dbg->t_final : nullptr;
    args.dbg_cnt = dbg ? dbg->n_contrib : nullptr;
    args.count_den = option_count_normalise() ? 1 : 0;
    const int64_t nitems = (int64_t)nv * ntiles;
    const bool vec = (d % 4 == 0);
    if (dtype == LUDVIG_F32) {
        if (vec) return launch_composite<float, true>(args, nitems, st);
        return launch_composite<float, false>(args, nitems, st);
    }
    if (vec) return launch_composite<__nv_bfloat16, true>(args, nitems, st);
    return launch_composite<__nv_bfloat16, false>(args, nitems, st);
}

// ---------------------------------------------------------------- group pipeline

bool src_padded(const FeatSrc& f) { return f.kind == 1 || (f.kind == 2 && f.d < kPadD); }
// A few channels: the weights pass accumulates itself (no weight rows or chunk capacity).
bool src_direct(const FeatSrc& f) { return src_padded(f) && tc_direct_supported(f.d); }

// How a group's work is ordered.
struct Exec {
    bool async = false;          // device-side capacity checks; front end on the scene's front stream and
                                 // aggregation on its aggregation stream; the host never waits
    cudaStream_t st = nullptr;   // checked runs: the stream everything runs on
    int group = 0;               // index within the call (async: selects the buffer set)
    GroupDiag* diag = nullptr;   // async: the group's device record
    int* ovf = nullptr;          // async: the call's overflow word
};

// Stages 1-6 of one group: each view's num/den (its padded numerator when
// padded) += the view's W^T F and weight sums.
ludvig_status uplift_group(ludvig_scene* ctx, const GroupViews& g, int width, int height, const FeatSrc& src,
                           const Exec& ex, bool* too_many, int64_t* pair_cap = nullptr,
                           int64_t* chunk_cap = nullptr) {
    ludvig_scene* s = ctx;
    const int nv = (int)g.v.size();
    const bool padded = src_padded(src);
    const int fdt = src.kind == 2 ? LUDVIG_BF16 : src.dtype;   // the dtype the kernels read
    const int deff = padded ? kPadD : src.d;
    const bool tc = padded || use_tensor_cores(fdt, deff);
    const bool one_call = single_call(g);
    cudaStream_t sf = ex.async ? s->st_front : ex.st;
    cudaStream_t sa = ex.async ? s->st_agg : ex.st;
    const int p = ex.group & 1;
    *too_many = false;
    if (!tc && !one_call) {
        set_error("views of several calls share a group only on the tensor-core path");
        return LUDVIG_ERR_INTERNAL;
    }
    FrontEnd fe;
    LV_TRY(front_end(s, g, width, height, !ex.async, ex.async ? ex.ovf : nullptr, nullptr, sf, &fe, tc));
    if (fe.too_many) {
        *too_many = true;
        return LUDVIG_OK;
    }
    if (ex.async) LV_CUDA(cudaMemcpyAsync(&ex.diag->pairs, fe.np, sizeof(uint64_t), cudaMemcpyDeviceToDevice, sf));
    if (pair_cap) *pair_cap = fe.cap;
    if (chunk_cap) *chunk_cap = 0x7fffffff;   // no weight rows on the CUDA-core path
    const int64_t view_elems = (int64_t)width * height * src.d;
    const size_t esize = src.kind == 2 ? 1 : (src.dtype == LUDVIG_F32 ? 4 : 2);
    const int fv0 = g.v[0].fview;
    int fmax = 0;
    for (const ViewRef& r : g.v) fmax = std::max(fmax, r.fview);
    // a one-scene group's features start at its first coordinate
    const void* f0 = static_cast<const char*>(src.feats) + (size_t)fv0 * view_elems * esize;
    if (!tc) return composite_cc(s, fe, nv, width, height, f0, fdt, deff, g.v[0].num, g.v[0].den, nullptr, sf);

    // tensor cores: the operand features and the weight rows go to the
    // buffer set of parity p, free once the aggregation of group - 2 is done
    if (ex.async && ex.group >= 2) LV_CUDA(cudaStreamWaitEvent(sf, s->ev_agg[p], 0));
    static const char* const kFb[2] = {"fp8.bf16.0", "fp8.bf16.1"};
    static const char* const kPad[2] = {"pad.feats.0", "pad.feats.1"};
    AggViews av;
    for (int k = 0; k < nv; ++k) {
        av.fview[k] = g.v[(size_t)k].fview;
        av.num[k] = g.v[(size_t)k].num;
        av.den[k] = g.v[(size_t)k].den;
    }
    const void* f = src.feats;   // the array the aggregation reads, at coordinates av.fview
    int fextent = fmax + 1;
    // FP8 codes the aggregation decodes itself (no bfloat16 copy in HBM)
    const bool f8_in_kernel = src.kind == 2 && !padded && tc_e4m3_supported(src.d) &&
                              (reinterpret_cast<uintptr_t>(src.feats) & 15) == 0;
    if (src.kind == 2 && !f8_in_kernel) {
        if (!one_call) {
            set_error("FP8 codes decoded before the aggregation need a one-scene group");
            return LUDVIG_ERR_INTERNAL;
        }
        __nv_bfloat16* fb;
        const int64_t total = (int64_t)nv * view_elems;
        LV_TRY(s->ws.get(kFb[p], (size_t)total, &fb));
        k_dequant_e4m3<<<grid_for(ceil_div(total, 4), 256), 256, 0, sf>>>(static_cast<const uint8_t*>(f0),
                                                                         src.scales + fv0, view_elems, total, fb);
        LV_LAUNCH();
        f = fb;
        fextent = nv;
        for (int k = 0; k < nv; ++k) av.fview[k] = k;
    }
    if (src_direct(src)) {
        // a few channels: the weights pass adds each row's W^T F and den into
        // the (padded) numerator itself; no weight rows, no aggregation
        int* cnt = nullptr;
        LV_TRY(tc_weights_direct(fe.L, nv, width, height, fdt == LUDVIG_F32 ? 2 : 1, src.d, kPadD, f, fdt, av, s->ws,
                                 p, s->dstat, !ex.async, sf, &cnt));
        if (ex.async) {
            LV_CUDA(cudaMemcpyAsync(&ex.diag->chunks, cnt, sizeof(int), cudaMemcpyDeviceToDevice, sf));
            LV_CUDA(cudaEventRecord(s->ev_front[p], sf));
            LV_CUDA(cudaStreamWaitEvent(sa, s->ev_front[p], 0));
            LV_CUDA(cudaEventRecord(s->ev_agg[p], sa));
        }
        return LUDVIG_OK;
    }
    if (padded) {
        const int64_t npx = (int64_t)nv * width * height;
        const size_t pes = fdt == LUDVIG_F32 ? 4 : 2;
        void* fpad;
        LV_TRY(s->ws.get(kPad[p], (size_t)npx * kPadD * pes, &fpad));
        FViews fvs;
        for (int k = 0; k < nv; ++k) fvs.f[k] = av.fview[k];
        // 16-byte groups per padded pixel: 8 (float) or 4 (bfloat16)
        const int64_t groups = npx * (kPadD * (int64_t)pes / 16);
        const int64_t view_px = (int64_t)width * height;
        if (fdt == LUDVIG_F32)
            k_pad_features<float><<<grid_for(groups, 256), 256, 0, sf>>>(static_cast<const float*>(f), fvs, view_px,
                                                                         npx, src.d, static_cast<float*>(fpad));
        else
            k_pad_features<__nv_bfloat16><<<grid_for(groups, 256), 256, 0, sf>>>(
                static_cast<const __nv_bfloat16*>(f), fvs, view_px, npx, src.d, static_cast<__nv_bfloat16*>(fpad));
        LV_LAUNCH();
        f = fpad;
        fextent = nv;
        for (int k = 0; k < nv; ++k) av.fview[k] = k;
    }
    TileWeights t;
    LV_TRY(tc_weights(fe.L, nv, width, height, fdt == LUDVIG_F32 ? 2 : 1, s->ws, p, s->dstat, &s->tc_chunk_cap,
                      !ex.async, sf, &t));
    if (chunk_cap) *chunk_cap = t.cap;
    if (ex.async) {
        LV_CUDA(cudaMemcpyAsync(&ex.diag->chunks, t.counter, sizeof(int), cudaMemcpyDeviceToDevice, sf));
        LV_CUDA(cudaEventRecord(s->ev_front[p], sf));
        LV_CUDA(cudaStreamWaitEvent(sa, s->ev_front[p], 0));
    }
    LV_TRY(tc_aggregate(t, nv, width, height, f, fextent, f8_in_kernel ? kDtypeE4M3 : fdt, deff, av, s->dstat,
                        ex.async ? ex.ovf : nullptr, sa, f8_in_kernel ? src.scales : nullptr));
    if (ex.async) LV_CUDA(cudaEventRecord(s->ev_agg[p], sa));
    return LUDVIG_OK;
}

// Pixels a group of the given scratch budget may hold: its weight rows and
// lists grow with its pixels (a few hundred bytes per pixel at paper scale),
// so a group holds at most budget / 256 pixels.
int64_t group_pixels(int64_t budget) { return std::max<int64_t>(1, budget / 256); }

// Views per group: up to kMaxViews, with the per-group Gaussian scratch
// (about 120 bytes per Gaussian and view) kept within the group budget
// (LUDVIG_OPT_GROUP_MB, 2 GB by default) and the pixels within
// group_pixels(budget).
int views_per_group(int64_t n, int n_views, int64_t view_px, int64_t budget) {
    int64_t vc = std::min<int>(kMaxViews, std::max<int>(1, n_views));
    vc = std::min<int64_t>(vc, group_pixels(budget) / std::max<int64_t>(1, view_px));
    const int64_t per_view = std::max<int64_t>(1, n) * 120;
    return (int)std::max<int64_t>(1, std::min<int64_t>(vc, budget / per_view));
}

// A group run checked on `st`; a group with more pairs than one group may
// hold is split in halves (each run the same way).
ludvig_status run_checked(ludvig_scene* ctx, const GroupViews& g, int width, int height, const FeatSrc& src,
                          cudaStream_t st) {
    Exec ex;
    ex.st = st;
    bool too_many = false;
    LV_TRY(uplift_group(ctx, g, width, height, src, ex, &too_many));
    if (!too_many) return LUDVIG_OK;
    if (g.v.size() == 1) {
        set_error("view %d produces more than 2^31 tile/Gaussian pairs", g.v[0].fview);
        return LUDVIG_ERR_UNSUPPORTED;
    }
    const size_t h = g.v.size() / 2;
    for (int half = 0; half < 2; ++half) {
        GroupViews part;
        part.v.assign(g.v.begin() + (half ? h : 0), half ? g.v.end() : g.v.begin() + h);
        for (const ViewRef& r : part.v) part.nmax = std::max(part.nmax, r.scene->n);
        LV_TRY(run_checked(ctx, part, width, height, src, st));
    }
    return LUDVIG_OK;
}

// Views [v0, v0 + nv_total) of one scene's call, group by group, checked.
ludvig_status run_checked_range(ludvig_scene* s, const ludvig_camera* cams, int v0, int nv_total, int width,
                                int height, const FeatSrc& src, float* num, float* den, cudaStream_t st) {
    const int vc = views_per_group(s->n, nv_total, (int64_t)width * height, option_group_bytes());
    for (int end = v0 + nv_total; v0 < end;) {
        const int nv = std::min(vc, end - v0);
        LV_TRY(run_checked(s, scene_group(s, cams, v0, nv, num, den), width, height, src, st));
        v0 += nv;
    }
    return LUDVIG_OK;
}

// Allocates what asynchronous groups of up to nv views use at the scene's
// current capacities (both buffer sets), so that they find it in place: a
// workspace that grows synchronises the device.
// Groups of up to nv views whose largest per-view Gaussian scratch is that of
// ng views of n Gaussians.
ludvig_status reserve_async(ludvig_scene* s, int nv, int ng, int64_t n, int width, int height, const FeatSrc& src,
                            bool tc) {
    Arena& ws = s->ws;
    void* q;
    FrontBufs fb;
    LV_TRY(front_buffers(ws, ng, n, &fb));
    const int64_t cap = std::max<int64_t>(s->pair_cap, kRadixTile);
    for (const char* name : {"up.pk", "up.pv", "up.pk2", "up.pv2"}) LV_TRY(ws.get(name, sizeof(uint32_t) * (size_t)cap, &q));
    // the radix sorts' digit histograms (pairs, and the depth sort of nv views of
    // up to n Gaussians) and their scan sums
    const int64_t npad = round_up(std::max<int64_t>(n, 1), kRadixTile);
    const int64_t hist = 256 * std::max<int64_t>(cap, (int64_t)ng * npad) / kRadixTile;
    if (s->onesweep) {
        LV_TRY(ws.get("os.status", sizeof(uint64_t) * (size_t)hist, &q));
        LV_TRY(ws.get("os.hist", sizeof(uint32_t) * 4 * 256 * (size_t)std::max(ng, 1), &q));
        LV_TRY(ws.get("os.counters", sizeof(uint32_t) * 4, &q));
    } else {
        LV_TRY(ws.get("radix.hist", sizeof(uint32_t) * (size_t)hist, &q));
    }
    LV_TRY(ws.get("scan.sums", sizeof(unsigned long long) * (size_t)ceil_div(std::max(hist, (int64_t)ng * npad), 4096),
                  &q));
    if (!tc) {
        LV_TRY(ws.get("up.pairs", sizeof(PairRec) * (size_t)cap, &q));
        return LUDVIG_OK;
    }
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const bool padded = src_padded(src);
    const int fdt = src.kind == 2 ? LUDVIG_BF16 : src.dtype;
    const bool direct = src_direct(src);   // no weight rows, no padded copy
    if (!direct) LV_TRY(tc_reserve(ws, fdt == LUDVIG_F32 ? 2 : 1, nv * TX * TY, s->tc_chunk_cap));
    const int64_t npx = (int64_t)nv * width * height;
    for (int p = 0; p < 2; ++p) {
        static const char* const kFb[2] = {"fp8.bf16.0", "fp8.bf16.1"};
        static const char* const kPad[2] = {"pad.feats.0", "pad.feats.1"};
        if (src.kind == 2 && (padded || !tc_e4m3_supported(src.d) || (reinterpret_cast<uintptr_t>(src.feats) & 15)))
            LV_TRY(ws.get(kFb[p], 2 * (size_t)npx * src.d, &q));
        if (padded && !direct) LV_TRY(ws.get(kPad[p], (size_t)npx * kPadD * (fdt == LUDVIG_F32 ? 4 : 2), &q));
    }
    return LUDVIG_OK;
}

// Streams, events and status words of the asynchronous path (first use).
ludvig_status ensure_async(ludvig_scene* s, int ngroups) {
    if (!s->st_front) {
        int lo = 0, hi = 0;
        LV_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        LV_CUDA(cudaStreamCreateWithFlags(&s->st_front, cudaStreamNonBlocking));
        // the aggregation streams the features: its blocks go first when SMs free up
        LV_CUDA(cudaStreamCreateWithPriority(&s->st_agg, cudaStreamNonBlocking, hi));
        LV_CUDA(cudaEventCreateWithFlags(&s->ev_call, cudaEventDisableTiming));
        LV_CUDA(cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming));
        for (int b = 0; b < 2; ++b) {
            LV_CUDA(cudaEventCreateWithFlags(&s->ev_front[b], cudaEventDisableTiming));
            LV_CUDA(cudaEventCreateWithFlags(&s->ev_agg[b], cudaEventDisableTiming));
            LV_CUDA(cudaEventCreateWithFlags(&s->ev_join[b], cudaEventDisableTiming));
        }
    }
    if (s->diag_cap < ngroups) {
        LV_CUDA(cudaDeviceSynchronize());
        if (s->ddiag) LV_CUDA(cudaFree(s->ddiag));
        if (s->hdiag) LV_CUDA(cudaFreeHost(s->hdiag));
        s->ddiag = nullptr;
        s->hdiag = nullptr;
        s->diag_cap = 0;
        const int cap = std::max(ngroups, 16);
        LV_CUDA(cudaMalloc(&s->ddiag, sizeof(GroupDiag) * (size_t)cap));
        LV_CUDA(cudaMallocHost(&s->hdiag, sizeof(GroupDiag) * (size_t)cap));
        s->diag_cap = cap;
    }
    return LUDVIG_OK;
}

// Reads the device status word after a checked call (synchronises `st`) and
// clears it; returns its code.
ludvig_status read_status(ludvig_scene* s, cudaStream_t st) {
    LV_CUDA(cudaMemcpyAsync(s->hstat, s->dstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    const int code = s->hstat[0];
    if (code != 0) {
        LV_CUDA(cudaMemsetAsync(s->dstat, 0, sizeof(int), st));
        LV_CUDA(cudaStreamSynchronize(st));
        set_error("tensor-core kernel reported status %d (a bounded wait expired)", code);
        return (ludvig_status)code;
    }
    return LUDVIG_OK;
}

ludvig_status normalise(int64_t n, int d, const float* num, const float* den, float* out, float* beta,
                        const int* skip, cudaStream_t st) {
    StageScope scope(LUDVIG_STAGE_NORMALISE, st);
    if (d >= 32) {
        const int vec4 = (d % 4 == 0) && (reinterpret_cast<uintptr_t>(num) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(out) % 16 == 0);
        k_normalise_rows<<<(unsigned)std::min<int64_t>(ceil_div(n, 8), 152 * 64), 256, 0, st>>>(num, den, out, beta,
                                                                                               n, d, vec4, skip);
    } else {
        k_normalise<<<grid_for(n * d, 256), 256, 0, st>>>(num, den, out, beta, n, d, skip);
    }
    LV_LAUNCH();
    return LUDVIG_OK;
}

// Whether a group that ran asynchronously with the capacities (pcap, ccap)
// completed: its pairs and weight chunks fitted.
bool group_fits(const GroupDiag& gd, int64_t pcap, int64_t ccap) {
    return gd.pairs <= (uint64_t)kMaxPairs && round_up((int64_t)gd.pairs, kRadixTile) <= pcap && gd.chunks <= ccap;
}

// Waits for the scene's asynchronous call, if one is pending, and finishes it:
// groups that did not fit the workspace are redone (checked, so the workspace
// grows) and the normalisation they held back runs.  Returns the device status
// word (bounded waits) of that call and clears it.
ludvig_status resolve_pending(ludvig_scene* s) {
    if (!s->pending.active) return LUDVIG_OK;
    PendingCall pc = std::move(s->pending);
    s->pending = PendingCall();
    LV_CUDA(cudaEventSynchronize(s->ev_done));
    const int code = s->hstat[0], ovf = s->hstat[1];
    if (ovf) {
        cudaStream_t st = s->st_front;
        FeatSrc src;
        src.kind = pc.src;
        src.feats = pc.feats;
        src.scales = pc.scales;
        src.dtype = pc.dtype;
        src.d = pc.d;
        const bool padded = src_padded(src);
        float* pad_num = nullptr;
        if (padded) {
            LV_TRY(s->ws.get("pad.num", (size_t)s->n * kPadD, &pad_num));
            LV_CUDA(cudaMemsetAsync(pad_num, 0, sizeof(float) * (size_t)s->n * kPadD, st));
        }
        LV_CUDA(cudaMemsetAsync(s->dstat + 1, 0, sizeof(int), st));
        for (size_t g = 0; g < pc.v0.size(); ++g) {
            if (group_fits(s->hdiag[g], pc.pair_cap[g], pc.chunk_cap[g])) continue;
            LV_TRY(run_checked(s, scene_group(s, pc.cams.data(), pc.v0[g], pc.nv[g], padded ? pad_num : pc.num, pc.den),
                               pc.width, pc.height, src, st));
        }
        if (padded) {
            k_add_columns<<<grid_for(s->n * pc.d, 256), 256, 0, st>>>(pad_num, s->n, pc.d, pc.num);
            LV_LAUNCH();
        }
        if (pc.kind == 1) LV_TRY(normalise(s->n, pc.d, pc.num, pc.den, pc.num, nullptr, nullptr, st));
        LV_TRY(read_status(s, st));
    }
    if (code != 0) {
        LV_CUDA(cudaMemsetAsync(s->dstat, 0, sizeof(int), s->st_front));
        LV_CUDA(cudaStreamSynchronize(s->st_front));
        set_error("tensor-core kernel reported status %d (a bounded wait expired)", code);
        return (ludvig_status)code;
    }
    return LUDVIG_OK;
}

// One uplift call: kind 0 adds into num/den, kind 1 zeroes them first and
// normalises at the end (num becomes f, den stays beta).  Asynchronous unless
// `checked`: see ludvig_sync.
// Enqueues groups[first ..] on ctx's front-end and aggregation streams after
// the work on `st` (device-side capacity checks, group k - first's sizes into
// ctx->ddiag), and makes `st` wait for them; pcap/ccap receive the
// capacities each group ran with.
ludvig_status enqueue_async(ludvig_scene* s, const std::vector<GroupViews>& groups, size_t first, int width,
                            int height, const FeatSrc& src, cudaStream_t st, std::vector<int64_t>* pcap,
                            std::vector<int64_t>* ccap) {
    cudaStream_t sf = s->st_front, sa = s->st_agg;
    LV_CUDA(cudaMemsetAsync(s->dstat + 1, 0, sizeof(int), st));
    LV_CUDA(cudaEventRecord(s->ev_call, st));
    LV_CUDA(cudaStreamWaitEvent(sf, s->ev_call, 0));
    LV_CUDA(cudaStreamWaitEvent(sa, s->ev_call, 0));
    for (size_t k = first; k < groups.size(); ++k) {
        const int g = (int)(k - first);
        Exec ex;
        ex.async = true;
        ex.group = g;
        ex.diag = s->ddiag + g;
        ex.ovf = s->dstat + 1;
        bool too_many = false;
        int64_t pc = 0, cc = 0;
        LV_TRY(uplift_group(s, groups[k], width, height, src, ex, &too_many, &pc, &cc));
        pcap->push_back(pc);
        ccap->push_back(cc);
    }
    LV_CUDA(cudaEventRecord(s->ev_join[0], sf));
    LV_CUDA(cudaEventRecord(s->ev_join[1], sa));
    LV_CUDA(cudaStreamWaitEvent(st, s->ev_join[0], 0));
    LV_CUDA(cudaStreamWaitEvent(st, s->ev_join[1], 0));
    return LUDVIG_OK;
}

// Sizes ctx's workspace for asynchronous groups: when it has not been sized
// (or `always`), groups[0] runs checked first (*first = 1: the groups after
// it run asynchronously) and capacities it had to grow get headroom; then
// everything the groups allocate is reserved.
ludvig_status size_for_async(ludvig_scene* s, const std::vector<GroupViews>& groups, int width, int height,
                             const FeatSrc& src, bool tc, bool always, cudaStream_t st, size_t* first) {
    *first = 0;
    if (groups.empty()) return LUDVIG_OK;
    if (always || s->pair_cap == 0 || (tc && !src_direct(src) && s->tc_chunk_cap == 0)) {
        const int64_t pc0 = s->pair_cap, cc0 = s->tc_chunk_cap;
        LV_TRY(run_checked(s, groups[0], width, height, src, st));
        if (s->pair_cap > pc0) s->pair_cap = round_up(s->pair_cap + s->pair_cap / 4, kRadixTile);
        if (s->tc_chunk_cap > cc0) s->tc_chunk_cap += s->tc_chunk_cap / 4;
        *first = 1;
    }
    int nv = 1, ng = 1;
    int64_t n = 1;
    for (const GroupViews& g : groups) {
        nv = std::max(nv, (int)g.v.size());
        const int64_t npad = round_up(std::max<int64_t>(g.nmax, 1), kRadixTile);
        if ((int64_t)g.v.size() * npad > (int64_t)ng * round_up(n, kRadixTile)) {
            ng = (int)g.v.size();
            n = std::max<int64_t>(g.nmax, 1);
        }
    }
    return reserve_async(s, nv, ng, n, width, height, src, tc);
}

// One uplift call: kind 0 adds into num/den, kind 1 zeroes them first and
// normalises at the end (num becomes f, den stays beta).  Asynchronous unless
// `checked`: see ludvig_sync.
ludvig_status run_call(ludvig_scene* s, int kind, const FeatSrc& src, const ludvig_camera* cams, int n_views,
                       int width, int height, float* num, float* den, cudaStream_t st, bool checked) {
    LV_TRY(resolve_pending(s));
    const int64_t n = s->n;
    const int d = src.d;
    const bool padded = src_padded(src);
    float* pad_num = nullptr;
    if (kind == 1) {
        LV_CUDA(cudaMemsetAsync(num, 0, sizeof(float) * (size_t)n * d, st));
        LV_CUDA(cudaMemsetAsync(den, 0, sizeof(float) * (size_t)n, st));
    }
    if (padded) {
        LV_TRY(s->ws.get("pad.num", (size_t)n * kPadD, &pad_num));
        LV_CUDA(cudaMemsetAsync(pad_num, 0, sizeof(float) * (size_t)n * kPadD, st));
    }
    const int vc = views_per_group(n, n_views, (int64_t)width * height, option_group_bytes());
    std::vector<GroupViews> groups;
    for (int v0 = 0; v0 < n_views; v0 += vc)
        groups.push_back(scene_group(s, cams, v0, std::min(vc, n_views - v0), padded ? pad_num : num, den));
    LV_TRY(ensure_async(s, (int)groups.size()));
    const int fdt = src.kind == 2 ? LUDVIG_BF16 : src.dtype;
    const bool tc = padded || use_tensor_cores(fdt, d);
    size_t first = groups.size();
    std::vector<int64_t> gpcap, gccap;
    if (checked) {
        for (const GroupViews& g : groups) LV_TRY(run_checked(s, g, width, height, src, st));
    } else {
        LV_TRY(size_for_async(s, groups, width, height, src, tc, false, st, &first));
        if (first < groups.size()) LV_TRY(enqueue_async(s, groups, first, width, height, src, st, &gpcap, &gccap));
    }
    const bool async = first < groups.size();
    if (padded) {
        k_add_columns<<<grid_for(n * d, 256), 256, 0, st>>>(pad_num, n, d, num);
        LV_LAUNCH();
    }
    if (kind == 1) LV_TRY(normalise(n, d, num, den, num, nullptr, async ? s->dstat + 1 : nullptr, st));
    if (!async) return read_status(s, st);
    LV_CUDA(cudaMemcpyAsync(s->hstat, s->dstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaMemcpyAsync(s->hdiag, s->ddiag, sizeof(GroupDiag) * (groups.size() - first),
                            cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaEventRecord(s->ev_done, st));
    PendingCall& pc = s->pending;
    pc.kind = kind;
    pc.src = src.kind;
    pc.cams.assign(cams, cams + n_views);
    pc.n_views = n_views;
    pc.width = width;
    pc.height = height;
    pc.dtype = src.dtype;
    pc.d = d;
    pc.feats = src.feats;
    pc.scales = src.scales;
    pc.num = num;
    pc.den = den;
    pc.v0.clear();
    pc.nv.clear();
    for (size_t k = first; k < groups.size(); ++k) {
        pc.v0.push_back(groups[k].v[0].fview);
        pc.nv.push_back((int)groups[k].v.size());
    }
    pc.pair_cap = std::move(gpcap);
    pc.chunk_cap = std::move(gccap);
    pc.active = true;
    return LUDVIG_OK;
}

ludvig_status check_views(const ludvig_camera* cams, int32_t n_views, int32_t width, int32_t height) {
    LV_ARG(n_views >= 0, "n_views must be >= 0");
    LV_ARG(n_views == 0 || cams != nullptr, "cams is NULL");
    LV_ARG(width > 0 && height > 0, "width and height must be positive");
    LV_ARG(width <= 16 * 4095 && height <= 16 * 4095, "image too large");
    for (int v = 0; v < n_views; ++v) {
        LV_ARG(cams[v].fx > 0.f && cams[v].fy > 0.f, "camera %d: focal lengths must be positive", v);
    }
    return LUDVIG_OK;
}

// Rendering of one group (Eq. 4): stages 1-5, then W f per tile (checked).
ludvig_status render_group(ludvig_scene* s, const ludvig_camera* cams, int nv, int width, int height,
                           const float* f, int d, float* out, cudaStream_t st, bool* too_many) {
    FrontEnd fe;
    LV_TRY(front_end(s, scene_group(s, cams, 0, nv, nullptr, nullptr), width, height, true, nullptr, nullptr, st,
                     &fe));
    *too_many = fe.too_many;
    if (fe.too_many) return LUDVIG_OK;
    StageScope scope(LUDVIG_STAGE_RENDER, st);
    if (use_tensor_cores(LUDVIG_F32, d)) {
        TileWeights t;
        LV_TRY(tc_weights(fe.L, nv, width, height, 2, s->ws, 0, s->dstat, &s->tc_chunk_cap, true, st, &t));
        return tc_render(t, s->ws, nv, width, height, f, d, out, s->dstat, st);
    }
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    PairRec* pairs;
    LV_TRY(s->ws.get("up.pairs", (size_t)fe.cap, &pairs));
    k_pair_records<<<kPairGrid, 256, 0, st>>>(fe.spk, fe.L.rank, fe.np, (uint64_t)fe.cap, TX * TY, TX, fe.L.npad,
                                              fe.L.srec, pairs);
    LV_LAUNCH();
    RenderArgs r;
    r.pairs = pairs;
    r.ranges = fe.L.ranges;
    r.ntiles = TX * TY;
    r.TX = TX;
    r.width = width;
    r.height = height;
    r.f = f;
    r.d = d;
    r.out = out;
    const int64_t nitems = (int64_t)nv * TX * TY;
    if (d <= 4) return launch_render_cc<4>(r, nitems, st);
    if (d <= 8) return launch_render_cc<8>(r, nitems, st);
    if (d <= 16) return launch_render_cc<16>(r, nitems, st);
    return launch_render_cc<32>(r, nitems, st);
}

// First use: the status words of a scene.
ludvig_status ensure_status(ludvig_scene* s) {
    if (s->dstat) return LUDVIG_OK;
    LV_CUDA(cudaMalloc(&s->dstat, 2 * sizeof(int)));
    LV_CUDA(cudaMemset(s->dstat, 0, 2 * sizeof(int)));
    LV_CUDA(cudaMallocHost(&s->hstat, 2 * sizeof(int)));
    s->hstat[0] = s->hstat[1] = 0;
    return LUDVIG_OK;
}

}  // namespace

// ---------------------------------------------------------------- packed batches
bool packed_supported(int dtype, int d) { return use_padded(dtype, d) || use_tensor_cores(dtype, d); }

// Packed groups may take more pixels than one call's groups (a batch runs
// one context at a time): about 32 bytes of the budget per pixel and weight
// term.
int64_t packed_pixels(int64_t group_bytes, int dtype) {
    return std::max<int64_t>(1, group_bytes / (dtype == LUDVIG_F32 ? 64 : 32));
}

ludvig_status uplift_packed(ludvig_scene* ctx, const PackedJob* jobs, int njobs, const void* feats, int dtype, int d,
                            int width, int height, int64_t group_bytes, cudaStream_t st, PackedStats* stats) {
    PackedStats dummy;
    if (!stats) stats = &dummy;
    *stats = PackedStats();
    if (njobs <= 0) return LUDVIG_OK;
    if (!packed_supported(dtype, d)) {
        set_error("packed uplift needs the tensor-core path (dtype %d, d %d)", dtype, d);
        return LUDVIG_ERR_UNSUPPORTED;
    }
    FeatSrc src;
    src.kind = use_padded(dtype, d) ? 1 : 0;
    src.feats = feats;
    src.dtype = dtype;
    src.d = d;
    const bool padded = src.kind == 1;
    LV_TRY(ensure_status(ctx));
    // per job: den (beta, else the context's), the padded numerator
    int64_t nden = 0, npadn = 0;
    for (int j = 0; j < njobs; ++j) {
        if (!jobs[j].beta) nden += jobs[j].scene->n;
        if (padded) npadn += jobs[j].scene->n * kPadD;
    }
    float *den_ws = nullptr, *pad_ws = nullptr;
    if (nden) LV_TRY(ctx->ws.get("pk.den", (size_t)nden, &den_ws));
    if (npadn) LV_TRY(ctx->ws.get("pk.pad", (size_t)npadn, &pad_ws));
    std::vector<float*> den(njobs), acc(njobs);
    for (int j = 0; j < njobs; ++j) {
        const int64_t n = jobs[j].scene->n;
        den[j] = jobs[j].beta ? jobs[j].beta : den_ws;
        if (!jobs[j].beta) den_ws += n;
        acc[j] = padded ? pad_ws : jobs[j].out;
        if (padded) pad_ws += n * kPadD;
        LV_CUDA(cudaMemsetAsync(jobs[j].out, 0, sizeof(float) * (size_t)n * d, st));
        LV_CUDA(cudaMemsetAsync(den[j], 0, sizeof(float) * (size_t)n, st));
        if (padded) LV_CUDA(cudaMemsetAsync(acc[j], 0, sizeof(float) * (size_t)n * kPadD, st));
    }
    // the groups: every job's views, the jobs taken by decreasing scene size
    // (a group's views are projected and depth-sorted at its largest scene's
    // size, so views of similar scenes share groups); a group closes at
    // kMaxViews views, at group_pixels(group_bytes) pixels, or when one more
    // view would take its Gaussian scratch past the budget
    const int64_t max_views = std::max<int64_t>(1, packed_pixels(group_bytes, dtype) / ((int64_t)width * height));
    std::vector<int> order(njobs);
    for (int j = 0; j < njobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return jobs[x].scene->n > jobs[y].scene->n; });
    std::vector<GroupViews> groups;
    GroupViews cur;
    for (int j : order) {
        const ludvig_scene* sc = jobs[j].scene;
        if (sc->n == 0) continue;
        for (int v = 0; v < jobs[j].n_views; ++v) {
            int64_t nmax = std::max(cur.nmax, sc->n);
            const int64_t need = (int64_t)(cur.v.size() + 1) * round_up(nmax, kRadixTile) * 120;
            if (!cur.v.empty() &&
                ((int)cur.v.size() == kMaxViews || (int64_t)cur.v.size() == max_views || need > group_bytes)) {
                groups.push_back(std::move(cur));
                cur = GroupViews();
                nmax = sc->n;
            }
            cur.v.push_back(ViewRef{sc, jobs[j].cams[v], jobs[j].fview0 + v, acc[j], den[j]});
            cur.nmax = nmax;
        }
    }
    if (!cur.v.empty()) groups.push_back(std::move(cur));
    stats->groups = (int)groups.size();
    // on a failure, nothing of the call may still run when it returns
    struct Drain {
        ludvig_scene* c;
        cudaStream_t st;
        bool armed = true;
        ~Drain() {
            if (!armed) return;
            if (c->st_front) cudaStreamSynchronize(c->st_front);
            if (c->st_agg) cudaStreamSynchronize(c->st_agg);
            cudaStreamSynchronize(st);
        }
    } drain{ctx, st};
    if (!groups.empty()) {
        LV_TRY(ensure_async(ctx, (int)groups.size()));
        size_t first = 0;
        // the context served other classes of jobs: size it on this class's first group
        LV_TRY(size_for_async(ctx, groups, width, height, src, true, true, st, &first));
        std::vector<int64_t> gpcap, gccap;
        if (first < groups.size()) {
            LV_TRY(enqueue_async(ctx, groups, first, width, height, src, st, &gpcap, &gccap));
            LV_CUDA(cudaMemcpyAsync(ctx->hstat, ctx->dstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
            LV_CUDA(cudaMemcpyAsync(ctx->hdiag, ctx->ddiag, sizeof(GroupDiag) * (groups.size() - first),
                                    cudaMemcpyDeviceToHost, st));
            LV_CUDA(cudaEventRecord(ctx->ev_done, st));
            LV_CUDA(cudaEventSynchronize(ctx->ev_done));
            if (ctx->hstat[1]) {   // groups that did not fit: redone checked (the workspace grows)
                for (size_t k = first; k < groups.size(); ++k)
                    if (!group_fits(ctx->hdiag[k - first], gpcap[k - first], gccap[k - first])) {
                        LV_TRY(run_checked(ctx, groups[k], width, height, src, st));
                        ++stats->redone;
                    }
                LV_CUDA(cudaMemsetAsync(ctx->dstat + 1, 0, sizeof(int), st));
            }
        }
    }
    for (int j = 0; j < njobs; ++j) {
        const int64_t n = jobs[j].scene->n;
        if (n == 0) continue;
        if (padded) {
            k_add_columns<<<grid_for(n * d, 256), 256, 0, st>>>(acc[j], n, d, jobs[j].out);
            LV_LAUNCH();
        }
        LV_TRY(normalise(n, d, jobs[j].out, den[j], jobs[j].out, nullptr, nullptr, st));
    }
    drain.armed = false;
    return read_status(ctx, st);
}

// ---------------------------------------------------------------- scene
ludvig_status scene_init(ludvig_scene* s, const float* means, const float* scales, const float* quats,
                         const float* opac, int scales_are_linear, cudaStream_t st) {
    if (s->n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(s));
    k_scene_init<<<grid_for(s->n, 256), 256, 0, st>>>(means, scales, quats, opac, s->n, scales_are_linear ? 0 : 1,
                                                      s->geo, s->cov_a, s->cov_b, s->means);
    LV_LAUNCH();
    return LUDVIG_OK;
}

// Releases the asynchronous path's streams, events and status words.
void scene_release_async(ludvig_scene* s) {
    if (s->st_front) cudaStreamDestroy(s->st_front);
    if (s->st_agg) cudaStreamDestroy(s->st_agg);
    cudaEvent_t* evs[] = {&s->ev_call, &s->ev_done, &s->ev_front[0], &s->ev_front[1], &s->ev_agg[0], &s->ev_agg[1],
                          &s->ev_join[0], &s->ev_join[1]};
    for (cudaEvent_t* e : evs)
        if (*e) cudaEventDestroy(*e);
    if (s->dstat) cudaFree(s->dstat);
    if (s->hstat) cudaFreeHost(s->hstat);
    if (s->ddiag) cudaFree(s->ddiag);
    if (s->hdiag) cudaFreeHost(s->hdiag);
}

// Finishes a scene's pending asynchronous call (ludvig_sync).
ludvig_status scene_sync(ludvig_scene* s) { return resolve_pending(s); }

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_sync(ludvig_scene_t scene) {
    LV_ARG(scene != nullptr, "scene is NULL");
    return scene_sync(scene);
}

extern "C" ludvig_status ludvig_uplift_accumulate(ludvig_scene_t scene, const ludvig_camera* cams,
                                                  int32_t n_views, int32_t width, int32_t height,
                                                  const void* feats, int32_t dtype, int32_t d,
                                                  float* num, float* den, void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_TRY(check_views(cams, n_views, width, height));
    LV_ARG(dtype == LUDVIG_F32 || dtype == LUDVIG_BF16, "unknown dtype %d", dtype);
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_ARG(num != nullptr && den != nullptr, "num/den is NULL");
    LV_ARG(n_views == 0 || feats != nullptr, "feats is NULL");
    if (d % 4 == 0) LV_ARG(((uintptr_t)num & 15) == 0, "num must be 16-byte aligned when d %% 4 == 0");
    if (scene->n == 0 || n_views == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    FeatSrc src;
    src.kind = use_padded(dtype, d) ? 1 : 0;
    src.feats = feats;
    src.dtype = dtype;
    src.d = d;
    return run_call(scene, 0, src, cams, n_views, width, height, num, den, static_cast<cudaStream_t>(stream), false);
}

extern "C" ludvig_status ludvig_uplift_finalize(int64_t n, int32_t d, const float* num, const float* den,
                                                float* out, float* beta, void* stream) {
    LV_ARG(n >= 0 && d >= 1, "bad sizes");
    if (n == 0) return LUDVIG_OK;
    LV_ARG(num != nullptr && den != nullptr && out != nullptr, "NULL buffer");
    return normalise(n, d, num, den, out, beta, nullptr, static_cast<cudaStream_t>(stream));
}

namespace ludvig {
ludvig_status check_uplift_args(const ludvig_scene* scene, const ludvig_camera* cams, int32_t n_views, int32_t width,
                                int32_t height, const void* feats, int32_t dtype, int32_t d, const float* out) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(out != nullptr || scene->n == 0, "out is NULL");
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_TRY(check_views(cams, n_views, width, height));
    LV_ARG(dtype == LUDVIG_F32 || dtype == LUDVIG_BF16, "unknown dtype %d", dtype);
    LV_ARG(n_views == 0 || feats != nullptr, "feats is NULL");
    if (d % 4 == 0) LV_ARG(((uintptr_t)out & 15) == 0, "out must be 16-byte aligned when d %% 4 == 0");
    return LUDVIG_OK;
}
}  // namespace ludvig

extern "C" ludvig_status ludvig_uplift(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                       int32_t width, int32_t height, const void* feats, int32_t dtype,
                                       int32_t d, float* out, float* beta, void* stream) {
    LV_TRY(check_uplift_args(scene, cams, n_views, width, height, feats, dtype, d, out));
    const int64_t n = scene->n;
    if (n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    float* den = beta;
    if (!den) LV_TRY(scene->ws.get("uplift.den", (size_t)n, &den));
    FeatSrc src;
    src.kind = use_padded(dtype, d) ? 1 : 0;
    src.feats = feats;
    src.dtype = dtype;
    src.d = d;
    return run_call(scene, 1, src, cams, n_views, width, height, out, den, static_cast<cudaStream_t>(stream), false);
}

extern "C" ludvig_status ludvig_uplift_fp8(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                           int32_t width, int32_t height, const uint8_t* q, const float* scales,
                                           int32_t d, float* out, float* beta, void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(out != nullptr || scene->n == 0, "out is NULL");
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_TRY(check_views(cams, n_views, width, height));
    LV_ARG(n_views == 0 || (q != nullptr && scales != nullptr), "q/scales is NULL");
    LV_ARG(((uintptr_t)q & 3) == 0, "q must be 4-byte aligned");
    if (d % 4 == 0) LV_ARG(((uintptr_t)out & 15) == 0, "out must be 16-byte aligned when d %% 4 == 0");
    const int64_t n = scene->n;
    if (n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    float* den = beta;
    if (!den) LV_TRY(scene->ws.get("uplift.den", (size_t)n, &den));
    FeatSrc src;
    src.kind = 2;
    src.feats = q;
    src.scales = scales;
    src.dtype = LUDVIG_BF16;
    src.d = d;
    return run_call(scene, 1, src, cams, n_views, width, height, out, den, static_cast<cudaStream_t>(stream), false);
}

extern "C" ludvig_status ludvig_render(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                       int32_t width, int32_t height, const float* f, int32_t d, float* out,
                                       void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_TRY(check_views(cams, n_views, width, height));
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_ARG(n_views == 0 || out != nullptr, "out is NULL");
    LV_ARG(scene->n == 0 || n_views == 0 || f != nullptr, "f is NULL");
    if (n_views == 0) return LUDVIG_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (scene->n == 0) {
        LV_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n_views * height * width * d, st));
        return LUDVIG_OK;
    }
    if (use_tensor_cores(LUDVIG_F32, d)) {
        LV_ARG(((uintptr_t)f & 15) == 0, "f must be 16-byte aligned");
    }
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    const int64_t view_elems = (int64_t)width * height * d;
    int vc = views_per_group(scene->n, n_views, (int64_t)width * height, option_group_bytes());
    int v0 = 0;
    while (v0 < n_views) {
        const int nv = std::min(vc, n_views - v0);
        bool too_many = false;
        LV_TRY(render_group(scene, cams + v0, nv, width, height, f, d, out + (size_t)v0 * view_elems, st, &too_many));
        if (too_many) {
            if (nv == 1) {
                set_error("view %d produces more than 2^31 tile/Gaussian pairs", v0);
                return LUDVIG_ERR_UNSUPPORTED;
            }
            vc = std::max(1, nv / 2);
            continue;
        }
        v0 += nv;
    }
    return read_status(scene, st);
}

extern "C" ludvig_status ludvig_uplift_host(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                            int32_t width, int32_t height, const void* feats, int32_t dtype,
                                            int32_t d, float* out, float* beta, void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(out != nullptr || scene->n == 0, "out is NULL");
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_ARG(dtype == LUDVIG_F32 || dtype == LUDVIG_BF16, "unknown dtype %d", dtype);
    LV_ARG(n_views == 0 || feats != nullptr, "feats is NULL");
    LV_TRY(check_views(cams, n_views, width, height));
    const int64_t n = scene->n;
    if (n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!scene->copy_stream) {
        LV_CUDA(cudaStreamCreateWithFlags(&scene->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            LV_CUDA(cudaEventCreateWithFlags(&scene->ev_ready[b], cudaEventDisableTiming));
            LV_CUDA(cudaEventCreateWithFlags(&scene->ev_free[b], cudaEventDisableTiming));
        }
    }
    const size_t esize = dtype == LUDVIG_F32 ? 4 : 2;
    const size_t view_bytes = (size_t)width * height * d * esize;
    // views per upload: about 1 GB per buffer, at least one view
    const int vc = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(1, n_views),
                                                            ((size_t)1 << 30) / std::max<size_t>(1, view_bytes)));
    void* fbuf[2];
    LV_TRY(scene->ws.get("host.f0", vc * view_bytes, &fbuf[0]));
    LV_TRY(scene->ws.get("host.f1", vc * view_bytes, &fbuf[1]));
    float *num, *den;
    LV_TRY(scene->ws.get("host.num", (size_t)n * d, &num));
    LV_TRY(scene->ws.get("host.den", (size_t)n, &den));
    LV_CUDA(cudaMemsetAsync(num, 0, sizeof(float) * (size_t)n * d, st));
    LV_CUDA(cudaMemsetAsync(den, 0, sizeof(float) * (size_t)n, st));
    FeatSrc src;
    src.kind = use_padded(dtype, d) ? 1 : 0;
    src.dtype = dtype;
    src.d = d;
    float* pad_num = nullptr;
    if (src.kind == 1) {
        LV_TRY(scene->ws.get("pad.num", (size_t)n * kPadD, &pad_num));
        LV_CUDA(cudaMemsetAsync(pad_num, 0, sizeof(float) * (size_t)n * kPadD, st));
    }
    // both buffers start free once the zeroing above is ordered
    for (int b = 0; b < 2; ++b) LV_CUDA(cudaEventRecord(scene->ev_free[b], st));
    const int nchunks = (int)ceil_div(n_views, vc);
    auto upload = [&](int c) -> ludvig_status {
        const int b = c & 1, v0 = c * vc, nv = std::min(vc, n_views - v0);
        LV_CUDA(cudaStreamWaitEvent(scene->copy_stream, scene->ev_free[b], 0));
        LV_CUDA(cudaMemcpyAsync(fbuf[b], static_cast<const char*>(feats) + (size_t)v0 * view_bytes,
                                (size_t)nv * view_bytes, cudaMemcpyHostToDevice, scene->copy_stream));
        LV_CUDA(cudaEventRecord(scene->ev_ready[b], scene->copy_stream));
        return LUDVIG_OK;
    };
    if (nchunks > 0) LV_TRY(upload(0));
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1, v0 = c * vc, nv = std::min(vc, n_views - v0);
        if (c + 1 < nchunks) LV_TRY(upload(c + 1));   // overlaps the compute of chunk c
        LV_CUDA(cudaStreamWaitEvent(st, scene->ev_ready[b], 0));
        src.feats = fbuf[b];
        LV_TRY(run_checked_range(scene, cams + v0, 0, nv, width, height, src, pad_num ? pad_num : num, den, st));
        LV_CUDA(cudaEventRecord(scene->ev_free[b], st));
    }
    if (pad_num) {
        k_add_columns<<<grid_for(n * d, 256), 256, 0, st>>>(pad_num, n, d, num);
        LV_LAUNCH();
    }
    LV_TRY(normalise(n, d, num, den, num, nullptr, nullptr, st));
    LV_CUDA(cudaMemcpyAsync(out, num, sizeof(float) * (size_t)n * d, cudaMemcpyDeviceToHost, st));
    if (beta) LV_CUDA(cudaMemcpyAsync(beta, den, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st));
    return read_status(scene, st);
}

extern "C" ludvig_status ludvig_debug_scene_timeout(ludvig_scene_t scene, int64_t cycles, void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(cycles >= 0 && cycles <= 4000000000ll, "cycles must be in [0, 4e9]");
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    LV_TRY(ensure_async(scene, 1));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LV_TRY(tc_wait_into_status(cycles, scene->dstat, st));
    LV_CUDA(cudaMemcpyAsync(scene->hstat, scene->dstat, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaEventRecord(scene->ev_done, st));
    scene->pending = PendingCall();
    scene->pending.kind = 2;   // nothing to redo: the status alone
    scene->pending.active = true;
    return LUDVIG_OK;
}

// ---------------------------------------------------------------- inspection
extern "C" ludvig_status ludvig_debug_project(ludvig_scene_t scene, const ludvig_camera* cam, int32_t width,
                                              int32_t height, float* rec, int32_t* rect, void* stream) {
    LV_ARG(scene != nullptr && rec != nullptr && rect != nullptr, "NULL argument");
    LV_TRY(check_views(cam, 1, width, height));
    if (scene->n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    ChunkDebug dbg;
    dbg.rec = rec;
    dbg.rect = rect;
    dbg.stop_after_project = true;
    FrontEnd fe;
    return front_end(scene, scene_group(scene, cam, 0, 1, nullptr, nullptr), width, height, true, nullptr, &dbg,
                     static_cast<cudaStream_t>(stream), &fe);
}

extern "C" ludvig_status ludvig_debug_tile_lists(ludvig_scene_t scene, const ludvig_camera* cam,
                                                 int32_t width, int32_t height, int32_t pruned,
                                                 int64_t* ranges, int32_t* list, int64_t cap,
                                                 int64_t* total, void* stream) {
    LV_ARG(scene != nullptr && ranges != nullptr && total != nullptr, "NULL argument");
    LV_TRY(check_views(cam, 1, width, height));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t ntiles = (int64_t)((width + 15) / 16) * ((height + 15) / 16);
    if (scene->n == 0) {
        LV_CUDA(cudaMemsetAsync(ranges, 0, sizeof(int64_t) * 2 * ntiles, st));
        *total = 0;
        return LUDVIG_OK;
    }
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    ChunkDebug dbg;
    dbg.ranges64 = ranges;
    dbg.list = list;
    dbg.list_cap = list ? cap : 0;
    dbg.list_total = total;
    dbg.stop_after_sort = true;
    dbg.unpruned = (pruned == 0);
    FrontEnd fe;
    LV_TRY(front_end(scene, scene_group(scene, cam, 0, 1, nullptr, nullptr), width, height, true, nullptr, &dbg, st,
                     &fe));
    if (fe.too_many) {
        set_error("too many pairs");
        return LUDVIG_ERR_UNSUPPORTED;
    }
    LV_CUDA(cudaStreamSynchronize(st));
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_debug_transmittance(ludvig_scene_t scene, const ludvig_camera* cam,
                                                    int32_t width, int32_t height, float* t_final,
                                                    int32_t* n_contrib, void* stream) {
    LV_ARG(scene != nullptr && t_final != nullptr && n_contrib != nullptr, "NULL argument");
    LV_TRY(check_views(cam, 1, width, height));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t npx = (int64_t)width * height;
    k_debug_fill<<<grid_for(npx, 256), 256, 0, st>>>(t_final, n_contrib, npx);
    LV_LAUNCH();
    if (scene->n == 0) return LUDVIG_OK;
    LV_TRY(ensure_status(scene));
    LV_TRY(resolve_pending(scene));
    float* num;
    float* den;
    LV_TRY(scene->ws.get("dbg.num", (size_t)scene->n, &num));
    LV_TRY(scene->ws.get("dbg.den", (size_t)scene->n, &den));
    float* fz;
    LV_TRY(scene->ws.get("dbg.feat", (size_t)npx, &fz));
    LV_CUDA(cudaMemsetAsync(fz, 0, sizeof(float) * npx, st));
    ChunkDebug dbg;
    dbg.t_final = t_final;
    dbg.n_contrib = n_contrib;
    FrontEnd fe;
    LV_TRY(front_end(scene, scene_group(scene, cam, 0, 1, nullptr, nullptr), width, height, true, nullptr, nullptr,
                     st, &fe));
    if (fe.too_many) {
        set_error("too many pairs");
        return LUDVIG_ERR_UNSUPPORTED;
    }
    return composite_cc(scene, fe, 1, width, height, fz, LUDVIG_F32, 1, num, den, &dbg, st);
}
