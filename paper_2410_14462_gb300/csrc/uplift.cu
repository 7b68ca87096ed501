// Uplifting of 2D feature maps onto a Gaussian Splatting scene
// (Sec. 3.2, Eq. 3 / Eq. 5): f_i = sum_{v,p} w_i(v,p) F_v[p] / sum_{v,p} w_i(v,p)
// with w the alpha-blending weights of Sec. 3.1 (Eq. 1).
//
// Pipeline per chunk of up to kMaxViews views (all stages are batched over the
// chunk's views):
//   1. project     one thread per (view, Gaussian): EWA footprint, depth key,
//                  tile rectangle, number of tiles touched
//   2. depth sort  stable radix sort of (depth bits, index) per view
//   3. bin         exclusive scan of tiles-touched in depth order, then one
//                  (view*tiles + tile, index) pair per touched tile
//   4. tile sort   stable radix sort of the pairs by (view, tile): every
//                  tile's list stays in (depth, index) order
//   5. ranges      [start, end) of every (view, tile) list, and the lists
//                  rewritten as 32-byte records (projected Gaussian, index,
//                  8x4 block mask) that the compositing kernels stream
//   6. composite + aggregate: on the tensor cores (uplift_tc.cu: weight rows
//                  of every tile, then W^T F by tcgen05) for d < 32 (features
//                  zero-padded to 32 channels) and for 32 <= d <= 512 with
//                  d % 8 == 0; otherwise here on CUDA cores, one CTA (256
//                  threads = 16x16 pixels) per
//                  (view, tile): walk the list in batches of 32 Gaussians,
//                  form w = alpha T per pixel, keep the non-zero weights of
//                  the tile in a shared-memory sparse store grouped by
//                  Gaussian, then multiply the store with the tile's feature
//                  rows (staged in shared memory by channel chunks) and add
//                  every Gaussian's partial sum into num / den with vector
//                  reductions.
//   7. normalise   f = num / den (den > 0), beta = den.
//
// Rendering (Eq. 4, F_hat = W f) runs stages 1-5 unchanged and replaces
// stage 6 by the transposed product: every pixel's sum of w_i(p) f_i over its
// contributors, written to the view's feature map.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "spec.cuh"

namespace ludvig {

constexpr int kMaxViews = 16;

bool tc_supported(int dtype, int d);
bool option_f32_tensor_cores();
bool option_count_normalise();
ludvig_status composite_tc(const PairRec* pairs, const uint2* ranges, int nv, int width, int height,
                           const void* feats, int dtype, int d, float* num, float* den, Arena& ws, int* status,
                           int64_t* chunk_cap, cudaStream_t st);
ludvig_status render_tc(const PairRec* pairs, const uint2* ranges, int nv, int width, int height, const float* f,
                        int d, float* out, Arena& ws, int* status, int64_t* chunk_cap, cudaStream_t st);

// Per-Gaussian features rendered into the views of a chunk (Eq. 4).
struct RenderJob {
    const float* f;   // device [n, d]
    float* out;       // device [views of the chunk, H, W, d]
};

struct CamBatch {
    Cam cam[kMaxViews];
};

// Whether a request's aggregation runs on the tensor cores (else CUDA cores).
bool use_tensor_cores(int dtype, int d) {
    if (!tc_supported(dtype, d)) return false;
    return dtype == LUDVIG_BF16 || option_f32_tensor_cores();
}

namespace {

// ------------------------------------------------------------ scene setup
__global__ void k_scene_init(const float* __restrict__ means, const float* __restrict__ scales,
                             const float* __restrict__ quats, const float* __restrict__ opac,
                             int64_t n, float4* __restrict__ geo, float4* __restrict__ cov_a,
                             float2* __restrict__ cov_b, float* __restrict__ means_copy) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float m[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
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

__global__ void __launch_bounds__(256) k_project(const float4* __restrict__ geo, const float4* __restrict__ cov_a,
                          const float2* __restrict__ cov_b, int64_t n, int64_t npad, int nv,
                          CamBatch cb, int width, int height, float4* __restrict__ rec_a,
                          float2* __restrict__ rec_b, uint2* __restrict__ rect,
                          uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                          uint32_t* __restrict__ ntile, float* __restrict__ dbg_rec,
                          int32_t* __restrict__ dbg_rect, int prune) {
    // every block is full: nv * npad is a multiple of the block size
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = (int)(idx / npad);
    const int64_t i = idx - (int64_t)v * npad;
    const bool real = i < n;
    Projected P{};
    float op = 0.f;
    if (real) {
        const float4 g = geo[i];
        const float4 ca = cov_a[i];
        const float2 cbv = cov_b[i];
        const float m[3] = {g.x, g.y, g.z};
        const float S6[6] = {ca.x, ca.y, ca.z, ca.w, cbv.x, cbv.y};
        P = project_gaussian(m, S6, cb.cam[v], width, height);
        op = g.w;
        const int64_t o = (int64_t)v * n + i;
        rec_a[o] = make_float4(P.mx, P.my, P.ca, P.cb);
        rec_b[o] = make_float2(P.cc, g.w);
        rect[o] = P.visible ? make_uint2((uint32_t)P.x0 | ((uint32_t)P.y0 << 16),
                                         (uint32_t)P.x1 | ((uint32_t)P.y1 << 16))
                            : make_uint2(0u, 0u);
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
__global__ void k_gather_counts(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                                const uint32_t* __restrict__ ntile, int64_t npad, int64_t total,
                                uint32_t* __restrict__ cnt) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t v = idx / npad;
    cnt[idx] = skeys[idx] == 0xffffffffu ? 0u : ntile[v * npad + svals[idx]];
}

__global__ void k_emit_pairs(const uint32_t* __restrict__ svals, const uint32_t* __restrict__ cnt,
                             const uint32_t* __restrict__ off, const uint2* __restrict__ rect,
                             const float4* __restrict__ rec_a, const float2* __restrict__ rec_b,
                             int64_t n, int64_t npad, int64_t total, int TX, int ntiles, int prune,
                             uint32_t sentinel, uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const uint32_t c = cnt[idx];
    if (c == 0) return;
    const int64_t v = idx / npad;
    const uint32_t i = svals[idx];
    const uint2 r = rect[v * n + i];
    const int x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff, y1 = r.y >> 16;
    const float4 ra = rec_a[v * n + i];
    const float2 rb = rec_b[v * n + i];
    EllipseX E{};
    E.state = 2;   // unpruned: every tile of the rectangle
    if (prune) E = ellipse_prep(reach_prep(ra.z, ra.w, rb.x, rb.y), ra.z, ra.w, rb.x);
    uint32_t o = off[idx];
    const uint32_t end = o + c;   // never write past the counted slots
    const uint32_t base = (uint32_t)(v * ntiles);
    for (int ty = y0; ty < y1 && o < end; ++ty) {
        int c0, c1;
        tile_row_range(E, ra.x, ra.y, ty, x0, x1, c0, c1);
        for (int tx = c0; tx < c1 && o < end; ++tx, ++o) {
            pkey[o] = base + (uint32_t)(ty * TX + tx);
            pval[o] = i;
        }
    }
    for (; o < end; ++o) {   // unreachable when both kernels agree; keeps the keys defined
        pkey[o] = sentinel;
        pval[o] = 0u;
    }
}

__global__ void k_fill(uint32_t* __restrict__ a, uint32_t value, int64_t from, int64_t to) {
    const int64_t j = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < to) a[j] = value;
}

// ------------------------------------------------------------ 5. ranges
__global__ void k_ranges(const uint32_t* __restrict__ pkey, int64_t P, uint32_t nkeys,
                         uint2* __restrict__ ranges) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const uint32_t k = pkey[j];
    if (k >= nkeys) return;
    if (j == 0 || pkey[j - 1] != k) ranges[k].x = (uint32_t)j;
    if (j == P - 1 || pkey[j + 1] != k) ranges[k].y = (uint32_t)(j + 1);
}

// The sorted lists as the compositing kernels stream them: one 32-byte record
// per entry, in list order, with the entry's 8x4 block mask.
__global__ void k_pair_records(const uint32_t* __restrict__ pkey, const uint32_t* __restrict__ pval, int64_t P,
                               int ntiles, int TX, int64_t n, const float4* __restrict__ rec_a,
                               const float2* __restrict__ rec_b, PairRec* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const uint32_t key = pkey[j], g = pval[j];
    const uint32_t v = key / (uint32_t)ntiles, tile = key - v * (uint32_t)ntiles;
    const int tx = (int)(tile % (uint32_t)TX), ty = (int)(tile / (uint32_t)TX);
    const float4 ra = rec_a[(int64_t)v * n + g];
    const float2 rb = rec_b[(int64_t)v * n + g];
    PairRec r;
    r.mx = ra.x;
    r.my = ra.y;
    r.ca = ra.z;
    r.cb = ra.w;
    r.cc = rb.x;
    r.op = rb.y;
    r.gid = g;
    r.mask = block_mask(reach_prep(ra.z, ra.w, rb.x, rb.y), ra.x, ra.y, ra.z, ra.w, rb.x, tx, ty);
    out[j] = r;
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
__global__ void k_normalise(const float* num, const float* __restrict__ den, float* out, float* beta,
                            int64_t n, int d) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * d) return;
    const int64_t i = idx / d;
    const float b = den[i];
    out[idx] = b > 0.f ? num[idx] / b : 0.f;
    if (beta && idx % d == 0) beta[i] = b;
}

// Same, one warp per Gaussian (d >= 32), float4 accesses when vec4 (d % 4 == 0
// and 16-byte aligned rows).
__global__ void k_normalise_rows(const float* num, const float* __restrict__ den, float* out, float* beta,
                                 int64_t n, int d, int vec4) {
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

__global__ void k_copy_u32_i32(const uint32_t* __restrict__ a, int32_t* __restrict__ b, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (int32_t)a[t];
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

// One chunk of views: stages 1-6 (stage 6 renders instead when `rj` is set).
ludvig_status run_chunk(ludvig_scene* s, const ludvig_camera* cams, int nv, int width, int height,
                        const void* feats, int dtype, int d, float* num, float* den, cudaStream_t st,
                        const ChunkDebug* dbg, bool* too_many_pairs, const RenderJob* rj = nullptr) {
    Arena& ws = s->ws;
    const int64_t n = s->n;
    const int64_t npad = round_up(n, kRadixTile);
    const int TX = (width + kTile - 1) / kTile, TY = (height + kTile - 1) / kTile;
    const int ntiles = TX * TY;
    const int64_t nG = (int64_t)nv * npad;
    const int prune = (dbg && dbg->unpruned) ? 0 : 1;
    *too_many_pairs = false;

    float4* rec_a;
    float2* rec_b;
    uint2* rect;
    uint32_t *keys, *vals, *keys2, *vals2, *ntile, *cnt, *off;
    uint64_t* total_d;
    LV_TRY(ws.get("up.rec_a", (size_t)nv * n, &rec_a));
    LV_TRY(ws.get("up.rec_b", (size_t)nv * n, &rec_b));
    LV_TRY(ws.get("up.rect", (size_t)nv * n, &rect));
    LV_TRY(ws.get("up.keys", (size_t)nG, &keys));
    LV_TRY(ws.get("up.vals", (size_t)nG, &vals));
    LV_TRY(ws.get("up.keys2", (size_t)nG, &keys2));
    LV_TRY(ws.get("up.vals2", (size_t)nG, &vals2));
    LV_TRY(ws.get("up.ntile", (size_t)nG, &ntile));
    LV_TRY(ws.get("up.cnt", (size_t)nG, &cnt));
    LV_TRY(ws.get("up.off", (size_t)nG, &off));
    LV_TRY(ws.get("up.total", 1, &total_d));
    uint64_t* total_h = nullptr;
    {
        void* p;
        LV_TRY(ws.pinned("up.total_h", 16, &p));
        total_h = static_cast<uint64_t*>(p);
    }

    CamBatch cb;
    for (int v = 0; v < nv; ++v) {
        const ludvig_camera& c = cams[v];
        for (int k = 0; k < 9; ++k) cb.cam[v].R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) cb.cam[v].t[k] = c.t[k];
        cb.cam[v].fx = c.fx;
        cb.cam[v].fy = c.fy;
        cb.cam[v].cx = c.cx;
        cb.cam[v].cy = c.cy;
    }
    int tslot = trace_on() ? trace_begin(LUDVIG_STAGE_PROJECT, st) : -1;
    k_project<<<grid_for(nG, 256), 256, 0, st>>>(s->geo, s->cov_a, s->cov_b, n, npad, nv, cb, width,
                                                  height, rec_a, rec_b, rect, keys, vals, ntile,
                                                  dbg ? dbg->rec : nullptr, dbg ? dbg->rect : nullptr,
                                                  prune);
    LV_LAUNCH();
    trace_end(tslot, st);
    if (dbg && dbg->stop_after_project) return LUDVIG_OK;

    uint32_t *sk = keys, *sv = vals;
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_DEPTH_SORT, st) : -1;
    LV_TRY(radix_sort_pairs(&sk, &sv, keys2, vals2, nv, npad, 32, ws, st));
    trace_end(tslot, st);
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_BIN, st) : -1;
    k_gather_counts<<<grid_for(nG, 256), 256, 0, st>>>(sk, sv, ntile, npad, nG, cnt);
    LV_LAUNCH();
    LV_TRY(scan_exclusive_u32(cnt, off, nG, total_d, ws, st));
    LV_CUDA(cudaMemcpyAsync(total_h, total_d, 8, cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    const int64_t P = (int64_t)*total_h;
    if (P > (int64_t)0x7fffffff - 2 * kRadixTile) {
        *too_many_pairs = true;
        return LUDVIG_OK;
    }
    const int64_t Ppad = round_up(std::max<int64_t>(P, 1), kRadixTile);
    const uint32_t sentinel = (uint32_t)nv * (uint32_t)ntiles;
    uint32_t *pk, *pv, *pk2, *pv2;
    LV_TRY(ws.get("up.pk", (size_t)Ppad, &pk));
    LV_TRY(ws.get("up.pv", (size_t)Ppad, &pv));
    LV_TRY(ws.get("up.pk2", (size_t)Ppad, &pk2));
    LV_TRY(ws.get("up.pv2", (size_t)Ppad, &pv2));
    k_emit_pairs<<<grid_for(nG, 256), 256, 0, st>>>(sv, cnt, off, rect, rec_a, rec_b, n, npad, nG, TX, ntiles,
                                                     prune, sentinel, pk, pv);
    LV_LAUNCH();
    trace_end(tslot, st);
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_TILE_SORT, st) : -1;
    if (Ppad > P) {
        k_fill<<<grid_for(Ppad - P, 256), 256, 0, st>>>(pk, sentinel, P, Ppad);
        LV_LAUNCH();
        k_fill<<<grid_for(Ppad - P, 256), 256, 0, st>>>(pv, 0u, P, Ppad);
        LV_LAUNCH();
    }
    int nbits = 1;
    while (((uint32_t)1 << nbits) <= sentinel) ++nbits;
    uint32_t *spk = pk, *spv = pv;
    LV_TRY(radix_sort_pairs(&spk, &spv, pk2, pv2, 1, Ppad, nbits, ws, st));
    uint2* ranges;
    LV_TRY(ws.get("up.ranges", (size_t)nv * ntiles, &ranges));
    LV_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)nv * ntiles, st));
    if (P > 0) {
        k_ranges<<<grid_for(P, 256), 256, 0, st>>>(spk, P, sentinel, ranges);
        LV_LAUNCH();
    }
    trace_end(tslot, st);
    if (dbg && dbg->ranges64) {
        k_export_ranges<<<grid_for(ntiles, 256), 256, 0, st>>>(ranges, ntiles, dbg->ranges64);
        LV_LAUNCH();
        *dbg->list_total = P;
        if (P <= dbg->list_cap && P > 0) {
            k_copy_u32_i32<<<grid_for(P, 256), 256, 0, st>>>(spv, dbg->list, P);
            LV_LAUNCH();
        }
    }
    if (dbg && dbg->stop_after_sort) return LUDVIG_OK;

    PairRec* pairs;
    LV_TRY(ws.get("up.pairs", (size_t)std::max<int64_t>(P, 1), &pairs));
    tslot = trace_on() ? trace_begin(LUDVIG_STAGE_TILE_SORT, st) : -1;
    if (P > 0) {
        k_pair_records<<<grid_for(P, 256), 256, 0, st>>>(spk, spv, P, ntiles, TX, n, rec_a, rec_b, pairs);
        LV_LAUNCH();
    }
    trace_end(tslot, st);

    const int64_t nitems = (int64_t)nv * ntiles;
    if (rj) {
        StageScope scope(LUDVIG_STAGE_RENDER, st);
        if (use_tensor_cores(LUDVIG_F32, d)) {
            int* status;
            LV_TRY(ws.get("tc.status", 1, &status));
            return render_tc(pairs, ranges, nv, width, height, rj->f, d, rj->out, ws, status, &s->tc_chunk_cap,
                             st);
        }
        RenderArgs r;
        r.pairs = pairs;
        r.ranges = ranges;
        r.ntiles = ntiles;
        r.TX = TX;
        r.width = width;
        r.height = height;
        r.f = rj->f;
        r.d = d;
        r.out = rj->out;
        if (d <= 4) return launch_render_cc<4>(r, nitems, st);
        if (d <= 8) return launch_render_cc<8>(r, nitems, st);
        if (d <= 16) return launch_render_cc<16>(r, nitems, st);
        return launch_render_cc<32>(r, nitems, st);
    }
    CompositeArgs args;
    args.pairs = pairs;
    args.ranges = ranges;
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
    const bool vec = (d % 4 == 0);
    StageScope scope(LUDVIG_STAGE_COMPOSITE, st);
    if (use_tensor_cores(dtype, d)) {
        int* status;
        LV_TRY(ws.get("tc.status", 1, &status));
        return composite_tc(pairs, ranges, nv, width, height, feats, dtype, d, num, den, ws, status,
                            &s->tc_chunk_cap, st);
    }
    if (dtype == LUDVIG_F32) {
        if (vec) return launch_composite<float, true>(args, nitems, st);
        return launch_composite<float, false>(args, nitems, st);
    }
    if (vec) return launch_composite<__nv_bfloat16, true>(args, nitems, st);
    return launch_composite<__nv_bfloat16, false>(args, nitems, st);
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

ludvig_status accumulate(ludvig_scene* s, const ludvig_camera* cams, int32_t n_views, int32_t width,
                         int32_t height, const void* feats, int32_t dtype, int32_t d, float* num,
                         float* den, cudaStream_t st, const ChunkDebug* dbg, const RenderJob* rj = nullptr) {
    const size_t esize = dtype == LUDVIG_F32 ? 4 : 2;
    const int64_t view_elems = (int64_t)width * height * d;
    int* status = nullptr;
    if (use_tensor_cores(dtype, d)) {
        LV_TRY(s->ws.get("tc.status", 1, &status));
        LV_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    }
    int v0 = 0;
    int vc = std::min<int>(kMaxViews, std::max<int>(1, n_views));
    // keep the per-chunk Gaussian scratch (about 80 bytes per Gaussian and view) near 2 GB
    const int64_t per_view = std::max<int64_t>(1, s->n) * 80;
    vc = (int)std::max<int64_t>(1, std::min<int64_t>(vc, ((int64_t)2 << 30) / per_view));
    while (v0 < n_views) {
        const int nv = std::min(vc, n_views - v0);
        bool too_many = false;
        const char* fp = feats ? static_cast<const char*>(feats) + (size_t)v0 * view_elems * esize : nullptr;
        RenderJob part{};
        if (rj) part = RenderJob{rj->f, rj->out + (size_t)v0 * view_elems};
        LV_TRY(run_chunk(s, cams + v0, nv, width, height, fp, dtype, d, num, den, st, dbg, &too_many,
                         rj ? &part : nullptr));
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
    if (status) {
        // device-side status of the tensor-core kernel (bounded waits)
        void* h;
        LV_TRY(s->ws.pinned("tc.status_h", 16, &h));
        LV_CUDA(cudaMemcpyAsync(h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        const int code = *static_cast<int*>(h);
        if (code != 0) {
            set_error("tensor-core kernel reported status %d (a bounded wait expired)", code);
            return (ludvig_status)code;
        }
    }
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
template <class T>
__global__ void k_pad_features(const T* __restrict__ src, int64_t npx, int d, T* __restrict__ dst) {
    constexpr int kPer = 16 / (int)sizeof(T);
    constexpr int kGroups = kPadD / kPer;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npx * kGroups) return;
    const int64_t p = e / kGroups;
    const int c0 = (int)(e - p * kGroups) * kPer;
    T vals[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) vals[k] = c0 + k < d ? src[p * d + c0 + k] : T(0.f);
    uint4 v;
    memcpy(&v, vals, sizeof(v));
    reinterpret_cast<uint4*>(dst)[e] = v;
}

__global__ void k_add_columns(const float* __restrict__ wide, int64_t n, int d, float* __restrict__ num) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    const int64_t i = e / d;
    num[e] += wide[i * kPadD + (e - i * d)];
}

bool use_padded(int dtype, int d) { return d < kPadD && use_tensor_cores(dtype, kPadD); }

ludvig_status accumulate_padded(ludvig_scene* s, const ludvig_camera* cams, int32_t n_views, int32_t width,
                                int32_t height, const void* feats, int32_t dtype, int32_t d, float* num,
                                float* den, cudaStream_t st) {
    const int64_t n = s->n;
    const int64_t px_view = (int64_t)width * height;
    const size_t esize = dtype == LUDVIG_F32 ? 4 : 2;
    const int vc = std::min<int>(kMaxViews, n_views);
    float* wide;
    void* fpad;
    LV_TRY(s->ws.get("pad.num", (size_t)n * kPadD, &wide));
    LV_TRY(s->ws.get("pad.feats", (size_t)vc * px_view * kPadD * esize, &fpad));
    LV_CUDA(cudaMemsetAsync(wide, 0, sizeof(float) * (size_t)n * kPadD, st));
    for (int v0 = 0; v0 < n_views; v0 += vc) {
        const int nv = std::min(vc, n_views - v0);
        const int64_t npx = (int64_t)nv * px_view;
        const char* src = static_cast<const char*>(feats) + (size_t)v0 * px_view * d * esize;
        // 16-byte groups per padded pixel: 8 (float) or 4 (bfloat16)
        const int64_t groups = npx * (kPadD * (int64_t)esize / 16);
        if (dtype == LUDVIG_F32)
            k_pad_features<float><<<grid_for(groups, 256), 256, 0, st>>>(
                reinterpret_cast<const float*>(src), npx, d, static_cast<float*>(fpad));
        else
            k_pad_features<__nv_bfloat16><<<grid_for(groups, 256), 256, 0, st>>>(
                reinterpret_cast<const __nv_bfloat16*>(src), npx, d, static_cast<__nv_bfloat16*>(fpad));
        LV_LAUNCH();
        LV_TRY(accumulate(s, cams + v0, nv, width, height, fpad, dtype, kPadD, wide, den, st, nullptr));
    }
    k_add_columns<<<grid_for(n * d, 256), 256, 0, st>>>(wide, n, d, num);
    LV_LAUNCH();
    return LUDVIG_OK;
}

// FP8-E4M3 features (codes q, per-view scales s): x = decode(q) s_v rounded
// to bfloat16 for the tensor-core path (the E4M3 value is exact in half
// precision; the bfloat16 rounding adds at most 2^-9 relative to an FP8
// quantisation error of up to 2^-4).  Thread t converts elements 4t .. 4t+3
// of the group (one 4-byte load, one 8-byte store); the scalar tail covers a
// total that is not a multiple of 4.
__device__ __forceinline__ __nv_bfloat16 dequant_e4m3(uint32_t code, float s) {
    const __half h(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3));
    return __float2bfloat16_rn(__half2float(h) * s);
}

__global__ void k_dequant_e4m3(const uint8_t* __restrict__ q, const float* __restrict__ s, int64_t view_elems,
                               int64_t total, __nv_bfloat16* __restrict__ out) {
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e0 >= total) return;
    if (e0 + 4 <= total) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(q + e0);
        __nv_bfloat16 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = dequant_e4m3((w >> (8 * k)) & 0xffu, s[(e0 + k) / view_elems]);
        uint2 v;
        memcpy(&v, o, sizeof(v));
        *reinterpret_cast<uint2*>(out + e0) = v;
    } else {
        for (int64_t e = e0; e < total; ++e) out[e] = dequant_e4m3(q[e], s[e / view_elems]);
    }
}

}  // namespace

// ---------------------------------------------------------------- scene
ludvig_status scene_init(ludvig_scene* s, const float* means, const float* scales, const float* quats,
                         const float* opac, cudaStream_t st) {
    if (s->n == 0) return LUDVIG_OK;
    k_scene_init<<<grid_for(s->n, 256), 256, 0, st>>>(means, scales, quats, opac, s->n, s->geo, s->cov_a,
                                                      s->cov_b, s->means);
    LV_LAUNCH();
    return LUDVIG_OK;
}

}  // namespace ludvig

using namespace ludvig;

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
    if (use_padded(dtype, d))
        return accumulate_padded(scene, cams, n_views, width, height, feats, dtype, d, num, den,
                                 static_cast<cudaStream_t>(stream));
    return accumulate(scene, cams, n_views, width, height, feats, dtype, d, num, den,
                      static_cast<cudaStream_t>(stream), nullptr);
}

extern "C" ludvig_status ludvig_uplift_finalize(int64_t n, int32_t d, const float* num, const float* den,
                                                float* out, float* beta, void* stream) {
    LV_ARG(n >= 0 && d >= 1, "bad sizes");
    if (n == 0) return LUDVIG_OK;
    LV_ARG(num != nullptr && den != nullptr && out != nullptr, "NULL buffer");
    StageScope scope(LUDVIG_STAGE_NORMALISE, static_cast<cudaStream_t>(stream));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d >= 32) {
        const int vec4 = (d % 4 == 0) && (reinterpret_cast<uintptr_t>(num) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(out) % 16 == 0);
        k_normalise_rows<<<(unsigned)std::min<int64_t>(ceil_div(n, 8), 152 * 64), 256, 0, st>>>(num, den, out, beta,
                                                                                               n, d, vec4);
    } else {
        k_normalise<<<grid_for(n * d, 256), 256, 0, st>>>(num, den, out, beta, n, d);
    }
    LV_LAUNCH();
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_uplift(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                       int32_t width, int32_t height, const void* feats, int32_t dtype,
                                       int32_t d, float* out, float* beta, void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(out != nullptr || scene->n == 0, "out is NULL");
    LV_ARG(d >= 1 && d <= 65536, "d must be in [1, 65536]");
    LV_TRY(check_views(cams, n_views, width, height));
    const int64_t n = scene->n;
    if (n == 0) return LUDVIG_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* den = beta;
    if (!den) LV_TRY(scene->ws.get("uplift.den", (size_t)n, &den));
    LV_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n * d, st));
    LV_CUDA(cudaMemsetAsync(den, 0, sizeof(float) * (size_t)n, st));
    LV_TRY(ludvig_uplift_accumulate(scene, cams, n_views, width, height, feats, dtype, d, out, den, stream));
    return ludvig_uplift_finalize(n, d, out, den, out, nullptr, stream);
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* den = beta;
    if (!den) LV_TRY(scene->ws.get("uplift.den", (size_t)n, &den));
    LV_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n * d, st));
    LV_CUDA(cudaMemsetAsync(den, 0, sizeof(float) * (size_t)n, st));
    const int64_t view_elems = (int64_t)width * height * d;
    const int vc = std::min<int>(kMaxViews, std::max(1, n_views));
    __nv_bfloat16* fb;
    LV_TRY(scene->ws.get("fp8.bf16", (size_t)vc * view_elems, &fb));
    for (int v0 = 0; v0 < n_views; v0 += vc) {
        const int nv = std::min(vc, n_views - v0);
        const int64_t total = (int64_t)nv * view_elems;
        // groups start a multiple of 16 views in: the codes stay 4-byte aligned
        k_dequant_e4m3<<<grid_for(ceil_div(total, 4), 256), 256, 0, st>>>(q + (size_t)v0 * view_elems, scales + v0,
                                                                         view_elems, total, fb);
        LV_LAUNCH();
        if (use_padded(LUDVIG_BF16, d))
            LV_TRY(accumulate_padded(scene, cams + v0, nv, width, height, fb, LUDVIG_BF16, d, out, den, st));
        else
            LV_TRY(accumulate(scene, cams + v0, nv, width, height, fb, LUDVIG_BF16, d, out, den, st, nullptr));
    }
    return ludvig_uplift_finalize(n, d, out, den, out, nullptr, stream);
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
    const RenderJob rj{f, out};
    return accumulate(scene, cams, n_views, width, height, nullptr, LUDVIG_F32, d, nullptr, nullptr, st, nullptr,
                      &rj);
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
        if (use_padded(dtype, d))
            LV_TRY(accumulate_padded(scene, cams + v0, nv, width, height, fbuf[b], dtype, d, num, den, st));
        else
            LV_TRY(accumulate(scene, cams + v0, nv, width, height, fbuf[b], dtype, d, num, den, st, nullptr));
        LV_CUDA(cudaEventRecord(scene->ev_free[b], st));
    }
    LV_TRY(ludvig_uplift_finalize(n, d, num, den, num, nullptr, stream));
    LV_CUDA(cudaMemcpyAsync(out, num, sizeof(float) * (size_t)n * d, cudaMemcpyDeviceToHost, st));
    if (beta) LV_CUDA(cudaMemcpyAsync(beta, den, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    return LUDVIG_OK;
}

// ---------------------------------------------------------------- inspection
extern "C" ludvig_status ludvig_debug_project(ludvig_scene_t scene, const ludvig_camera* cam, int32_t width,
                                              int32_t height, float* rec, int32_t* rect, void* stream) {
    LV_ARG(scene != nullptr && rec != nullptr && rect != nullptr, "NULL argument");
    LV_TRY(check_views(cam, 1, width, height));
    if (scene->n == 0) return LUDVIG_OK;
    ChunkDebug dbg;
    dbg.rec = rec;
    dbg.rect = rect;
    dbg.stop_after_project = true;
    bool tm;
    return run_chunk(scene, cam, 1, width, height, nullptr, LUDVIG_F32, 1, nullptr, nullptr,
                     static_cast<cudaStream_t>(stream), &dbg, &tm);
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
    ChunkDebug dbg;
    dbg.ranges64 = ranges;
    dbg.list = list;
    dbg.list_cap = list ? cap : 0;
    dbg.list_total = total;
    dbg.stop_after_sort = true;
    dbg.unpruned = (pruned == 0);
    bool tm;
    LV_TRY(run_chunk(scene, cam, 1, width, height, nullptr, LUDVIG_F32, 1, nullptr, nullptr, st, &dbg, &tm));
    if (tm) {
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
    bool tm;
    return run_chunk(scene, cam, 1, width, height, fz, LUDVIG_F32, 1, num, den, st, &dbg, &tm);
}
