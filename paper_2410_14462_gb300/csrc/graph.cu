// Graph diffusion over the Gaussians (Sec. 3.3): exact kNN of the centres,
// the union edge set with similarity weights (Eq. 7 / the diffusion
// workload's spatial x cosine weight), and the power iteration of Eq. 8.
//
// kNN: points are bucketed in a uniform grid (cells sorted by the radix sort);
// one thread per query scans cells ring by ring (Chebyshev distance r around
// its own cell) and stops once the k-th best squared distance is below the
// squared gap r*cell to the unvisited rings.  Squared distances are float32
// (dx*dx + dy*dy) + dz*dz with d = x_j - x_i and ties go to the lower index,
// so the result is exact and independent of the scan order.
//
// Graph: own neighbours plus reverse edges per row, one warp sorts and
// de-duplicates each row, then weights are computed per edge from the two
// feature rows and optionally thresholded and row-normalised.
//
// Diffusion: one kernel per step computes y = A x * (1/||x||) row by row and
// accumulates ||y||^2 (float64) for the next step's scaling.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace ludvig {

namespace {

unsigned grid_for(int64_t work, int threads) { return (unsigned)ceil_div(work, threads); }

// ------------------------------------------------------------ bounding box
__global__ void k_bbox(const float* __restrict__ x, int64_t n, float* __restrict__ out6) {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], x[3 * i + a]);
            hi[a] = fmaxf(hi[a], x[3 * i + a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // order-preserving integer encoding of floats for atomicMin/Max
            const int l = __float_as_int(lo[a]), h = __float_as_int(hi[a]);
            atomicMin(reinterpret_cast<int*>(out6) + a, l >= 0 ? l : l ^ 0x7fffffff);
            atomicMax(reinterpret_cast<int*>(out6) + 3 + a, h >= 0 ? h : h ^ 0x7fffffff);
        }
    }
}

struct Grid {
    float lo[3];
    float cell;
    float inv_cell;
    int g[3];
};

__device__ __forceinline__ int cell_coord(float x, float lo, float inv, int g) {
    int c = (int)floorf((x - lo) * inv);
    return c < 0 ? 0 : (c >= g ? g - 1 : c);
}

__global__ void k_cell_keys(const float* __restrict__ x, int64_t n, int64_t npad, Grid gr,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) {
        keys[i] = 0xffffffffu;
        vals[i] = 0xffffffffu;
        return;
    }
    const int cx = cell_coord(x[3 * i], gr.lo[0], gr.inv_cell, gr.g[0]);
    const int cy = cell_coord(x[3 * i + 1], gr.lo[1], gr.inv_cell, gr.g[1]);
    const int cz = cell_coord(x[3 * i + 2], gr.lo[2], gr.inv_cell, gr.g[2]);
    keys[i] = (uint32_t)(((int64_t)cz * gr.g[1] + cy) * gr.g[0] + cx);
    vals[i] = (uint32_t)i;
}

__global__ void k_cell_ranges(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t k = keys[j];
    if (j == 0 || keys[j - 1] != k) ranges[k].x = (uint32_t)j;
    if (j == n - 1 || keys[j + 1] != k) ranges[k].y = (uint32_t)(j + 1);
}

__device__ __forceinline__ bool closer(float d, uint32_t i, float bd, uint32_t bi) {
    return d < bd || (d == bd && i < bi);
}

// Points sorted by cell are stored as float4 (x, y, z, index) in cell order.
__global__ void k_gather_sorted(const float* __restrict__ x, const uint32_t* __restrict__ order,
                                int64_t n, float4* __restrict__ pts) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t i = order[j];
    pts[j] = make_float4(x[3 * i], x[3 * i + 1], x[3 * i + 2], __uint_as_float(i));
}

template <int K>
__global__ void __launch_bounds__(128) k_knn(const float4* __restrict__ pts, int64_t n, Grid gr,
                                             const uint2* __restrict__ cells, int k,
                                             int32_t* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float4 q = pts[j];
    const uint32_t qi = __float_as_uint(q.w);
    float bd[K];
    uint32_t bi[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        bd[t] = FLT_MAX;
        bi[t] = 0xffffffffu;
    }
    int have = 0;
    const int cx = cell_coord(q.x, gr.lo[0], gr.inv_cell, gr.g[0]);
    const int cy = cell_coord(q.y, gr.lo[1], gr.inv_cell, gr.g[1]);
    const int cz = cell_coord(q.z, gr.lo[2], gr.inv_cell, gr.g[2]);
    const int rmax = max(gr.g[0], max(gr.g[1], gr.g[2]));
    for (int r = 0; r <= rmax; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= gr.g[2]) continue;
            for (int dy = -r; dy <= r; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= gr.g[1]) continue;
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                const int step = face ? 1 : 2 * r;
                for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                    const int x = cx + dx;
                    if (x < 0 || x >= gr.g[0]) continue;
                    const uint2 rg = cells[((int64_t)z * gr.g[1] + y) * gr.g[0] + x];
                    for (uint32_t p = rg.x; p < rg.y; ++p) {
                        const float4 c = pts[p];
                        const uint32_t ci = __float_as_uint(c.w);
                        if (ci == qi) continue;
                        const float ex = __fsub_rn(c.x, q.x), ey = __fsub_rn(c.y, q.y),
                                    ez = __fsub_rn(c.z, q.z);
                        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)),
                                                   __fmul_rn(ez, ez));
                        if (!closer(d2, ci, bd[K - 1], bi[K - 1])) continue;
                        float cd = d2;
                        uint32_t cidx = ci;
#pragma unroll
                        for (int t = 0; t < K; ++t) {
                            if (closer(cd, cidx, bd[t], bi[t])) {
                                const float td = bd[t];
                                const uint32_t ti = bi[t];
                                bd[t] = cd;
                                bi[t] = cidx;
                                cd = td;
                                cidx = ti;
                            }
                        }
                        ++have;
                    }
                }
            }
        }
        // every point outside the visited (2r+1)^3 block is at least r cells away
        if (have >= k) {
            const float gap = (float)r * gr.cell;
            // 0.1% margin: rounding can put a point next to a cell border in the neighbour cell
            const float bound = gap * gap * 0.999f;
            float kth = 0.f;
#pragma unroll
            for (int t = 0; t < K; ++t)
                if (t == k - 1) kth = bd[t];
            if (kth < bound) break;
        }
    }
#pragma unroll
    for (int t = 0; t < K; ++t)
        if (t < k) out[(int64_t)qi * k + t] = bi[t] == 0xffffffffu ? -1 : (int32_t)bi[t];
}

// ------------------------------------------------------------ graph build
__global__ void k_own_and_indegree(const int32_t* __restrict__ nbr, int64_t n, int k,
                                   uint32_t* __restrict__ own, uint32_t* __restrict__ indeg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = 0;
    for (int t = 0; t < k; ++t) {
        const int32_t j = nbr[i * k + t];
        if (j >= 0 && j != i) {
            ++c;
            atomicAdd(&indeg[j], 1u);
        }
    }
    own[i] = c;
}

__global__ void k_row_counts(const uint32_t* __restrict__ own, const uint32_t* __restrict__ indeg,
                             int64_t n, uint32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = own[i] + indeg[i];
}

__global__ void k_fill_rows(const int32_t* __restrict__ nbr, int64_t n, int k,
                            const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ own,
                            uint32_t* __restrict__ cursor, uint32_t* __restrict__ tcol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t o = ptr[i];
    for (int t = 0; t < k; ++t) {
        const int32_t j = nbr[i * k + t];
        if (j >= 0 && j != i) {
            tcol[o++] = (uint32_t)j;
            const uint32_t pos = atomicAdd(&cursor[j], 1u);
            tcol[ptr[j] + own[j] + pos] = (uint32_t)i;
        }
    }
}

// One warp per row: sort the row's column indices (insertion sort through
// shared memory for short rows, a serial heap sort in place for long ones),
// then count the distinct values.
constexpr int kRowSmem = 256;
__global__ void __launch_bounds__(256) k_sort_unique_rows(uint32_t* __restrict__ tcol,
                                                         const uint32_t* __restrict__ ptr,
                                                         const uint32_t* __restrict__ cnt, int64_t n,
                                                         uint32_t* __restrict__ ucnt) {
    __shared__ uint32_t buf[8][kRowSmem];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    uint32_t* row = tcol + ptr[i];
    const uint32_t c = cnt[i];
    uint32_t* b = buf[warp];
    if (c <= kRowSmem) {
        for (uint32_t t = lane; t < c; t += 32) b[t] = row[t];
        __syncwarp();
        // rank sort: each element's position = number of smaller elements
        // (+ equal elements before it), which is a stable sort of the row
        for (uint32_t t = lane; t < c; t += 32) {
            const uint32_t v = b[t];
            uint32_t pos = 0;
            for (uint32_t u = 0; u < c; ++u) {
                const uint32_t w = b[u];
                pos += (w < v) || (w == v && u < t);
            }
            row[pos] = v;
        }
        __syncwarp();
    } else if (lane == 0) {
        // heap sort in place
        auto sift = [&](uint32_t start, uint32_t end) {
            uint32_t root = start;
            while (2 * root + 1 < end) {
                uint32_t child = 2 * root + 1;
                if (child + 1 < end && row[child] < row[child + 1]) ++child;
                if (row[root] < row[child]) {
                    const uint32_t t = row[root];
                    row[root] = row[child];
                    row[child] = t;
                    root = child;
                } else {
                    break;
                }
            }
        };
        for (int64_t s = (int64_t)c / 2 - 1; s >= 0; --s) sift((uint32_t)s, c);
        for (uint32_t e = c - 1; e > 0; --e) {
            const uint32_t t = row[0];
            row[0] = row[e];
            row[e] = t;
            sift(0, e);
        }
    }
    __syncwarp();
    uint32_t u = 0;
    for (uint32_t t = lane; t < c; t += 32) u += (t == 0 || row[t] != row[t - 1]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) ucnt[i] = u;
}

__global__ void k_norms(const float* __restrict__ f, int64_t n, int df, float* __restrict__ nrm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= n) return;
    float s = 0.f;
    for (int c = lane; c < df; c += 32) {
        const float v = f[i * df + c];
        s = fmaf(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[i] = sqrtf(s);
}

// Edge value modes: the diffusion workload's spatial x cosine weight, or the
// squared distance ||f^_i - f^_j||^2 of the l2-normalised features (for the
// RBF similarity of the appendix; a zero feature vector normalises to zero):
// 2 - 2 cos for two non-zero rows, 1 with one zero row, 0 with two.
constexpr int kEdgeSpatialCos = 0, kEdgeFeatureDist2 = 1;

__device__ __forceinline__ float feature_dist2(float ni, float nj, float cs) {
    const float zi = ni > 0.f ? 1.f : 0.f, zj = nj > 0.f ? 1.f : 0.f;
    return fmaxf(0.f, zi + zj - 2.f * cs);
}

// One warp per row: compact the distinct columns, weight every edge, then
// threshold / normalise the row (any df).  Row r of the launch is Gaussian
// order[r] (grid-cell order, so that neighbours' feature rows stay in L2), or
// r when order is null.
__global__ void __launch_bounds__(256) k_edge_weights_any(const uint32_t* __restrict__ tcol,
                                                const uint32_t* __restrict__ tptr,
                                                const uint32_t* __restrict__ tcnt,
                                                const int64_t* __restrict__ row_ptr,
                                                const float* __restrict__ x, const float* __restrict__ f,
                                                const float* __restrict__ nrm, int64_t n, int df,
                                                float inv_h, float binarize, int row_normalize,
                                                const uint32_t* __restrict__ order, int mode,
                                                int32_t* __restrict__ col, float* __restrict__ val) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + warp;
    if (r >= n) return;
    const int64_t i = order ? (int64_t)order[r] : r;
    const uint32_t* row = tcol + tptr[i];
    const uint32_t c = tcnt[i];
    const int64_t o0 = row_ptr[i];
    const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const float ni = nrm[i];
    const float* fi = f + i * df;
    int64_t o = o0;
    float rsum = 0.f;
    for (uint32_t t = 0; t < c; ++t) {
        const uint32_t j = row[t];
        if (t > 0 && row[t - 1] == j) continue;   // duplicate (mutual neighbours)
        float dot = 0.f;
        const float* fj = f + (int64_t)j * df;
        for (int ch = lane; ch < df; ch += 32) dot = fmaf(fi[ch], fj[ch], dot);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, s);
        if (lane == 0) {
            const float ex = x[3 * j] - xi, ey = x[3 * j + 1] - yi, ez = x[3 * j + 2] - zi;
            const float d2 = ex * ex + ey * ey + ez * ez;
            const float den = ni * nrm[j];
            const float cs = den > 0.f ? dot / den : 0.f;
            float w = mode == kEdgeFeatureDist2 ? feature_dist2(ni, nrm[j], cs) : expf(-d2 * inv_h) * fmaxf(0.f, cs);
            if (binarize > 0.f) w = w > binarize ? 1.f : 0.f;
            col[o] = (int32_t)j;
            val[o] = w;
            rsum += w;
        }
        ++o;
    }
    if (row_normalize && lane == 0 && rsum > 0.f)   // divide: a denormal sum has an infinite reciprocal
        for (int64_t e = o0; e < o; ++e) val[e] = val[e] / rsum;
}

// Same for df <= 32 kR: one warp per row with f_i in registers; the row's
// distinct columns are found 32 at a time (a sorted row repeats a column for
// mutual neighbours) and dotted two at a time; the row sum normalises in
// parallel.
template <int kR>
__global__ void __launch_bounds__(256) k_edge_weights(const uint32_t* __restrict__ tcol,
                                                     const uint32_t* __restrict__ tptr,
                                                     const uint32_t* __restrict__ tcnt,
                                                     const int64_t* __restrict__ row_ptr,
                                                     const float* __restrict__ x, const float* __restrict__ f,
                                                     const float* __restrict__ nrm, int64_t n, int df,
                                                     float inv_h, float binarize, int row_normalize,
                                                     const uint32_t* __restrict__ order, int mode,
                                                     int32_t* __restrict__ col, float* __restrict__ val) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + warp;
    if (r >= n) return;   // whole warp
    const int64_t i = order ? (int64_t)order[r] : r;
    const uint32_t* row = tcol + tptr[i];
    const uint32_t c = tcnt[i];
    const int64_t o0 = row_ptr[i];
    const float xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const float ni = nrm[i];
    float fr[kR];
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        const int ch = lane + 32 * k;
        fr[k] = ch < df ? f[i * df + ch] : 0.f;
    }
    auto weight = [&](uint32_t j, float dot) {
        const float ex = x[3 * j] - xi, ey = x[3 * j + 1] - yi, ez = x[3 * j + 2] - zi;
        const float d2 = ex * ex + ey * ey + ez * ez;
        const float den = ni * nrm[j];
        const float cs = den > 0.f ? dot / den : 0.f;
        float w = mode == kEdgeFeatureDist2 ? feature_dist2(ni, nrm[j], cs) : expf(-d2 * inv_h) * fmaxf(0.f, cs);
        if (binarize > 0.f) w = w > binarize ? 1.f : 0.f;
        return w;
    };
    int64_t o = o0;
    float rsum = 0.f;   // lane 0
    for (uint32_t t0 = 0; t0 < c; t0 += 32) {
        const uint32_t t = t0 + lane;
        const uint32_t j = t < c ? row[t] : 0u;
        const bool keep = t < c && !(t > 0 && row[t - 1] == j);
        uint32_t m = __ballot_sync(0xffffffffu, keep);
        while (m) {
            const int l0 = __ffs(m) - 1;
            m &= m - 1u;
            const bool two = m != 0u;
            const int l1 = two ? __ffs(m) - 1 : l0;
            if (two) m &= m - 1u;
            const uint32_t j0 = __shfl_sync(0xffffffffu, j, l0), j1 = __shfl_sync(0xffffffffu, j, l1);
            const float* f0 = f + (int64_t)j0 * df;
            const float* f1 = f + (int64_t)j1 * df;
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                const int ch = lane + 32 * k;
                if (ch < df) {
                    d0 = fmaf(fr[k], f0[ch], d0);
                    d1 = fmaf(fr[k], f1[ch], d1);
                }
            }
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) {
                d0 += __shfl_xor_sync(0xffffffffu, d0, sft);
                d1 += __shfl_xor_sync(0xffffffffu, d1, sft);
            }
            if (lane == 0) {
                const float w0 = weight(j0, d0);
                col[o] = (int32_t)j0;
                val[o] = w0;
                rsum += w0;
                if (two) {
                    const float w1 = weight(j1, d1);
                    col[o + 1] = (int32_t)j1;
                    val[o + 1] = w1;
                    rsum += w1;
                }
            }
            o += two ? 2 : 1;
        }
    }
    if (row_normalize) {
        rsum = __shfl_sync(0xffffffffu, rsum, 0);
        __syncwarp();
        if (rsum > 0.f)   // divide: a denormal sum has an infinite reciprocal
            for (int64_t e = o0 + lane; e < o; e += 32) val[e] = val[e] / rsum;
    }
}

// exclusive scan into int64 row pointers (u32 scan + widening is enough while nnz < 2^32)
__global__ void k_widen_ptr(const uint32_t* __restrict__ p, int64_t n, const uint64_t* __restrict__ total,
                            int64_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = p[i];
    if (i == n) out[n] = (int64_t)*total;
}

// ------------------------------------------------------------ diffusion
__global__ void k_colnorm2(const float* __restrict__ x, int64_t n, int dx, double* __restrict__ acc) {
    __shared__ double part[32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < dx; ++c) {
        double v = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double t = x[i * dx + c];
            v += t * t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < dx) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += part[w][threadIdx.x];
        atomicAdd(acc + threadIdx.x, v);
    }
}

// y = A (x / ||x||) for one column (dx == 1, the CSR form): groups of kLanes
// lanes per row over a grid-stride range of rows.  ||y||^2 is reduced in the
// block and added once per block (float64).
template <int kLanes>
__global__ void __launch_bounds__(256) k_spmv_scaled(const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col,
                                                    const float* __restrict__ val,
                                                    const float* __restrict__ x, int64_t n, int dx,
                                                    const double* __restrict__ n2_in,
                                                    float* __restrict__ y, double* __restrict__ n2_out) {
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane % kLanes;
    const double nn = n2_in[0];
    const float s = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    double mine = 0.0;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kLanes);
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kLanes;
    for (int64_t base = 0; base < n; base += groups) {
        const int64_t i = base + g0;
        float acc = 0.f;
        if (i < n)
            for (int64_t e = rp[i] + sub; e < rp[i + 1]; e += kLanes) acc = fmaf(val[e], x[col[e]], acc);
#pragma unroll
        for (int o = kLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && sub == 0) {
            acc *= s;
            y[i] = acc;
            mine += (double)acc * acc;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) part[warp][0] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += part[w][0];
        atomicAdd(n2_out, t);
    }
}

// Several columns (2 <= dx <= 32): L = ceil(dx / 4) lanes per row, each
// owning 4 consecutive columns, so a warp works on 32 / L rows at once (a row
// is a chain of dependent loads: its pointer, then per entry the column and
// the x values).  Each (row, column) sum is one fmaf chain over the row's
// entries in order, then the column's scale; the columns' squared norms are
// summed per block in shared memory, then added to n2_out.
__global__ void __launch_bounds__(256) k_spmv_cols(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                   const float* __restrict__ val, const float* __restrict__ x,
                                                   int64_t n, int dx, const double* __restrict__ n2_in,
                                                   float* __restrict__ y, double* __restrict__ n2_out) {
    __shared__ double colsum[32];
    const int L = (dx + 3) >> 2, G = 32 / L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / L, c0 = 4 * (lane - grp * L);
    const bool act = grp < G;
    if (threadIdx.x < 32) colsum[threadIdx.x] = 0.0;
    __syncthreads();
    float sc[4];
    double mine[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double nn = (act && c0 + q < dx) ? n2_in[c0 + q] : 0.0;
        sc[q] = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    }
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * G; base < n; base += nw * G) {
        const int64_t i = base + grp;
        if (!act || i >= n) continue;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t e = rp[i], e1 = rp[i + 1]; e < e1; ++e) {
            const float v = val[e];
            const float* xr = x + (int64_t)col[e] * dx + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + q < dx) acc[q] = fmaf(v, xr[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + q < dx) {
                const float a = acc[q] * sc[q];
                y[i * dx + c0 + q] = a;
                mine[q] += (double)a * a;
            }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (act && c0 + q < dx) atomicAdd(&colsum[c0 + q], mine[q]);
    __syncthreads();
    if (threadIdx.x < dx) atomicAdd(n2_out + threadIdx.x, colsum[threadIdx.x]);
}

// Sliced copy of the matrix for single-column diffusion: slices of 32
// consecutive rows, each padded to its longest row and stored column-major
// (slot j of row r at off[slice] + 32 j + r % 32; padding: column = the row,
// value 0).  One thread per row then reads its columns and values with
// coalesced 128-byte warp loads and no row-pointer dependence.
// With perm (the kNN grid's cell order) the sliced copy is renumbered: its
// row r is node perm[r] and its columns are positions (inv), so that the rows
// of a slice and the x entries they gather are spatial neighbours; the
// diffusion then runs on the permuted vector.
__global__ void k_sell_width(const int64_t* __restrict__ rp, int64_t n, int64_t nslices,
                             const int32_t* __restrict__ perm, uint32_t* __restrict__ slots) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s > nslices) return;
    if (s == nslices) {   // the scan's total
        if (lane == 0) slots[s] = 0u;
        return;
    }
    const int64_t r = s * 32 + lane;
    const int64_t i = r < n ? (perm ? (int64_t)perm[r] : r) : 0;
    uint32_t len = r < n ? (uint32_t)(rp[i + 1] - rp[i]) : 0u;
    len = __reduce_max_sync(0xffffffffu, len);
    if (lane == 0) slots[s] = 32u * len;
}

__global__ void k_sell_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const float* __restrict__ val, int64_t n, int64_t nslices,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                            const uint32_t* __restrict__ off, int32_t* __restrict__ scol, float* __restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (s >= nslices) return;
    const int64_t r = s * 32 + lane;
    const int64_t i = r < n ? (perm ? (int64_t)perm[r] : r) : 0;
    const int64_t e0 = r < n ? rp[i] : 0;
    const uint32_t len = r < n ? (uint32_t)(rp[i + 1] - e0) : 0u;
    const uint32_t w = (off[s + 1] - off[s]) / 32u;
    for (uint32_t j = 0; j < w; ++j) {
        const uint32_t p = off[s] + 32u * j + (uint32_t)lane;
        const bool real = j < len;
        const int32_t c = real ? col[e0 + j] : 0;
        scol[p] = real ? (inv ? inv[c] : c) : (int32_t)(r < n ? r : 0);
        sval[p] = real ? val[e0 + j] : 0.f;
    }
}

__global__ void k_invert_perm(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) inv[perm[r]] = (int32_t)r;
}

__global__ void k_gather_perm(const float* __restrict__ x, const int32_t* __restrict__ perm, int64_t n,
                              float* __restrict__ y) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) y[r] = x[perm[r]];
}

__global__ void k_scatter_perm(const float* __restrict__ y, const int32_t* __restrict__ perm, int64_t n,
                               float* __restrict__ x) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) x[perm[r]] = y[r];
}

// y = A (x / ||x||) for one column on the sliced copy: a warp per slice, a
// thread per row; ||y||^2 reduced per block, added once per block (float64).
__global__ void __launch_bounds__(256) k_spmv_sell(const uint32_t* __restrict__ off, const int32_t* __restrict__ scol,
                                                  const float* __restrict__ sval, const float* __restrict__ x,
                                                  int64_t n, int64_t nslices, const double* __restrict__ n2_in,
                                                  float* __restrict__ y, double* __restrict__ n2_out) {
    __shared__ double part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double nn = n2_in[0];
    const float sc = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    double mine = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * 8 + warp; s < nslices; s += (int64_t)gridDim.x * 8) {
        const uint32_t o1 = off[s + 1];
        float acc = 0.f;
#pragma unroll 4
        for (uint32_t p = off[s] + (uint32_t)lane; p < o1; p += 32u) acc = fmaf(sval[p], x[scol[p]], acc);
        const int64_t r = s * 32 + lane;
        if (r < n) {
            acc *= sc;
            y[r] = acc;
            mine += (double)acc * acc;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) part[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += part[w];
        atomicAdd(n2_out, t);
    }
}

// *order (if given) receives the points' indices sorted by grid cell (valid
// until the scene's workspace is reused), or null.
ludvig_status knn_impl(ludvig_scene* s, int k, int32_t* nbr, cudaStream_t st, const uint32_t** order = nullptr) {
    Arena& ws = s->ws;
    if (order) *order = nullptr;
    const int64_t n = s->n;
    float* bb;
    LV_TRY(ws.get("knn.bbox", 8, &bb));
    {
        const int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000,
                             (int)0x80000000};
        void* h;
        LV_TRY(ws.pinned("knn.bbox_h", 64, &h));
        std::memcpy(h, init, sizeof(init));
        LV_CUDA(cudaMemcpyAsync(bb, h, sizeof(init), cudaMemcpyHostToDevice, st));
        k_bbox<<<(unsigned)std::min<int64_t>(1024, ceil_div(n, 256)), 256, 0, st>>>(s->means, n, bb);
        LV_LAUNCH();
        LV_CUDA(cudaMemcpyAsync(static_cast<char*>(h) + 32, bb, 24, cudaMemcpyDeviceToHost, st));
        LV_CUDA(cudaStreamSynchronize(st));
        int enc[6];
        std::memcpy(enc, static_cast<char*>(h) + 32, 24);
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            int l = enc[a] >= 0 ? enc[a] : enc[a] ^ 0x7fffffff;
            int hh = enc[3 + a] >= 0 ? enc[3 + a] : enc[3 + a] ^ 0x7fffffff;
            std::memcpy(&lo[a], &l, 4);
            std::memcpy(&hi[a], &hh, 4);
        }
        Grid gr;
        double ext[3], vol = 1.0;
        for (int a = 0; a < 3; ++a) {
            ext[a] = std::max(1e-6, (double)hi[a] - (double)lo[a]);
            vol *= ext[a];
        }
        // about two points per cell on average, at most 2^24 cells
        double cell = std::cbrt(vol * 2.0 / (double)std::max<int64_t>(n, 1));
        for (;;) {
            int64_t tot = 1;
            for (int a = 0; a < 3; ++a) tot *= (int64_t)(ext[a] / cell) + 1;
            if (tot <= ((int64_t)1 << 24)) break;
            cell *= 1.25;
        }
        for (int a = 0; a < 3; ++a) {
            gr.lo[a] = lo[a];
            gr.g[a] = (int)(ext[a] / cell) + 1;
        }
        gr.cell = (float)cell;
        gr.inv_cell = (float)(1.0 / cell);
        const int64_t ncell = (int64_t)gr.g[0] * gr.g[1] * gr.g[2];
        const int64_t npad = round_up(n, kRadixTile);
        uint32_t *keys, *vals, *keys2, *vals2;
        LV_TRY(ws.get("knn.keys", (size_t)npad, &keys));
        LV_TRY(ws.get("knn.vals", (size_t)npad, &vals));
        LV_TRY(ws.get("knn.keys2", (size_t)npad, &keys2));
        LV_TRY(ws.get("knn.vals2", (size_t)npad, &vals2));
        k_cell_keys<<<grid_for(npad, 256), 256, 0, st>>>(s->means, n, npad, gr, keys, vals);
        LV_LAUNCH();
        int nbits = 1;
        while (((int64_t)1 << nbits) <= ncell) ++nbits;
        uint32_t *sk = keys, *sv = vals;
        LV_TRY(radix_sort_pairs(&sk, &sv, keys2, vals2, 1, npad, nbits, ws, st));
        uint2* cells;
        LV_TRY(ws.get("knn.cells", (size_t)ncell, &cells));
        LV_CUDA(cudaMemsetAsync(cells, 0, sizeof(uint2) * (size_t)ncell, st));
        k_cell_ranges<<<grid_for(n, 256), 256, 0, st>>>(sk, n, cells);
        LV_LAUNCH();
        float4* pts;
        LV_TRY(ws.get("knn.pts", (size_t)n, &pts));
        k_gather_sorted<<<grid_for(n, 256), 256, 0, st>>>(s->means, sv, n, pts);
        LV_LAUNCH();
        if (order) *order = sv;
        const unsigned g = grid_for(n, 128);
        if (k <= 8) k_knn<8><<<g, 128, 0, st>>>(pts, n, gr, cells, k, nbr);
        else if (k <= 16) k_knn<16><<<g, 128, 0, st>>>(pts, n, gr, cells, k, nbr);
        else if (k <= 32) k_knn<32><<<g, 128, 0, st>>>(pts, n, gr, cells, k, nbr);
        else k_knn<64><<<g, 128, 0, st>>>(pts, n, gr, cells, k, nbr);
        LV_LAUNCH();
    }
    return LUDVIG_OK;
}

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_knn(ludvig_scene_t scene, int32_t k, int32_t* nbr, void* stream) {
    LV_ARG(scene != nullptr && nbr != nullptr, "NULL argument");
    LV_ARG(k >= 1 && k <= 64, "k must be in [1, 64]");
    if (scene->n == 0) return LUDVIG_OK;
    StageScope scope(LUDVIG_STAGE_KNN, static_cast<cudaStream_t>(stream));
    return knn_impl(scene, k, nbr, static_cast<cudaStream_t>(stream));
}

namespace ludvig {
namespace {

// The union kNN graph with per-edge values of `mode` (see kEdgeSpatialCos).
ludvig_status graph_build_impl(ludvig_scene_t scene, int32_t k, const float* feats, int32_t df, float spatial_h,
                               float binarize, int32_t row_normalize, int mode, cudaStream_t st,
                               ludvig_graph_t* out) {
    ludvig_graph* g = new ludvig_graph();
    g->n = scene->n;
    LV_CUDA(cudaGetDevice(&g->device));
    const int64_t n = scene->n;
    Arena& ws = scene->ws;
    auto fail = [&](ludvig_status s) {
        ludvig_graph_destroy(g);
        return s;
    };
    ludvig_status r;
    if (cudaMalloc(&g->row_ptr, sizeof(int64_t) * (size_t)(n + 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("graph allocation failed");
        return fail(LUDVIG_ERR_OOM);
    }
    if (n == 0) {
        if (cudaMemsetAsync(g->row_ptr, 0, sizeof(int64_t), st) != cudaSuccess) return fail(LUDVIG_ERR_CUDA);
        *out = g;
        return LUDVIG_OK;
    }
    int32_t* nbr;
    uint32_t *own, *indeg, *cnt, *tptr, *cursor, *ucnt, *uptr;
    uint64_t *tot_d, *utot_d;
    float* nrm;
#define GB_TRY(expr)                   \
    do {                               \
        r = (expr);                    \
        if (r != LUDVIG_OK) return fail(r); \
    } while (0)
    GB_TRY(ws.get("g.nbr", (size_t)n * k, &nbr));
    GB_TRY(ws.get("g.own", (size_t)n, &own));
    GB_TRY(ws.get("g.indeg", (size_t)n, &indeg));
    GB_TRY(ws.get("g.cnt", (size_t)n, &cnt));
    GB_TRY(ws.get("g.tptr", (size_t)n, &tptr));
    GB_TRY(ws.get("g.cursor", (size_t)n, &cursor));
    GB_TRY(ws.get("g.ucnt", (size_t)n, &ucnt));
    GB_TRY(ws.get("g.uptr", (size_t)n, &uptr));
    GB_TRY(ws.get("g.tot", 2, &tot_d));
    utot_d = tot_d + 1;
    GB_TRY(ws.get("g.nrm", (size_t)n, &nrm));
    const uint32_t* sorder = nullptr;   // rows in grid-cell order: neighbours' feature rows stay in L2
    {
        StageScope scope(LUDVIG_STAGE_KNN, st);
        GB_TRY(knn_impl(scene, k, nbr, st, &sorder));
    }
    if (sorder) {   // the graph keeps the cell order for its diffusion (sliced copy renumbered)
        if (cudaMalloc(&g->perm, sizeof(int32_t) * (size_t)n) != cudaSuccess ||
            cudaMalloc(&g->inv, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            set_error("graph allocation failed");
            return fail(LUDVIG_ERR_OOM);
        }
        if (cudaMemcpyAsync(g->perm, sorder, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return fail(LUDVIG_ERR_CUDA);
        k_invert_perm<<<grid_for(n, 256), 256, 0, st>>>(g->perm, n, g->inv);
        count_launch();
    }
    StageScope gscope(LUDVIG_STAGE_GRAPH, st);
    if (cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * n, st) != cudaSuccess ||
        cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * n, st) != cudaSuccess)
        return fail(LUDVIG_ERR_CUDA);
    k_own_and_indegree<<<grid_for(n, 256), 256, 0, st>>>(nbr, n, k, own, indeg);
    count_launch();
    k_row_counts<<<grid_for(n, 256), 256, 0, st>>>(own, indeg, n, cnt);
    count_launch();
    GB_TRY(scan_exclusive_u32(cnt, tptr, n, tot_d, ws, st));
    void* hbuf;
    GB_TRY(ws.pinned("g.tot_h", 16, &hbuf));
    uint64_t* tot_h = static_cast<uint64_t*>(hbuf);
    if (cudaMemcpyAsync(tot_h, tot_d, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(LUDVIG_ERR_CUDA);
    const int64_t tnnz = (int64_t)tot_h[0];
    if (tnnz >= ((int64_t)1 << 32)) {
        set_error("graph too large");
        return fail(LUDVIG_ERR_UNSUPPORTED);
    }
    uint32_t* tcol;
    GB_TRY(ws.get("g.tcol", (size_t)std::max<int64_t>(tnnz, 1), &tcol));
    k_fill_rows<<<grid_for(n, 256), 256, 0, st>>>(nbr, n, k, tptr, own, cursor, tcol);
    count_launch();
    k_sort_unique_rows<<<grid_for(n, 8), 256, 0, st>>>(tcol, tptr, cnt, n, ucnt);
    count_launch();
    GB_TRY(scan_exclusive_u32(ucnt, uptr, n, utot_d, ws, st));
    k_widen_ptr<<<grid_for(n + 1, 256), 256, 0, st>>>(uptr, n, utot_d, g->row_ptr);
    count_launch();
    k_norms<<<grid_for(n, 8), 256, 0, st>>>(feats, n, df, nrm);
    count_launch();
    if (cudaMemcpyAsync(tot_h + 1, utot_d, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(LUDVIG_ERR_CUDA);
    g->nnz = (int64_t)tot_h[1];
    if (cudaMalloc(&g->col, sizeof(int32_t) * (size_t)std::max<int64_t>(g->nnz, 1)) != cudaSuccess ||
        cudaMalloc(&g->val, sizeof(float) * (size_t)std::max<int64_t>(g->nnz, 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("graph allocation failed");
        return fail(LUDVIG_ERR_OOM);
    }
    {
        const unsigned gb = grid_for(n, 8);
        const float ih = 1.0f / spatial_h;
#define LV_EW(R) k_edge_weights<R><<<gb, 256, 0, st>>>(tcol, tptr, cnt, g->row_ptr, scene->means, feats, nrm, n, \
                                                        df, ih, binarize, row_normalize, sorder, mode, g->col, g->val)
        if (df <= 32) LV_EW(1);
        else if (df <= 128) LV_EW(4);
        else if (df <= 256) LV_EW(8);
        else if (df <= 384) LV_EW(12);
        else if (df <= 512) LV_EW(16);
        else
            k_edge_weights_any<<<gb, 256, 0, st>>>(tcol, tptr, cnt, g->row_ptr, scene->means, feats, nrm, n, df, ih,
                                                   binarize, row_normalize, sorder, mode, g->col, g->val);
#undef LV_EW
    }
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
        set_error("graph kernels failed to launch");
        return fail(LUDVIG_ERR_CUDA);
    }
#undef GB_TRY
    *out = g;
    return LUDVIG_OK;
}

}  // namespace
}  // namespace ludvig

extern "C" ludvig_status ludvig_graph_build(ludvig_scene_t scene, int32_t k, const float* feats, int32_t df,
                                            float spatial_h, float binarize, int32_t row_normalize,
                                            void* stream, ludvig_graph_t* out) {
    LV_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(k >= 1 && k <= 64, "k must be in [1, 64]");
    LV_ARG(df >= 1 && feats != nullptr, "features required (df >= 1)");
    LV_ARG(spatial_h > 0.f, "spatial_h must be positive");
    return graph_build_impl(scene, k, feats, df, spatial_h, binarize, row_normalize, kEdgeSpatialCos,
                            static_cast<cudaStream_t>(stream), out);
}

extern "C" ludvig_status ludvig_graph_destroy(ludvig_graph_t g) {
    if (!g) return LUDVIG_OK;
    cudaDeviceSynchronize();
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->val);
    cudaFree(g->d2);
    cudaFree(g->perm);
    cudaFree(g->inv);
    g->ws.release();
    delete g;
    return LUDVIG_OK;
}

extern "C" int64_t ludvig_graph_nnz(ludvig_graph_t g) { return g ? g->nnz : -1; }

extern "C" int64_t ludvig_graph_workspace_bytes(ludvig_graph_t g) { return g ? (int64_t)g->ws.device_bytes() : -1; }

extern "C" ludvig_status ludvig_graph_export(ludvig_graph_t g, int64_t* row_ptr, int32_t* col, float* val,
                                             void* stream) {
    LV_ARG(g != nullptr, "graph is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (row_ptr) LV_CUDA(cudaMemcpyAsync(row_ptr, g->row_ptr, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToDevice, st));
    if (g->nnz > 0) {
        if (col) LV_CUDA(cudaMemcpyAsync(col, g->col, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToDevice, st));
        if (val) LV_CUDA(cudaMemcpyAsync(val, g->val, sizeof(float) * g->nnz, cudaMemcpyDeviceToDevice, st));
    }
    return LUDVIG_OK;
}

namespace ludvig {
namespace {

// The sliced copy of g's current values (built on first use and again after
// the values change; synchronises once to size it).  *ok = false when its
// slot count does not fit 32 bits (the CSR kernel is used then).
ludvig_status ensure_sell(ludvig_graph* g, cudaStream_t st, bool* ok, uint32_t** off, int32_t** scol,
                          float** sval) {
    *ok = false;
    const int64_t n = g->n, nslices = ceil_div(n, 32);
    uint32_t* slots;
    uint64_t* total_d;
    void* hb;
    LV_TRY(g->ws.get("sell.slots", (size_t)nslices + 1, &slots));
    LV_TRY(g->ws.get("sell.off", (size_t)nslices + 1, off));
    LV_TRY(g->ws.get("sell.total", 1, &total_d));
    LV_TRY(g->ws.pinned("sell.total_h", 16, &hb));
    uint64_t* total_h = static_cast<uint64_t*>(hb);
    if (g->sell_version == g->val_version) {
        LV_TRY(g->ws.get("sell.col", (size_t)std::max<uint64_t>(*total_h, 1), scol));
        LV_TRY(g->ws.get("sell.val", (size_t)std::max<uint64_t>(*total_h, 1), sval));
        *ok = true;
        return LUDVIG_OK;
    }
    k_sell_width<<<grid_for(nslices + 1, 8), 256, 0, st>>>(g->row_ptr, n, nslices, g->perm, slots);
    LV_LAUNCH();
    LV_TRY(scan_exclusive_u32(slots, *off, nslices + 1, total_d, g->ws, st));
    LV_CUDA(cudaMemcpyAsync(total_h, total_d, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    LV_CUDA(cudaStreamSynchronize(st));
    if (*total_h >= ((uint64_t)1 << 32)) return LUDVIG_OK;
    LV_TRY(g->ws.get("sell.col", (size_t)std::max<uint64_t>(*total_h, 1), scol));
    LV_TRY(g->ws.get("sell.val", (size_t)std::max<uint64_t>(*total_h, 1), sval));
    k_sell_fill<<<grid_for(nslices, 8), 256, 0, st>>>(g->row_ptr, g->col, g->val, n, nslices, g->perm, g->inv,
                                                      *off, *scol, *sval);
    LV_LAUNCH();
    g->sell_version = g->val_version;
    g->sell_slices = nslices;
    *ok = true;
    return LUDVIG_OK;
}

}  // namespace
}  // namespace ludvig

extern "C" ludvig_status ludvig_diffuse(ludvig_graph_t g, const float* x0, int32_t dx, int32_t iters,
                                        float* out, void* stream) {
    LV_ARG(g != nullptr, "graph is NULL");
    LV_ARG(dx >= 1 && dx <= 32, "dx must be in [1, 32]");
    LV_ARG(iters >= 0, "iters must be >= 0");
    LV_ARG(x0 != nullptr && out != nullptr, "NULL buffer");
    LV_ARG(x0 != out, "out must not alias x0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = g->n;
    if (n == 0) return LUDVIG_OK;
    const size_t bytes = sizeof(float) * (size_t)n * dx;
    if (iters == 0) {
        LV_CUDA(cudaMemcpyAsync(out, x0, bytes, cudaMemcpyDeviceToDevice, st));
        return LUDVIG_OK;
    }
    float* tmp;
    double* n2;
    LV_TRY(g->ws.get("d.tmp", (size_t)n * dx, &tmp));
    // n2[t*32 + c] = ||column c of g_t||^2, every step's slot zeroed up front
    LV_TRY(g->ws.get("d.n2", (size_t)(iters + 1) * 32, &n2));
    // ping-pong so that the last step writes `out`
    float* bufs[2] = {(iters % 2 == 1) ? out : tmp, (iters % 2 == 1) ? tmp : out};
    StageScope scope(LUDVIG_STAGE_DIFFUSE, st);
    LV_CUDA(cudaMemsetAsync(n2, 0, sizeof(double) * 32 * (size_t)(iters + 1), st));
    k_colnorm2<<<(unsigned)std::min<int64_t>(592, ceil_div(n, 256)), 256, 0, st>>>(x0, n, dx, n2);
    LV_LAUNCH();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(n, 32)));
    bool sell = false;
    uint32_t* soff = nullptr;
    int32_t* scol = nullptr;
    float* sval = nullptr;
    if (dx == 1) LV_TRY(ensure_sell(g, st, &sell, &soff, &scol, &sval));
    // the renumbered sliced copy works on the permuted vector: x0 gathered in,
    // the last step's vector scattered back to out
    const bool permuted = sell && g->perm;
    float *pa = nullptr, *pb = nullptr;
    if (permuted) {
        LV_TRY(g->ws.get("d.pa", (size_t)n, &pa));
        LV_TRY(g->ws.get("d.pb", (size_t)n, &pb));
        k_gather_perm<<<grid_for(n, 256), 256, 0, st>>>(x0, g->perm, n, pa);
        LV_LAUNCH();
    }
    const float* xin = permuted ? pa : x0;
    for (int t = 0; t < iters; ++t) {
        float* y = permuted ? ((t & 1) ? pa : pb) : bufs[t & 1];
        if (sell)
            k_spmv_sell<<<blocks, 256, 0, st>>>(soff, scol, sval, xin, n, g->sell_slices, n2 + 32 * t, y,
                                                n2 + 32 * (t + 1));
        else if (dx == 1)
            k_spmv_scaled<8><<<blocks, 256, 0, st>>>(g->row_ptr, g->col, g->val, xin, n, 1, n2 + 32 * t, y,
                                                     n2 + 32 * (t + 1));
        else
            k_spmv_cols<<<blocks, 256, 0, st>>>(g->row_ptr, g->col, g->val, xin, n, dx, n2 + 32 * t, y,
                                                n2 + 32 * (t + 1));
        LV_LAUNCH();
        xin = y;
    }
    if (permuted) {
        k_scatter_perm<<<grid_for(n, 256), 256, 0, st>>>(xin, g->perm, n, out);
        LV_LAUNCH();
    }
    return LUDVIG_OK;
}

// ---------------------------------------------------------------- diffusion without allocation
// Scratch of ludvig_diffuse_noalloc in statically allocated device memory:
// the ping-pong vector (at most kNoAllocMaxElems = n * dx floats, 4 MiB) and
// the per-step column norms (at most kNoAllocMaxIters steps, 32 columns,
// float64).  Every GPU that loads the library holds these 4.3 MB until the
// process exits.  All calls share them, so calls that overlap on the GPU race.
static constexpr int64_t kNoAllocMaxElems = (int64_t)1 << 20;
static constexpr int32_t kNoAllocMaxIters = 1024;
static constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) float g_noalloc_tmp[kNoAllocMaxElems];
static __device__ __align__(256) double g_noalloc_norm2[(kNoAllocMaxIters + 1) * 32];

namespace {
std::mutex g_noalloc_mu;
float* g_noalloc_tmp_ptr[kNoAllocMaxDevices] = {};
double* g_noalloc_norm2_ptr[kNoAllocMaxDevices] = {};

// Device addresses of the static scratch for the current device.  In host code
// the array names are host-side stand-ins, not device addresses, so they are
// translated once per device with cudaGetSymbolAddress.
ludvig_status noalloc_scratch(float** tmp, double** norm2) {
    int dev = 0;
    LV_CUDA(cudaGetDevice(&dev));
    LV_ARG(dev >= 0 && dev < kNoAllocMaxDevices, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_tmp_ptr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        LV_CUDA(cudaGetSymbolAddress(&a, g_noalloc_tmp));
        LV_CUDA(cudaGetSymbolAddress(&b, g_noalloc_norm2));
        g_noalloc_tmp_ptr[dev] = static_cast<float*>(a);
        g_noalloc_norm2_ptr[dev] = static_cast<double*>(b);
    }
    *tmp = g_noalloc_tmp_ptr[dev];
    *norm2 = g_noalloc_norm2_ptr[dev];
    return LUDVIG_OK;
}
}  // namespace

extern "C" ludvig_status ludvig_diffuse_noalloc(ludvig_graph_t g, const float* x0, int32_t dx, int32_t iters,
                                                float* out, void* stream) {
    LV_ARG(g != nullptr, "graph is NULL");
    LV_ARG(dx >= 1 && dx <= 32, "dx must be in [1, 32]");
    LV_ARG(iters >= 0 && iters <= kNoAllocMaxIters, "iters must be in [0, %d] for the allocation-free call",
           kNoAllocMaxIters);
    LV_ARG(x0 != nullptr && out != nullptr, "NULL buffer");
    LV_ARG(x0 != out, "out must not alias x0");
    const int64_t n = g->n;
    LV_ARG(n * dx <= kNoAllocMaxElems, "n * dx = %lld exceeds the allocation-free limit of %lld elements",
           (long long)(n * dx), (long long)kNoAllocMaxElems);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) return LUDVIG_OK;
    const size_t bytes = sizeof(float) * (size_t)n * dx;
    if (iters == 0) {
        LV_CUDA(cudaMemcpyAsync(out, x0, bytes, cudaMemcpyDeviceToDevice, st));
        return LUDVIG_OK;
    }
    float* tmp;
    double* n2;
    LV_TRY(noalloc_scratch(&tmp, &n2));
    float* bufs[2] = {(iters % 2 == 1) ? out : tmp, (iters % 2 == 1) ? tmp : out};
    // the norm accumulators keep the previous call's sums: clear the slots used
    LV_CUDA(cudaMemsetAsync(n2, 0, sizeof(double) * 32 * (size_t)(iters + 1), st));
    k_colnorm2<<<(unsigned)std::min<int64_t>(592, ceil_div(n, 256)), 256, 0, st>>>(x0, n, dx, n2);
    LV_LAUNCH();
    int dev = 0, sms = 152;
    LV_CUDA(cudaGetDevice(&dev));
    LV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(n, 32)));
    const float* xin = x0;
    for (int t = 0; t < iters; ++t) {
        float* y = bufs[t & 1];
        if (dx == 1)
            k_spmv_scaled<8><<<blocks, 256, 0, st>>>(g->row_ptr, g->col, g->val, xin, n, 1, n2 + 32 * t, y,
                                                     n2 + 32 * (t + 1));
        else
            k_spmv_cols<<<blocks, 256, 0, st>>>(g->row_ptr, g->col, g->val, xin, n, dx, n2 + 32 * t, y,
                                                n2 + 32 * (t + 1));
        LV_LAUNCH();
        xin = y;
    }
    return LUDVIG_OK;
}

// ---------------------------------------------------------------- paper-form diffusion
// Eq. 7 with the appendix's similarity and unary term, and the segmentation
// variant of Sec. 4.1:
//   S_f(f_i, f_j) = exp(-||f^_i - f^_j||^2 / (b s_f^2))   (f^ l2-normalised,
//                   s_f the median edge distance),
//   P(f_i) = S_f(f_i, f_bar) with bandwidth b_P (f_bar the normalised mean of
//            the anchors' normalised features),
//   A_ij = S_f(f_i, f_j) P_i^1/2 P_j^1/2, thresholded at 1e-5 for segmentation,
//   g_0 = the top 10 % of the uplifted reference mask's positive values,
//   h_i = P_i on the nodes that g_T reaches, 0 elsewhere.
// The graph keeps each edge's ||f^_i - f^_j||^2 (the scene part, computed
// once); ludvig_graph_reweight forms A for a prompt's P.

namespace ludvig {
namespace {

__global__ void k_float_keys(const float* __restrict__ v, int64_t m, int64_t mpad, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mpad) return;
    keys[i] = i < m ? __float_as_uint(v[i]) : 0xffffffffu;   // non-negative floats order like their bits
    vals[i] = (uint32_t)i;
}

// s_f = median of sqrt(d2) over the edges: the mean of the two middle values
// of the sorted squared distances' roots (one value for an odd count).
__global__ void k_median_sf(const uint32_t* __restrict__ sorted, int64_t m, float* __restrict__ sf) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (m == 0) {
        *sf = 0.f;
        return;
    }
    const float a = sqrtf(__uint_as_float(sorted[(m - 1) / 2])), b = sqrtf(__uint_as_float(sorted[m / 2]));
    *sf = (m & 1) ? a : 0.5f * (a + b);
}

// One warp per row: A_ij = exp(-d2 inv) sqrt(P_i P_j), thresholded and
// row-normalised on request.
__global__ void __launch_bounds__(256) k_rbf_reweight(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const float* __restrict__ d2, const float* __restrict__ P,
                                                      int64_t n, float inv, float binarize, int row_normalize,
                                                      float* __restrict__ val) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    const float spi = P ? sqrtf(P[i]) : 1.f;   // sqrt(P_i) sqrt(P_j): the product P_i P_j may underflow
    float rsum = 0.f;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
        float w = expf(-d2[e] * inv);
        if (P) w *= spi * sqrtf(P[col[e]]);
        if (binarize > 0.f) w = w > binarize ? 1.f : 0.f;
        val[e] = w;
        rsum += w;
    }
    if (!row_normalize) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    // divide (not multiply by 1/sum): a denormal sum has an infinite reciprocal
    if (rsum > 0.f)
        for (int64_t e = e0 + lane; e < e1; e += 32) val[e] = val[e] / rsum;
}

// Sum of the normalised features of the anchor nodes (g0_i > 0), per channel,
// in float64: block b takes rows [b R, (b + 1) R), thread t channels t, t + 256, ...
constexpr int kAnchorRows = 1024;
__global__ void __launch_bounds__(256) k_anchor_sum(const float* __restrict__ f, const float* __restrict__ nrm,
                                                    const float* __restrict__ g0, int64_t n, int df,
                                                    double* __restrict__ acc) {
    const int64_t r0 = (int64_t)blockIdx.x * kAnchorRows, r1 = n < r0 + kAnchorRows ? n : r0 + kAnchorRows;
    for (int c = threadIdx.x; c < df; c += blockDim.x) {
        float s = 0.f;
        for (int64_t i = r0; i < r1; ++i)
            if (g0[i] > 0.f && nrm[i] > 0.f) s += f[i * df + c] / nrm[i];
        if (s != 0.f) atomicAdd(acc + c, (double)s);
    }
}

// f_bar = acc / ||acc|| (zero when acc is zero), one block.
__global__ void k_anchor_finish(const double* __restrict__ acc, int df, float* __restrict__ fbar) {
    __shared__ double red[256];
    double s = 0.0;
    for (int c = threadIdx.x; c < df; c += blockDim.x) s += acc[c] * acc[c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double nr = sqrt(red[0]);
    for (int c = threadIdx.x; c < df; c += blockDim.x) fbar[c] = nr > 0.0 ? (float)(acc[c] / nr) : 0.f;
}

// P_i = exp(-||f^_i - f_bar||^2 inv), one warp per row.
__global__ void __launch_bounds__(256) k_unary(const float* __restrict__ f, const float* __restrict__ nrm,
                                               const float* __restrict__ fbar, int64_t n, int df, float inv,
                                               float* __restrict__ P) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + warp;
    if (i >= n) return;
    const float ni = nrm[i];
    const float sc = ni > 0.f ? 1.0f / ni : 0.f;
    float d2 = 0.f;
    for (int c = lane; c < df; c += 32) {
        const float t = f[i * df + c] * sc - fbar[c];
        d2 = fmaf(t, t, d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if (lane == 0) P[i] = expf(-d2 * inv);
}

// Top-percent selection of the positive values: keys as in the beta
// selection (descending value, ties in index order), positives counted.
__global__ void k_topfrac_keys(const float* __restrict__ u, int64_t n, int64_t npad, uint32_t* __restrict__ keys,
                               uint32_t* __restrict__ vals, unsigned long long* __restrict__ npos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool pos = false;
    if (i < npad) {
        uint32_t k = 0xffffffffu;
        if (i < n && u[i] > 0.f) {
            k = ~__float_as_uint(u[i]);
            pos = true;
        }
        keys[i] = k;
        vals[i] = (uint32_t)i;
    }
    const unsigned m = __ballot_sync(0xffffffffu, pos);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(npos, (unsigned long long)__popc(m));
}

__global__ void k_topfrac_mark(const uint32_t* __restrict__ vals, const float* __restrict__ u, int64_t n,
                               const unsigned long long* __restrict__ npos, int percent, float* __restrict__ g0) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t keep = (int64_t)((*npos * (unsigned long long)percent + 99ull) / 100ull);
    if (k < keep && k < n) g0[vals[k]] = u[vals[k]];
}

// Reachability as bit sets (bit q = query column q): s_{t+1,i} = OR over the
// row's edges with A_ij > 0 of s_t,j, one warp per row.
__global__ void k_reach_init(const float* __restrict__ g0, int64_t n, int dx, uint32_t* __restrict__ s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t b = 0u;
    for (int q = 0; q < dx; ++q)
        if (g0[i * dx + q] > 0.f) b |= 1u << q;
    s[i] = b;
}

// Eight lanes per row (a row holds k to 2k entries): four rows per warp are in
// flight at once, since each row is a short chain of dependent loads (row
// pointer, entries, the neighbours' bits).
constexpr int kReachLanes = 8;

__global__ void __launch_bounds__(256) k_reach_step(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                    const float* __restrict__ val, const uint32_t* __restrict__ s,
                                                    int64_t n, uint32_t* __restrict__ s2) {
    const int sub = threadIdx.x & (kReachLanes - 1);
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kReachLanes;
    uint32_t b = 0u;
    if (i < n)
        for (int64_t e = rp[i] + sub, e1 = rp[i + 1]; e < e1; e += kReachLanes)
            if (val[e] > 0.f) b |= s[col[e]];
#pragma unroll
    for (int o = kReachLanes / 2; o > 0; o >>= 1) b |= __shfl_xor_sync(0xffffffffu, b, o);
    if (i < n && sub == 0) s2[i] = b;
}

__global__ void k_reach_out(const uint32_t* __restrict__ s, const float* __restrict__ P, int64_t n, int dx,
                            float* __restrict__ h) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * dx) return;
    const int64_t i = t / dx;
    const int q = (int)(t - i * dx);
    h[t] = ((s[i] >> q) & 1u) ? (P ? P[i] : 1.f) : 0.f;
}

}  // namespace
}  // namespace ludvig

extern "C" ludvig_status ludvig_graph_build_rbf(ludvig_scene_t scene, int32_t k, const float* feats, int32_t df,
                                                void* stream, ludvig_graph_t* out) {
    LV_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(k >= 1 && k <= 64, "k must be in [1, 64]");
    LV_ARG(df >= 1 && (feats != nullptr || scene->n == 0), "features required (df >= 1)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ludvig_graph_t g = nullptr;
    LV_TRY(graph_build_impl(scene, k, feats, df, 1.0f, 0.f, 0, kEdgeFeatureDist2, st, &g));
    // the squared distances move to d2; val gets S_f with b = 1 and no unary term
    g->d2 = g->val;
    g->val = nullptr;
    const int64_t m = g->nnz;
    auto fail = [&](ludvig_status r) {
        ludvig_graph_destroy(g);
        return r;
    };
    if (cudaMalloc(&g->val, sizeof(float) * (size_t)std::max<int64_t>(m, 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("graph allocation failed");
        return fail(LUDVIG_ERR_OOM);
    }
    if (g->n == 0) {
        *out = g;
        return LUDVIG_OK;
    }
    const int64_t mpad = round_up(std::max<int64_t>(m, 1), kRadixTile);
    uint32_t *keys, *vals, *keys2, *vals2;
    float* sf_d;
    void* hb;
    Arena& ws = g->ws;
    ludvig_status r = LUDVIG_OK;
    if ((r = ws.get("rbf.keys", (size_t)mpad, &keys)) != LUDVIG_OK || (r = ws.get("rbf.vals", (size_t)mpad, &vals)) ||
        (r = ws.get("rbf.keys2", (size_t)mpad, &keys2)) || (r = ws.get("rbf.vals2", (size_t)mpad, &vals2)) ||
        (r = ws.get("rbf.sf", 1, &sf_d)) || (r = ws.pinned("rbf.sf_h", 16, &hb)))
        return fail(r);
    {
        StageScope scope(LUDVIG_STAGE_GRAPH, st);
        k_float_keys<<<grid_for(mpad, 256), 256, 0, st>>>(g->d2, m, mpad, keys, vals);
        count_launch();
        uint32_t *sk = keys, *sv = vals;
        if ((r = radix_sort_pairs(&sk, &sv, keys2, vals2, 1, mpad, 32, ws, st)) != LUDVIG_OK) return fail(r);
        k_median_sf<<<1, 32, 0, st>>>(sk, m, sf_d);
        count_launch();
        if (cudaMemcpyAsync(hb, sf_d, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("graph: CUDA failure");
            return fail(LUDVIG_ERR_CUDA);
        }
    }
    g->s_f = *static_cast<float*>(hb);
    if (g->s_f > 0.f) {
        if ((r = ludvig_graph_reweight(g, 1.0f, nullptr, 0.f, 0, stream)) != LUDVIG_OK) return fail(r);
    } else if (m > 0 && cudaMemsetAsync(g->val, 0, sizeof(float) * (size_t)m, st) != cudaSuccess) {
        set_error("graph: CUDA failure");
        return fail(LUDVIG_ERR_CUDA);
    }
    *out = g;
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_graph_feature_scale(ludvig_graph_t graph, float* s_f) {
    LV_ARG(graph != nullptr && s_f != nullptr, "NULL argument");
    LV_ARG(graph->d2 != nullptr || graph->n == 0, "not an RBF graph (ludvig_graph_build_rbf)");
    *s_f = graph->s_f;
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_graph_reweight(ludvig_graph_t graph, float bandwidth, const float* unary,
                                               float binarize, int32_t row_normalize, void* stream) {
    LV_ARG(graph != nullptr, "graph is NULL");
    LV_ARG(graph->d2 != nullptr || graph->n == 0, "not an RBF graph (ludvig_graph_build_rbf)");
    LV_ARG(bandwidth > 0.f, "bandwidth must be positive");
    if (graph->n == 0 || graph->nnz == 0) return LUDVIG_OK;
    LV_ARG(graph->s_f > 0.f, "the median edge distance is 0: the RBF similarity is undefined");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StageScope scope(LUDVIG_STAGE_GRAPH, st);
    ++graph->val_version;
    const float inv = 1.0f / (bandwidth * graph->s_f * graph->s_f);
    k_rbf_reweight<<<grid_for(graph->n, 8), 256, 0, st>>>(graph->row_ptr, graph->col, graph->d2, unary, graph->n,
                                                          inv, binarize, row_normalize, graph->val);
    LV_LAUNCH();
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_unary_anchor(ludvig_graph_t graph, const float* feats, int32_t df, const float* g0,
                                             float bandwidth, float* unary, void* stream) {
    LV_ARG(graph != nullptr, "graph is NULL");
    LV_ARG(graph->d2 != nullptr || graph->n == 0, "not an RBF graph (ludvig_graph_build_rbf)");
    LV_ARG(df >= 1 && df <= 4096, "df must be in [1, 4096]");
    LV_ARG(bandwidth > 0.f, "bandwidth must be positive");
    const int64_t n = graph->n;
    if (n == 0) return LUDVIG_OK;
    LV_ARG(feats != nullptr && g0 != nullptr && unary != nullptr, "NULL buffer");
    LV_ARG(graph->s_f > 0.f, "the median edge distance is 0: the RBF similarity is undefined");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena& ws = graph->ws;
    float *nrm, *fbar;
    double* acc;
    LV_TRY(ws.get("un.nrm", (size_t)n, &nrm));
    LV_TRY(ws.get("un.fbar", (size_t)df, &fbar));
    LV_TRY(ws.get("un.acc", (size_t)df, &acc));
    StageScope scope(LUDVIG_STAGE_GRAPH, st);
    LV_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)df, st));
    k_norms<<<grid_for(n, 8), 256, 0, st>>>(feats, n, df, nrm);
    LV_LAUNCH();
    k_anchor_sum<<<(unsigned)ceil_div(n, kAnchorRows), 256, 0, st>>>(feats, nrm, g0, n, df, acc);
    LV_LAUNCH();
    k_anchor_finish<<<1, 256, 0, st>>>(acc, df, fbar);
    LV_LAUNCH();
    const float inv = 1.0f / (bandwidth * graph->s_f * graph->s_f);
    k_unary<<<grid_for(n, 8), 256, 0, st>>>(feats, nrm, fbar, n, df, inv, unary);
    LV_LAUNCH();
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_topfrac_positive(ludvig_scene_t scene, const float* u, int32_t percent, float* g0,
                                                 void* stream) {
    LV_ARG(scene != nullptr, "scene is NULL");
    LV_ARG(percent >= 0 && percent <= 100, "percent must be in [0, 100]");
    const int64_t n = scene->n;
    if (n == 0) return LUDVIG_OK;
    LV_ARG(u != nullptr && g0 != nullptr, "NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Arena& ws = scene->ws;
    const int64_t npad = round_up(n, kRadixTile);
    uint32_t *keys, *vals, *keys2, *vals2;
    unsigned long long* npos;
    LV_TRY(ws.get("tf.keys", (size_t)npad, &keys));
    LV_TRY(ws.get("tf.vals", (size_t)npad, &vals));
    LV_TRY(ws.get("tf.keys2", (size_t)npad, &keys2));
    LV_TRY(ws.get("tf.vals2", (size_t)npad, &vals2));
    LV_TRY(ws.get("tf.npos", 1, &npos));
    StageScope scope(LUDVIG_STAGE_FILTER, st);
    LV_CUDA(cudaMemsetAsync(npos, 0, sizeof(unsigned long long), st));
    LV_CUDA(cudaMemsetAsync(g0, 0, sizeof(float) * (size_t)n, st));
    k_topfrac_keys<<<grid_for(npad, 256), 256, 0, st>>>(u, n, npad, keys, vals, npos);
    LV_LAUNCH();
    uint32_t *sk = keys, *sv = vals;
    LV_TRY(radix_sort_pairs(&sk, &sv, keys2, vals2, 1, npad, 32, ws, st));
    k_topfrac_mark<<<grid_for(n, 256), 256, 0, st>>>(sv, u, n, npos, percent, g0);
    LV_LAUNCH();
    return LUDVIG_OK;
}

extern "C" ludvig_status ludvig_reach_weight(ludvig_graph_t graph, const float* g0, int32_t dx, int32_t steps,
                                             const float* unary, float* h, void* stream) {
    LV_ARG(graph != nullptr, "graph is NULL");
    LV_ARG(dx >= 1 && dx <= 32, "dx must be in [1, 32]");
    LV_ARG(steps >= 0, "steps must be >= 0");
    const int64_t n = graph->n;
    if (n == 0) return LUDVIG_OK;
    LV_ARG(g0 != nullptr && h != nullptr, "NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *s0, *s1;
    LV_TRY(graph->ws.get("reach.s0", (size_t)n, &s0));
    LV_TRY(graph->ws.get("reach.s1", (size_t)n, &s1));
    StageScope scope(LUDVIG_STAGE_DIFFUSE, st);
    k_reach_init<<<grid_for(n, 256), 256, 0, st>>>(g0, n, dx, s0);
    LV_LAUNCH();
    for (int t = 0; t < steps; ++t) {
        k_reach_step<<<grid_for(n * kReachLanes, 256), 256, 0, st>>>(graph->row_ptr, graph->col, graph->val, s0, n,
                                                                      s1);
        LV_LAUNCH();
        std::swap(s0, s1);
    }
    k_reach_out<<<grid_for(n * dx, 256), 256, 0, st>>>(s0, unary, n, dx, h);
    LV_LAUNCH();
    return LUDVIG_OK;
}
