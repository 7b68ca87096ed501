// Device-wide exclusive scan and stable LSD radix sort (reduce-then-scan).
//
// The radix sort orders (key, value) pairs by 8-bit digits, least significant
// first.  Each pass: (1) every block histograms the digits of its 4096-key
// tile, (2) one exclusive scan over the histograms laid out
// [segment][digit][block] gives every (block, digit) its output base, (3)
// every block re-reads its tile, ranks each key among the equal digits before
// it in the tile (warp match/popc, then a prefix over the warps), sorts the
// tile by digit in shared memory and writes each digit's run to its base.
// Segment-major histogram order keeps equal-length segments apart, so one
// launch sorts many views.
#include "common.cuh"

namespace ludvig {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* out_excl) {
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nwarps ? warp_tot[lane] : 0u;
        t = warp_incl_scan(t);
        warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? warp_tot[warp - 1] : 0u;
    *out_excl = before + incl - v;
    const uint32_t total = warp_tot[nwarps - 1];
    __syncthreads();
    return total;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// 64-bit block sum (a tile of 4096 counts may exceed 32 bits).
__device__ __forceinline__ unsigned long long block_sum64(unsigned long long v) {
    __shared__ unsigned long long part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (warp == 0) {
        t = lane < (int)((blockDim.x + 31) >> 5) ? part[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in warp 0
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                              unsigned long long* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    const unsigned long long tot = block_sum64(s);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place, carrying across chunks.
__global__ void k_scan_sums(unsigned long long* __restrict__ sums, int64_t nb,
                            unsigned long long* __restrict__ total) {
    __shared__ unsigned long long wt[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    unsigned long long carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const unsigned long long v = i < nb ? sums[i] : 0ull;
        const unsigned long long incl = warp_incl_scan64(v);
        if (lane == 31) wt[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = lane < nwarps ? wt[lane] : 0ull;
            wt[lane] = warp_incl_scan64(t);
        }
        __syncthreads();
        const unsigned long long before = warp > 0 ? wt[warp - 1] : 0ull;
        if (i < nb) sums[i] = carry + before + incl - v;
        carry += wt[nwarps - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             const unsigned long long* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t excl;
    block_excl_scan(s, &excl);
    uint32_t run = (uint32_t)sums[blockIdx.x] + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// ------------------------------------------------------------------ radix

// Keys of a sort whose length lives in device memory (`len`, one segment):
// entries at or past the length read as the largest key (they sort last), and
// blocks that start past it take no part (zero histogram, no output).
__device__ __forceinline__ int64_t radix_valid(const uint64_t* len, int64_t seg_len) {
    return len ? (int64_t)min((uint64_t)seg_len, *len) : seg_len;
}

// Keys are 32-bit or 16-bit (KeyT); entries past the valid length read as the
// type's largest key.
template <class KeyT>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_upsweep(const KeyT* __restrict__ keys, int shift, uint32_t* __restrict__ hist, int64_t bps,
                const uint64_t* __restrict__ len) {
    constexpr uint32_t kFill = (uint32_t)(KeyT)~(KeyT)0;
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    // positions within the block's segment are compared with the valid length
    const int64_t seg_base = (int64_t)(blockIdx.x % bps) * kRadixTile;
    const int64_t valid = radix_valid(len, bps * kRadixTile);
    if (seg_base < valid) {
#pragma unroll 4
        for (int i = 0; i < kRadixItems; ++i) {
            const int64_t off = i * kRadixThreads + threadIdx.x;
            const uint32_t k = seg_base + off < valid ? (uint32_t)keys[base + off] : kFill;
            atomicAdd(&h[(k >> shift) & 0xffu], 1u);
        }
    }
    __syncthreads();
    const int64_t seg = blockIdx.x / bps, b = blockIdx.x % bps;
    hist[(seg * 256 + threadIdx.x) * bps + b] = h[threadIdx.x];
}

// Warp w owns keys [512 w, 512 w + 512) of the block's tile (16 rounds of 32
// consecutive keys), so per-digit counts accumulate warp-locally in tile order;
// one block prefix over the warps then gives every key its place in the tile
// sorted by digit (stable).  The tile is sorted in shared memory and written
// out in digit runs, so the stores coalesce.
template <class KeyT>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_downsweep(const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
                  KeyT* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
                  const uint32_t* __restrict__ hist, int64_t bps, const uint64_t* __restrict__ len) {
    constexpr int kWarps = kRadixThreads / 32;
    constexpr uint32_t kFill = (uint32_t)(KeyT)~(KeyT)0;
    __shared__ uint32_t s_key[kRadixTile];
    __shared__ uint32_t s_val[kRadixTile];
    __shared__ uint32_t wcnt[kWarps][256];   // per-warp digit counts, then their prefix
    __shared__ uint32_t dstart[256];          // first tile position of each digit
    __shared__ uint32_t obase[256];           // output position of each digit's first key
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t seg = blockIdx.x / bps, b = blockIdx.x % bps;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    const int64_t seg_base = b * kRadixTile;   // the block's position within its segment
    const int64_t valid = radix_valid(len, bps * kRadixTile);
    if (seg_base >= valid) return;   // (whole block uniform)
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    uint32_t k[kRadixItems], v[kRadixItems], rk[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t off = warp * (32 * kRadixItems) + i * 32 + lane;
        k[i] = seg_base + off < valid ? (uint32_t)kin[base + off] : kFill;
        v[i] = seg_base + off < valid ? vin[base + off] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const uint32_t d = (k[i] >> shift) & 0xffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = wcnt[warp][d];   // equal digits in this warp's earlier rounds
        rk[i] = before + __popc(peers & lt_mask);
        __syncwarp();
        if ((peers & lt_mask) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit tid: exclusive prefix over the warps, tile total
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = tot;
        tot += c;
    }
    obase[tid] = hist[(seg * 256 + tid) * bps + b];
    uint32_t ex;
    {
        // exclusive scan of tot over the 256 digits
        __shared__ uint32_t wsum[kWarps];
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w)
            if (w < warp) before += wsum[w];
        ex = before + incl - tot;
    }
    dstart[tid] = ex;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const uint32_t d = (k[i] >> shift) & 0xffu;
        const uint32_t pos = dstart[d] + wcnt[warp][d] + rk[i];
        s_key[pos] = k[i];
        s_val[pos] = v[i];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < kRadixItems; ++i) {
        const int p = i * kRadixThreads + tid;
        const uint32_t kk = s_key[p];
        const uint32_t d = (kk >> shift) & 0xffu;
        const uint32_t o = obase[d] + (uint32_t)p - dstart[d];
        kout[o] = (KeyT)kk;
        vout[o] = s_val[p];
    }
}

// ------------------------------------------------------------------ one-sweep radix
// The same stable LSD sort with the per-pass histogram scan chained through
// the blocks of each pass instead of a device-wide scan between kernels (the
// one-sweep scheme of Adinets and Merrill, 2022, "Onesweep: a faster least
// significant digit radix sort for GPUs"): one kernel histograms the digits of
// every pass per segment up front; each pass is then one kernel in which a
// block takes the next tile in order (a counter, so every earlier tile belongs
// to a block that has started), ranks its keys as k_radix_downsweep does,
// publishes its per-digit counts, and adds up the counts of the earlier tiles
// of its segment (the last inclusive prefix published, plus the counts after
// it) to find where each digit's run goes.  Waits are bounded: past the limit
// the block records LUDVIG_ERR_TIMEOUT in *err and goes on with what it has.

constexpr uint64_t kOsAgg = 1ull << 62, kOsIncl = 2ull << 62, kOsValMask = (1ull << 62) - 1ull;
constexpr int kOsSpinLimit = 1 << 22;

__global__ void __launch_bounds__(kRadixThreads)
k_os_hist(const uint32_t* __restrict__ keys, int64_t bps, const uint64_t* __restrict__ len, int npass,
          uint32_t* __restrict__ ghist) {
    __shared__ uint32_t h[4][256];
    for (int p = 0; p < 4; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    const int64_t seg = blockIdx.x / bps, seg_base = (int64_t)(blockIdx.x % bps) * kRadixTile;
    const int64_t valid = radix_valid(len, bps * kRadixTile);
    if (seg_base >= valid) return;   // (whole block uniform)
#pragma unroll 4
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t off = i * kRadixThreads + threadIdx.x;
        const uint32_t k = seg_base + off < valid ? keys[base + off] : 0xffffffffu;
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int p = 0; p < npass; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[(seg * npass + p) * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// A status word as the L2 holds it (a relaxed device-scope load; the word
// itself carries everything the reader uses).
__device__ __forceinline__ uint64_t os_read(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(kRadixThreads)
k_os_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
          uint32_t* __restrict__ vout, int pass, int npass, const uint32_t* __restrict__ ghist, int64_t bps,
          const uint64_t* __restrict__ len, uint64_t* __restrict__ status, uint32_t* __restrict__ counter,
          int* __restrict__ err) {
    constexpr int kWarps = kRadixThreads / 32;
    __shared__ uint32_t s_key[kRadixTile];
    __shared__ uint32_t s_val[kRadixTile];
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ uint64_t obase[256];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = 8 * pass;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    const int64_t seg = t / bps, b = t - seg * bps;
    const int64_t base = t * kRadixTile;
    const int64_t seg_base = b * kRadixTile;
    const int64_t valid = radix_valid(len, bps * kRadixTile);
    // tiles past the valid length take no part; no tile before them waits on them
    if (seg_base >= valid) return;
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    uint32_t k[kRadixItems], v[kRadixItems], rk[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t off = warp * (32 * kRadixItems) + i * 32 + lane;
        k[i] = seg_base + off < valid ? kin[base + off] : 0xffffffffu;
        v[i] = seg_base + off < valid ? vin[base + off] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const uint32_t d = (k[i] >> shift) & 0xffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = wcnt[warp][d];
        rk[i] = before + __popc(peers & lt_mask);
        __syncwarp();
        if ((peers & lt_mask) == 0) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit tid: exclusive prefix over the warps, the tile's count
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = tot;
        tot += c;
    }
    // publish the tile's count of digit tid, then add up the earlier tiles' counts
    uint64_t* my = status + t * 256 + tid;
    if (b == 0) {
        atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(kOsIncl | tot));
    } else {
        atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(kOsAgg | tot));
    }
    uint64_t excl = 0;
    if (b > 0) {
        // windows of up to kOsWin earlier tiles, read together: the nearest
        // inclusive prefix ends the walk (the segment's first tile has one)
        constexpr int kOsWin = 8;
        const int64_t first = t - b;
        bool gave_up = false, found = false;
        for (int64_t top = t - 1; !found && !gave_up; top -= kOsWin) {
            uint64_t w[kOsWin];
#pragma unroll
            for (int j = 0; j < kOsWin; ++j) w[j] = top - j >= first ? os_read(status + (top - j) * 256 + tid) : kOsIncl;
#pragma unroll
            for (int j = 0; j < kOsWin; ++j) {
                for (int it = 0; !gave_up && (w[j] >> 62) == 0; ++it) {
                    if (it >= kOsSpinLimit) {
                        gave_up = true;
                        break;
                    }
                    if (it >= 32) __nanosleep(32);
                    w[j] = os_read(status + (top - j) * 256 + tid);
                }
            }
#pragma unroll
            for (int j = 0; j < kOsWin; ++j) {
                if (found) continue;
                excl += w[j] & kOsValMask;   // (the tiles before the segment read as an empty inclusive prefix)
                if (w[j] & kOsIncl) found = true;
            }
        }
        if (gave_up && err) atomicExch(err, (int)LUDVIG_ERR_TIMEOUT);
        atomicExch(reinterpret_cast<unsigned long long*>(my), (unsigned long long)(kOsIncl | (excl + tot)));
    }
    // where digit tid's run of this tile starts: the segment's start, the keys
    // of smaller digits in the segment, the earlier tiles' keys of this digit
    const uint32_t g = ghist[(seg * npass + pass) * 256 + tid];
    uint32_t incl = g;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint64_t gbefore = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
        if (w < warp) gbefore += wsum[w];
    obase[tid] = (uint64_t)seg * (uint64_t)(bps * kRadixTile) + gbefore + (incl - g) + excl;
    // the tile sorted by digit in shared memory (as k_radix_downsweep)
    uint32_t tincl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, tincl, o);
        if (lane >= o) tincl += x;
    }
    __syncthreads();   // wsum is reused
    if (lane == 31) wsum[warp] = tincl;
    __syncthreads();
    uint32_t tbefore = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
        if (w < warp) tbefore += wsum[w];
    dstart[tid] = tbefore + tincl - tot;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const uint32_t d = (k[i] >> shift) & 0xffu;
        const uint32_t pos = dstart[d] + wcnt[warp][d] + rk[i];
        s_key[pos] = k[i];
        s_val[pos] = v[i];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < kRadixItems; ++i) {
        const int p = i * kRadixThreads + tid;
        const uint32_t kk = s_key[p];
        const uint32_t d = (kk >> shift) & 0xffu;
        const uint64_t o = obase[d] + (uint64_t)(p - (int)dstart[d]);
        kout[o] = kk;
        vout[o] = s_val[p];
    }
}

}  // namespace

ludvig_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total_dev,
                                 Arena& ws, cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) LV_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), st));
        return LUDVIG_OK;
    }
    const int64_t nb = ceil_div(n, kScanTile);
    unsigned long long* sums = nullptr;
    LV_TRY(ws.get("scan.sums", (size_t)nb, &sums));
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    LV_LAUNCH();
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb, reinterpret_cast<unsigned long long*>(total_dev));
    LV_LAUNCH();
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
    LV_LAUNCH();
    return LUDVIG_OK;
}

ludvig_status radix_sort_pairs(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt,
                               uint32_t* vals_alt, int64_t nseg, int64_t seg_len, int nbits,
                               Arena& ws, cudaStream_t st) {
    return radix_sort_pairs_len(keys, vals, keys_alt, vals_alt, nseg, seg_len, nullptr, nbits, ws, st);
}

namespace {
template <class KeyT>
ludvig_status radix_sort_impl(KeyT** keys, uint32_t** vals, KeyT* keys_alt, uint32_t* vals_alt, int64_t nseg,
                              int64_t seg_len, const uint64_t* len, int nbits, Arena& ws, cudaStream_t st) {
    if (len && nseg != 1) {
        set_error("radix_sort_pairs_len: a device length needs one segment");
        return LUDVIG_ERR_INTERNAL;
    }
    if (nseg <= 0 || seg_len <= 0 || nbits <= 0) return LUDVIG_OK;
    if (seg_len % kRadixTile != 0) {
        set_error("radix_sort_pairs: segment length %lld not a multiple of %d", (long long)seg_len,
                  kRadixTile);
        return LUDVIG_ERR_INTERNAL;
    }
    const int64_t bps = seg_len / kRadixTile;
    const int64_t nblocks = bps * nseg;
    if (nblocks > 0x7fffffff) {
        set_error("radix_sort_pairs: too many blocks");
        return LUDVIG_ERR_ARG;
    }
    const int64_t nh = nseg * 256 * bps;
    uint32_t* hist = nullptr;
    LV_TRY(ws.get("radix.hist", (size_t)nh, &hist));
    KeyT *kin = *keys, *kout = keys_alt;
    uint32_t *vin = *vals, *vout = vals_alt;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_radix_upsweep<KeyT><<<(unsigned)nblocks, kRadixThreads, 0, st>>>(kin, shift, hist, bps, len);
        LV_LAUNCH();
        LV_TRY(scan_exclusive_u32(hist, hist, nh, nullptr, ws, st));
        k_radix_downsweep<KeyT><<<(unsigned)nblocks, kRadixThreads, 0, st>>>(kin, vin, kout, vout, shift,
                                                                             hist, bps, len);
        LV_LAUNCH();
        KeyT* tk = kin;
        kin = kout;
        kout = tk;
        uint32_t* tv = vin;
        vin = vout;
        vout = tv;
    }
    *keys = kin;
    *vals = vin;
    return LUDVIG_OK;
}
}  // namespace

ludvig_status radix_sort_pairs_len(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt,
                                   uint32_t* vals_alt, int64_t nseg, int64_t seg_len, const uint64_t* len,
                                   int nbits, Arena& ws, cudaStream_t st) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, nseg, seg_len, len, nbits, ws, st);
}

ludvig_status radix_sort_pairs_len16(uint16_t** keys, uint32_t** vals, uint16_t* keys_alt, uint32_t* vals_alt,
                                     int64_t nseg, int64_t seg_len, const uint64_t* len, int nbits, Arena& ws,
                                     cudaStream_t st) {
    if (nbits > 16) {
        set_error("radix_sort_pairs_len16: %d key bits", nbits);
        return LUDVIG_ERR_INTERNAL;
    }
    return radix_sort_impl<uint16_t>(keys, vals, keys_alt, vals_alt, nseg, seg_len, len, nbits, ws, st);
}

}  // namespace ludvig

namespace ludvig {

ludvig_status radix_sort_onesweep(uint32_t** keys, uint32_t** vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                  int64_t nseg, int64_t seg_len, const uint64_t* len, int nbits, int* err,
                                  Arena& ws, cudaStream_t st) {
    if (len && nseg != 1) {
        set_error("radix_sort_onesweep: a device length needs one segment");
        return LUDVIG_ERR_INTERNAL;
    }
    if (nseg <= 0 || seg_len <= 0 || nbits <= 0) return LUDVIG_OK;
    if (seg_len % kRadixTile != 0 || nbits > 32) {
        set_error("radix_sort_onesweep: segment length %lld not a multiple of %d", (long long)seg_len, kRadixTile);
        return LUDVIG_ERR_INTERNAL;
    }
    const int64_t bps = seg_len / kRadixTile;
    const int64_t nblocks = bps * nseg;
    if (nblocks > 0x7fffffff || seg_len * nseg >= ((int64_t)1 << 40)) {
        set_error("radix_sort_onesweep: too many blocks");
        return LUDVIG_ERR_ARG;
    }
    const int npass = (nbits + 7) / 8;
    uint32_t* ghist = nullptr;
    uint64_t* status = nullptr;
    uint32_t* counters = nullptr;
    LV_TRY(ws.get("os.hist", (size_t)nseg * npass * 256, &ghist));
    LV_TRY(ws.get("os.status", (size_t)nblocks * 256, &status));
    LV_TRY(ws.get("os.counters", 4, &counters));
    LV_CUDA(cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * (size_t)nseg * npass * 256, st));
    LV_CUDA(cudaMemsetAsync(counters, 0, sizeof(uint32_t) * 4, st));
    k_os_hist<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(*keys, bps, len, npass, ghist);
    LV_LAUNCH();
    uint32_t *kin = *keys, *vin = *vals, *kout = keys_alt, *vout = vals_alt;
    for (int pass = 0; pass < npass; ++pass) {
        LV_CUDA(cudaMemsetAsync(status, 0, sizeof(uint64_t) * (size_t)nblocks * 256, st));
        k_os_pass<<<(unsigned)nblocks, kRadixThreads, 0, st>>>(kin, vin, kout, vout, pass, npass, ghist, bps, len,
                                                              status, counters + pass, err);
        LV_LAUNCH();
        uint32_t* t = kin;
        kin = kout;
        kout = t;
        t = vin;
        vin = vout;
        vout = t;
    }
    *keys = kin;
    *vals = vin;
    return LUDVIG_OK;
}

}  // namespace ludvig
