// Declarations shared by the uplift translation units: uplift.cu (front end,
// group pipeline, entry points) and uplift_tc.cu (tensor-core kernels).
#pragma once

#include "common.cuh"
#include "spec.cuh"

namespace ludvig {

// The per-tile lists of a group of views as the compositing kernels read them.
struct GroupLists {
    const uint2* ranges;   // [nv * ntiles]: [start, end) into rank (empty tiles {0, 0})
    const uint32_t* rank;  // list entries: the Gaussian's depth rank within its view
    const PairRec* srec;   // [nv, npad]: projected records in depth order (mask word unused)
    int64_t npad;
};

// The weight rows of a group (k_weights output) in chunks of 128 rows.
struct TileWeights {
    int64_t cap = 0;          // chunks the buffers hold
    int count = -1;           // chunks used, when read back by a checked run (else -1)
    int* counter = nullptr;   // device: chunks used
    uint8_t *wg1 = nullptr, *wg2 = nullptr;
    uint32_t* cgid = nullptr;
    int *crows = nullptr, *cnext = nullptr, *ifirst = nullptr;
    float* cden = nullptr;
    uint32_t* plan_off = nullptr;   // [nitems + 1]: each tile's entries in plan
    int2* plan = nullptr;           // [cap]: {chunk, rows} of the non-empty chunks, tile after tile
};

bool tc_supported(int dtype, int d);

// Internal dtype code of FP8-E4M3 codes read by the aggregation (decoded in
// the kernel: x = decode(q) s_v rounded to bfloat16); d % 16 == 0, 32..512.
constexpr int kDtypeE4M3 = 2;
inline bool tc_e4m3_supported(int d) { return d >= 32 && d <= 512 && d % 16 == 0; }

// k_weights over every (view, tile) of a group into the buffers of `parity`
// (0 or 1, so that a group's weights can be formed while the previous group's
// are aggregated).  checked: the chunk count is read back (synchronises `st`)
// and the pass re-run with more chunks until they fit.  Otherwise it runs once
// with *chunk_cap chunks and the aggregation checks the count on the device.
ludvig_status tc_weights(const GroupLists& L, int nv, int width, int height, int NT, Arena& ws, int parity,
                         int* status, int64_t* chunk_cap, bool checked, cudaStream_t st, TileWeights* tw);

// Allocates both buffer sets of the weight rows for groups of up to nitems
// (view, tile) items and cap chunks (allocation synchronises the device, so an
// asynchronous call that finds them in place never waits).
ludvig_status tc_reserve(Arena& ws, int NT, int nitems, int64_t cap);

// num[i,:] += W^T F and den[i] += row sums for the group's weight rows
// (k_aggregate_tc).  When the weights overflowed their chunks the kernel adds
// nothing and sets bit 1 (value 2) of *ovf (ovf may be null for checked runs).
ludvig_status tc_aggregate(const TileWeights& t, int nv, int width, int height, const void* feats, int dtype,
                           int d, float* num, float* den, int* status, int* ovf, cudaStream_t st,
                           const float* scales = nullptr);

// F_hat = W f for the group (k_render_tc); t must come from a checked tc_weights.
ludvig_status tc_render(const TileWeights& t, Arena& ws, int nv, int width, int height, const float* f, int d,
                        float* out, int* status, cudaStream_t st);

// Enqueues the bounded-wait check kernel: on expiry after `cycles` clock
// cycles it sets *status to LUDVIG_ERR_TIMEOUT.
ludvig_status tc_wait_into_status(int64_t cycles, int* status, cudaStream_t st);

}  // namespace ludvig
