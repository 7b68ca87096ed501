// Declarations shared by the uplift translation units: uplift.cu (front end,
// group pipeline, entry points) and uplift_tc.cu (tensor-core kernels).
#pragma once

#include <vector>

#include "common.cuh"
#include "spec.cuh"

namespace ludvig {

// Most views one group of the pipeline holds.  Each view carries its own
// camera, scene, feature coordinate and accumulation targets in the kernels'
// parameters (so a group may mix views of several scenes).
constexpr int kMaxGroupViews = 128;

// Per-view operands of the aggregation: the view's coordinate in the feature
// array the tensor map covers, and the num [n, d] / den [n] it adds into.
struct AggViews {
    int fview[kMaxGroupViews];
    float* num[kMaxGroupViews];
    float* den[kMaxGroupViews];
};

// One view of a group: the scene it projects, its camera, its coordinate in
// the features the group reads, and the num [n, d] / den [n] it adds into (on
// the zero-padded path, num is the padded numerator [n, 32]).
struct ViewRef {
    const ludvig_scene* scene;
    ludvig_camera cam;
    int fview;
    float* num;
    float* den;
};

// The views of one group (at most kMaxGroupViews) and the largest of their
// scenes (the stride of the group's per-view Gaussian scratch).
struct GroupViews {
    std::vector<ViewRef> v;
    int64_t nmax = 0;
};

// The features of a call as its groups read them: views [*, H, W, d] at the
// coordinates the group's views name.
struct FeatSrc {
    int kind = 0;                  // 0: as given, 1: zero-padded to 32 channels, 2: FP8-E4M3 codes
    const void* feats = nullptr;   // features, or codes for kind 2
    const float* scales = nullptr; // kind 2: scales by view coordinate
    int dtype = LUDVIG_F32;        // of the given features (kind 2: decoded to bfloat16)
    int d = 1;
};

// One job of a packed batch: the arguments of one ludvig_uplift call, with its
// features at view coordinates fview0 .. fview0 + n_views - 1 of the batch's
// feature array.
struct PackedJob {
    ludvig_scene* scene;
    const ludvig_camera* cams;
    int n_views;
    int fview0;
    float* out;
    float* beta;   // may be null
};

// Uplift of jobs that share the feature array `feats` ([*, height, width, d],
// dtype), each exactly ludvig_uplift on its own scene: their views are packed
// in job order into common groups (views of several jobs in one group, up to
// kMaxGroupViews views and group_bytes of per-view Gaussian scratch), run on
// ctx's streams and workspace with device-side capacity checks; what did not
// fit is redone before the call returns (it waits for the work).  Every job's
// work is ordered after the work on `st`, and `st` waits for all of it.
// A group also holds at most packed_pixels(group_bytes, dtype) pixels (its
// weight rows grow with them).  *stats (may be null) receives the groups
// formed and those redone.
struct PackedStats {
    int groups = 0;
    int redone = 0;
};
int64_t packed_pixels(int64_t group_bytes, int dtype);
ludvig_status uplift_packed(ludvig_scene* ctx, const PackedJob* jobs, int njobs, const void* feats, int dtype, int d,
                            int width, int height, int64_t group_bytes, cudaStream_t st, PackedStats* stats);

// Whether ludvig_uplift with these features runs on the tensor cores (the
// precondition of uplift_packed).
bool packed_supported(int dtype, int d);

// The argument checks of ludvig_uplift (LUDVIG_ERR_ARG with the message set).
ludvig_status check_uplift_args(const ludvig_scene* scene, const ludvig_camera* cams, int32_t n_views, int32_t width,
                                int32_t height, const void* feats, int32_t dtype, int32_t d, const float* out);

// Finishes a scene's pending asynchronous call (ludvig_sync).
ludvig_status scene_sync(ludvig_scene* s);

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
bool tc_direct_supported(int d);
ludvig_status tc_weights_direct(const GroupLists& L, int nv, int width, int height, int NT, int d, int num_stride,
                                const void* feats, int feat_dtype, const AggViews& av, Arena& ws, int parity,
                                int* status, bool checked, cudaStream_t st, int** counter);
ludvig_status tc_weights(const GroupLists& L, int nv, int width, int height, int NT, Arena& ws, int parity,
                         int* status, int64_t* chunk_cap, bool checked, cudaStream_t st, TileWeights* tw);

// Allocates both buffer sets of the weight rows for groups of up to nitems
// (view, tile) items and cap chunks (allocation synchronises the device, so an
// asynchronous call that finds them in place never waits).
ludvig_status tc_reserve(Arena& ws, int NT, int nitems, int64_t cap);

// num_v[i,:] += W^T F and den_v[i] += row sums for the group's weight rows
// (k_aggregate_tc), view v's features at coordinate av.fview[v] of `feats`
// ([fextent, height, width, d]) and its sums into av.num[v] / av.den[v].
// FP8 codes take the scale scales[av.fview[v]].  When the weights overflowed
// their chunks the kernel adds nothing and sets bit 1 (value 2) of *ovf (ovf
// may be null for checked runs).
ludvig_status tc_aggregate(const TileWeights& t, int nv, int width, int height, const void* feats, int fextent,
                           int dtype, int d, const AggViews& av, int* status, int* ovf, cudaStream_t st,
                           const float* scales = nullptr);

// F_hat = W f for the group (k_render_tc); t must come from a checked tc_weights.
ludvig_status tc_render(const TileWeights& t, Arena& ws, int nv, int width, int height, const float* f, int d,
                        float* out, int* status, cudaStream_t st);

// Enqueues the bounded-wait check kernel: on expiry after `cycles` clock
// cycles it sets *status to LUDVIG_ERR_TIMEOUT.
ludvig_status tc_wait_into_status(int64_t cycles, int* status, cudaStream_t st);

}  // namespace ludvig
