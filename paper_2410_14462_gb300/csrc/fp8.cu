// FP8-E4M3 storage of feature maps (the precision form's 8-bit variant; the
// format is the OCP 8-bit floating point one): every view v is scaled by
// s_v = max|x| / 448 over the view (1 for an all-zero view), so that its
// largest magnitude lands on the largest finite E4M3 value, and each scaled
// value is rounded to the nearest E4M3 code (ties to even, saturating).
// The uplift of FP8 features (ludvig_uplift_fp8, with the uplift kernels)
// multiplies the codes back by s_v.
//
// Three passes over the features: a per-view maximum of |x| (the float bits
// of non-negative values order like unsigned integers, so atomicMax on them
// is exact), the scales, and the rounding of x / s_v (IEEE division, then the
// hardware's round-to-nearest-even E4M3 conversion), four values per thread.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace ludvig {

namespace {

__device__ __forceinline__ float load_x(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float load_x(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

// blockIdx.y = view; grid-stride over the view's elements.
template <class T>
__global__ void __launch_bounds__(256) k_view_absmax(const T* __restrict__ x, int64_t view_elems,
                                                     uint32_t* __restrict__ amax_bits) {
    const T* xv = x + (int64_t)blockIdx.y * view_elems;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < view_elems;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(load_x(xv, i)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = wm[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wm[w]);
        atomicMax(amax_bits + blockIdx.y, __float_as_uint(b));
    }
}

// In place: the maximum's bits become the scale.
__global__ void k_view_scales(float* __restrict__ s, int n_views) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    const float amax = __uint_as_float(reinterpret_cast<const uint32_t*>(s)[v]);
    s[v] = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
}

__device__ __forceinline__ uint32_t e4m3_of(float x, float s) {
    return (uint32_t)__nv_cvt_float_to_fp8(__fdiv_rn(x, s), __NV_SATFINITE, __NV_E4M3);
}

// Thread t rounds elements 4t .. 4t + 3 of the whole array (one 4-byte store;
// the scalar tail covers a total that is not a multiple of 4).
template <class T>
__global__ void k_quantize_e4m3(const T* __restrict__ x, const float* __restrict__ s, int64_t view_elems,
                                int64_t total, uint8_t* __restrict__ q) {
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e0 >= total) return;
    if (e0 + 4 <= total) {
        uint32_t w = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) w |= e4m3_of(load_x(x, e0 + k), s[(e0 + k) / view_elems]) << (8 * k);
        *reinterpret_cast<uint32_t*>(q + e0) = w;
    } else {
        for (int64_t e = e0; e < total; ++e) q[e] = (uint8_t)e4m3_of(load_x(x, e), s[e / view_elems]);
    }
}

}  // namespace

}  // namespace ludvig

using namespace ludvig;

extern "C" ludvig_status ludvig_fp8_quantize(const void* feats, int32_t dtype, int32_t n_views, int64_t view_elems,
                                             uint8_t* q, float* scales, void* stream) {
    LV_ARG(dtype == LUDVIG_F32 || dtype == LUDVIG_BF16, "unknown dtype %d", dtype);
    LV_ARG(n_views >= 0 && n_views <= 65535, "n_views must be in [0, 65535]");
    LV_ARG(view_elems >= 0, "view_elems must be >= 0");
    if (n_views == 0) return LUDVIG_OK;
    LV_ARG(scales != nullptr, "scales is NULL");
    LV_ARG(view_elems == 0 || (feats != nullptr && q != nullptr), "NULL buffer");
    LV_ARG(((uintptr_t)q & 3) == 0, "q must be 4-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LV_CUDA(cudaMemsetAsync(scales, 0, sizeof(float) * (size_t)n_views, st));
    if (view_elems > 0) {
        const unsigned gx = (unsigned)std::min<int64_t>(ceil_div(view_elems, 256), 1024);
        const dim3 grid(gx, (unsigned)n_views);
        if (dtype == LUDVIG_F32)
            k_view_absmax<float><<<grid, 256, 0, st>>>(static_cast<const float*>(feats), view_elems,
                                                       reinterpret_cast<uint32_t*>(scales));
        else
            k_view_absmax<__nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(feats), view_elems,
                                                               reinterpret_cast<uint32_t*>(scales));
        LV_LAUNCH();
    }
    k_view_scales<<<(unsigned)ceil_div(n_views, 256), 256, 0, st>>>(scales, n_views);
    LV_LAUNCH();
    const int64_t total = (int64_t)n_views * view_elems;
    if (total > 0) {
        const unsigned blocks = (unsigned)ceil_div(ceil_div(total, 4), 256);
        if (dtype == LUDVIG_F32)
            k_quantize_e4m3<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(feats), scales, view_elems,
                                                          total, q);
        else
            k_quantize_e4m3<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(feats), scales,
                                                                  view_elems, total, q);
        LV_LAUNCH();
    }
    return LUDVIG_OK;
}
