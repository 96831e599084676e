// Device-side helpers shared by the kernel translation units: typed
// population loads and stores (deviations s = f - w kept as FP32, FP16,
// BF16 or FP64, arithmetic in R), the compact-cell row lookup, and the
// precision switch of the launchers.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_kernels.h"

namespace lbm {

template <class S> struct Storage;
template <> struct Storage<float> {
    using R = float;
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Storage<double> {
    using R = double;
    static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Storage<__half> {
    using R = float;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// row of compact cell c: the row of its 32-cell chunk's first cell plus the
// number of rows that begin within the chunk up to c's lane
__device__ __forceinline__ int find_row(const KParams &p, int c) {
    const int2 ch = __ldg(reinterpret_cast<const int2 *>(p.chunk_row) + (c >> 5));
    const uint32_t upto = (2u << (c & 31)) - 1u;  // lanes 0..(c & 31)
    return ch.x + __popc((uint32_t)ch.y & upto);
}

// relaxation rate of an instance in the arithmetic type R
template <class R> __device__ __forceinline__ R omega_of(const KParams &p, int inst);
template <> __device__ __forceinline__ float omega_of<float>(const KParams &p, int inst) { return __ldg(&p.omega_f[inst]); }
template <> __device__ __forceinline__ double omega_of<double>(const KParams &p, int inst) { return __ldg(&p.omega[inst]); }

template <class S> static S *as(void *p) { return static_cast<S *>(p); }

#define DISPATCH(prec, CALL)                                   \
    switch (prec) {                                            \
    case 0: { using S = float; CALL; } break;                  \
    case 1: { using S = __half; CALL; } break;                 \
    case 2: { using S = __nv_bfloat16; CALL; } break;          \
    default: { using S = double; CALL; } break;                \
    }

}  // namespace lbm
