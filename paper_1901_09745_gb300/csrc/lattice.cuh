// lattice.cuh -- compile-time lattice and storage traits for the sm_103a kernels.
//
// Velocity sets (Sec. 2.1): D3Q19 with weights 1/3, 1/18, 1/36 as printed after Eq. 3;
// D2Q9 with the textbook weights 4/9, 1/9, 1/36 (the paper names D2Q9 without printing
// them). The velocity order is the library's interface order (include/psc_lbm.h); every
// non-rest velocity i has its opposite at i + 1 (i odd) or i - 1 (i even).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace psc {

struct D2Q9 {
    static constexpr int Q = 9, D = 2;
    static constexpr int TX = 32, TY = 8, TZ = 1;   // tile = one thread block
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

struct D3Q19 {
    static constexpr int Q = 19, D = 3;
    static constexpr int TX = 32, TY = 4, TZ = 2;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
};

template <class L>
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <class L>
__host__ __device__ constexpr double weight(int i) {
    return (L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i)) == 0
               ? (L::Q == 9 ? 4.0 / 9.0 : 1.0 / 3.0)
               : ((L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i)) == 1
                      ? (L::Q == 9 ? 1.0 / 9.0 : 1.0 / 18.0)
                      : 1.0 / 36.0);
}

// Storage of the deviation d_i = f_i - w_i: FP64 and FP32 hold it as is; FP16 and BF16 hold
// scale * d_i rounded to nearest and are widened to FP32 for compute. `sc` carries
// (scale, 1/scale). ld/st convert between d_i and the stored value; ldr/str only widen and
// narrow (kScaled says whether the stored value carries the scale), for kernels that fold
// the scale into their own arithmetic.
template <typename S> struct Store;

template <> struct Store<double> {
    using T = double;
    static constexpr bool kScaled = false;
    __device__ __forceinline__ static double ld(const double *p, long long i, float2) { return p[i]; }
    __device__ __forceinline__ static void st(double *p, long long i, double v, float2) { p[i] = v; }
    __device__ __forceinline__ static double ldr(const double *p, long long i) { return p[i]; }
    __device__ __forceinline__ static void str(double *p, long long i, double v) { p[i] = v; }
};
template <> struct Store<float> {
    using T = float;
    static constexpr bool kScaled = false;
    __device__ __forceinline__ static float ld(const float *p, long long i, float2) { return p[i]; }
    __device__ __forceinline__ static void st(float *p, long long i, float v, float2) { p[i] = v; }
    __device__ __forceinline__ static float ldr(const float *p, long long i) { return p[i]; }
    __device__ __forceinline__ static void str(float *p, long long i, float v) { p[i] = v; }
};
template <> struct Store<__half> {
    using T = float;
    static constexpr bool kScaled = true;
    __device__ __forceinline__ static float ld(const __half *p, long long i, float2 sc) {
        return __half2float(p[i]) * sc.y;
    }
    __device__ __forceinline__ static void st(__half *p, long long i, float v, float2 sc) {
        p[i] = __float2half_rn(v * sc.x);
    }
    __device__ __forceinline__ static float ldr(const __half *p, long long i) { return __half2float(p[i]); }
    __device__ __forceinline__ static void str(__half *p, long long i, float v) { p[i] = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    using T = float;
    static constexpr bool kScaled = true;
    __device__ __forceinline__ static float ld(const __nv_bfloat16 *p, long long i, float2 sc) {
        return __bfloat162float(p[i]) * sc.y;
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, long long i, float v, float2 sc) {
        p[i] = __float2bfloat16_rn(v * sc.x);
    }
    __device__ __forceinline__ static float ldr(const __nv_bfloat16 *p, long long i) { return __bfloat162float(p[i]); }
    __device__ __forceinline__ static void str(__nv_bfloat16 *p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }
};

}  // namespace psc
