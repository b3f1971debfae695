// Storage-type conversion and the real spherical-harmonic basis shared by
// the projection (project.cu) and the ray-order renderer (raycast.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace dl {

template <typename T>
__device__ __forceinline__ float to_f(T x);
template <>
__device__ __forceinline__ float to_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float to_f<__half>(__half x) { return __half2float(x); }

// Real spherical-harmonic normalisations (closed forms in the comments).
constexpr float kY00 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15 / pi) / 2
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5 / pi) / 4
constexpr float kY2c = 0.54627421529603959f;   // sqrt(15 / pi) / 4
constexpr float kY3a = 0.59004358992664352f;   // sqrt(35 / (2 pi)) / 4
constexpr float kY3b = 2.8906114426405538f;    // sqrt(105 / pi) / 2
constexpr float kY3c = 0.45704579946446572f;   // sqrt(21 / (2 pi)) / 4
constexpr float kY3d = 0.37317633259011540f;   // sqrt(7 / pi) / 4
constexpr float kY3e = 1.4453057213202769f;    // sqrt(105 / pi) / 4
constexpr float kLog2e = 1.4426950408889634f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kY00;
    if (DEG >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

}  // namespace dl
