// Scene layout on load: Gaussians are reordered along a 3D Morton curve of
// their means, so that the 32 Gaussians a warp projects together are close in
// space.  They then land in the same few (view, tile) groups, which lets the
// projection and the key emission merge their atomic counter updates per
// warp, and the records a tile composites sit close together in memory.  The
// order only changes which index breaks exact depth ties.
#include "dl_internal.cuh"

namespace dl {
namespace {

__device__ __forceinline__ uint32_t ordered_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// bounds[0..2] = ordered min of x, y, z; bounds[3..5] = ordered max.
__global__ void bounds_kernel(const float* __restrict__ mean, int64_t n, uint32_t* __restrict__ bounds) {
    uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float f = mean[3 * i + a];
            if (!(f == f)) continue;  // NaN: ignored
            const uint32_t o = ordered_bits(f);
            lo[a] = min(lo[a], o);
            hi[a] = max(hi[a], o);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
        hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(bounds + a, lo[a]);
            atomicMax(bounds + 3 + a, hi[a]);
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void morton_kernel(const float* __restrict__ mean, int64_t n,
                              const uint32_t* __restrict__ bounds, unsigned long long* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    float lo[3], ext[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = from_ordered(bounds[a]);
        const float hi = from_ordered(bounds[3 + a]);
        ext[a] = hi > lo[a] ? 1023.999f / (hi - lo[a]) : 0.f;
    }
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        uint32_t q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float t = (mean[3 * i + a] - lo[a]) * ext[a];
            t = fminf(fmaxf(t, 0.f), 1023.f);  // NaN -> 0 through fmaxf
            q[a] = uint32_t(t);
        }
        keys[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
        vals[i] = uint32_t(i);
    }
}

// dst record i = src record perm[i]; records of `words` 16-bit words.
__global__ void gather_kernel(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst,
                              const uint32_t* __restrict__ perm, int64_t n, int words) {
    const int64_t total = n * words;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = t / words, w = t - i * words;
        dst[t] = src[int64_t(perm[i]) * words + w];
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

}  // namespace

size_t spatial_order_tmp_bytes(int64_t n) {
    return 256 + 2 * 8 * size_t(n) + 2 * 4 * size_t(n) + radix_tmp_bytes(n) + 1024;
}

cudaError_t launch_spatial_order(const float* mean, int64_t n, void* tmp, uint32_t** perm,
                                 cudaStream_t s) {
    char* p = static_cast<char*>(tmp);
    uint32_t* bounds = reinterpret_cast<uint32_t*>(p);
    p += 256;
    unsigned long long* k0 = reinterpret_cast<unsigned long long*>(p);
    p += 8 * size_t(n);
    unsigned long long* k1 = reinterpret_cast<unsigned long long*>(p);
    p += 8 * size_t(n);
    uint32_t* v0 = reinterpret_cast<uint32_t*>(p);
    p += 4 * size_t(n);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(p);
    p += 4 * size_t(n);
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
    cudaError_t e = cudaMemsetAsync(bounds, 0xFF, 3 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(bounds + 3, 0, 3 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    bounds_kernel<<<grid_of(n), 256, 0, s>>>(mean, n, bounds);
    morton_kernel<<<grid_of(n), 256, 0, s>>>(mean, n, bounds, k0, v0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int alt = 0;
    e = radix_sort_pairs(k0, v0, k1, v1, n, 30, p, &alt, s);
    if (e != cudaSuccess) return e;
    *perm = alt ? v1 : v0;
    return cudaSuccess;
}

cudaError_t launch_gather_records(const void* src, void* dst, const uint32_t* perm, int64_t n,
                                  size_t record_bytes, cudaStream_t s) {
    const int words = int(record_bytes / 2);
    gather_kernel<<<grid_of(n * words), 256, 0, s>>>(static_cast<const uint16_t*>(src),
                                                     static_cast<uint16_t*>(dst), perm, n, words);
    return cudaGetLastError();
}

}  // namespace dl
