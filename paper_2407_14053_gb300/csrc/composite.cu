// Front-to-back alpha compositing (Sec. 3.2 Eq. (5), Sec. 3.3 Eq. (10)) and
// the standard paradigm's interweave (Alg. 1).
//
// Both compositing kernels stream one (view, tile) list of depth-sorted
// Gaussian records through shared memory in batches; every thread composites
// its own ray against the whole batch and the block stops as soon as every
// ray's transmittance would fall below 1e-4 (block-wide vote).
//  - composite_rays_kernel (DirectL): one block per work item, i.e. up to
//    kRayThreads required rays of one (view, tile); each ray writes only the
//    subpixels it feeds (Sec. 4 step (3), the channel reorder folded in).
//  - composite_full_kernel (standard paradigm): one block per (view, tile),
//    one thread per pixel, every pixel of every view into M_m.
#include "dl_internal.cuh"

namespace dl {
namespace {

constexpr int kRayThreads = 128;

struct Acc {
    float T, c0, c1, c2;
    uint32_t blended;
};

// One record against one ray.  Returns false once the ray is finished.
// log2 alpha = A dx^2 + B dx dy + C dy^2 + log2 o; alpha = min(0.99, 2^that);
// skip alpha < 1/255; stop before T would drop below 1e-4.
__device__ __forceinline__ bool blend(Acc& a, float px, float py, const float4& q0,
                                      const float4& q1, float b) {
    const float dx = px - q0.x, dy = py - q0.y;
    const float l2 = fmaf(q0.z * dx, dx, fmaf(q0.w * dx, dy, fmaf(q1.x * dy, dy, q1.y)));
    const float alpha = fminf(0.99f, exp2f(l2));
    if (alpha < (1.0f / 255.0f)) return true;
    const float Tn = a.T * (1.f - alpha);
    if (Tn < 1e-4f) return false;
    const float w = alpha * a.T;
    a.c0 = fmaf(w, q1.z, a.c0);
    a.c1 = fmaf(w, q1.w, a.c1);
    a.c2 = fmaf(w, b, a.c2);
    a.T = Tn;
    ++a.blended;
    return true;
}

// Adds the block's evaluated and composited pair counts to pairs[0..1].
__device__ __forceinline__ void count_pairs(unsigned long long* pairs, uint32_t evals,
                                            uint32_t blended) {
    unsigned long long e = evals, b = blended;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(pairs, e);
        atomicAdd(pairs + 1, b);
    }
}

__global__ void __launch_bounds__(kRayThreads)
composite_rays_kernel(CompositeParams p, const int4* __restrict__ work,
                      const int4* __restrict__ grouped, const uint2* __restrict__ ranges,
                      const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                      float* __restrict__ out, unsigned long long* __restrict__ pairs) {
    __shared__ float4 s0[kRayThreads];
    __shared__ float4 s1[kRayThreads];
    __shared__ float s2[kRayThreads];
    const int4 wi = work[blockIdx.x];
    const int v = wi.x / p.ntiles;
    const int rid = wi.y + int(threadIdx.x);
    const bool active = rid < wi.z;
    const int4 ray = active ? grouped[rid] : make_int4(0, -1, -1, -1);
    const float px = float(uint32_t(ray.x) & 0xFFFFu) - p.half_w;
    const float py = float(uint32_t(ray.x) >> 16) - p.half_h;
    const uint2 rg = ranges[wi.x];
    const int64_t vbase = int64_t(v) * p.n;
    Acc a{1.f, 0.f, 0.f, 0.f, 0u};
    uint32_t evals = 0;
    bool done = !active;
    for (uint32_t b = rg.x; b < rg.y; b += kRayThreads) {
        const uint32_t i = b + threadIdx.x;
        if (i < rg.y) {
            const int64_t e = vbase + vals[i];
            s0[threadIdx.x] = rec[3 * e];
            s1[threadIdx.x] = rec[3 * e + 1];
            s2[threadIdx.x] = rec[3 * e + 2].x;
        }
        __syncthreads();
        const int nb = int(rg.y - b < kRayThreads ? rg.y - b : kRayThreads);
        if (!done) {
            int j = 0;
            for (; j < nb; ++j) {
                if (!blend(a, px, py, s0[j], s1[j], s2[j])) {
                    done = true;
                    ++j;
                    break;
                }
            }
            evals += uint32_t(j);
        }
        if (__syncthreads_count(done) == int(blockDim.x)) break;
    }
    if (pairs) count_pairs(pairs, evals, a.blended);
    if (active) {
        if (ray.y >= 0) out[ray.y] = a.c0;
        if (ray.z >= 0) out[ray.z] = a.c1;
        if (ray.w >= 0) out[ray.w] = a.c2;
    }
}

__global__ void composite_full_kernel(CompositeParams p, const uint2* __restrict__ ranges,
                                      const uint32_t* __restrict__ vals,
                                      const float4* __restrict__ rec, float* __restrict__ Mm,
                                      unsigned long long* __restrict__ pairs) {
    extern __shared__ float4 sm[];
    const int nthr = blockDim.x;
    float4* s0 = sm;
    float4* s1 = sm + nthr;
    float* s2 = reinterpret_cast<float*>(sm + 2 * nthr);
    const int group = blockIdx.x;
    const int v = group / p.ntiles;
    const int tile = group - v * p.ntiles;
    const int tx = tile % p.ntx, ty = tile / p.ntx;
    const int col = tx * p.tile_w + int(threadIdx.x) % p.tile_w;
    const int row = ty * p.tile_h + int(threadIdx.x) / p.tile_w;
    const bool inside = col < p.width && row < p.height;
    const float px = float(col) - p.half_w, py = float(row) - p.half_h;
    const uint2 rg = ranges[group];
    const int64_t vbase = int64_t(v) * p.n;
    Acc a{1.f, 0.f, 0.f, 0.f, 0u};
    uint32_t evals = 0;
    bool done = !inside;
    for (uint32_t b = rg.x; b < rg.y; b += nthr) {
        const uint32_t i = b + threadIdx.x;
        if (i < rg.y) {
            const int64_t e = vbase + vals[i];
            s0[threadIdx.x] = rec[3 * e];
            s1[threadIdx.x] = rec[3 * e + 1];
            s2[threadIdx.x] = rec[3 * e + 2].x;
        }
        __syncthreads();
        const int nb = int(rg.y - b < uint32_t(nthr) ? rg.y - b : uint32_t(nthr));
        if (!done) {
            int j = 0;
            for (; j < nb; ++j) {
                if (!blend(a, px, py, s0[j], s1[j], s2[j])) {
                    done = true;
                    ++j;
                    break;
                }
            }
            evals += uint32_t(j);
        }
        if (__syncthreads_count(done) == nthr) break;
    }
    if (pairs) count_pairs(pairs, evals, a.blended);
    if (inside) {
        float* o = Mm + ((int64_t(v) * p.height + row) * p.width + col) * 3;
        o[0] = a.c0;
        o[1] = a.c1;
        o[2] = a.c2;
    }
}

// M_e[x, y, k] = M_m[V(x, 3y + k), x, y, k] (Alg. 1, native resolution).
__global__ void interweave_kernel(int32_t w, int32_t h, const uint16_t* __restrict__ V,
                                  const float* __restrict__ Mm, float* __restrict__ out) {
    const int64_t S = 3 * int64_t(w);
    const int64_t total = S * h;
    const int64_t plane = int64_t(h) * w * 3;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t x = i / S;
        const int64_t rem = i - x * S;
        out[i] = Mm[int64_t(V[i]) * plane + x * S + rem];
    }
}

}  // namespace

cudaError_t launch_composite_rays(const CompositeParams& p, const int4* work, int64_t n_work,
                                  const int4* grouped, const uint2* ranges, const uint32_t* vals,
                                  const float4* rec, float* out, unsigned long long* pairs,
                                  cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    composite_rays_kernel<<<unsigned(n_work), kRayThreads, 0, s>>>(p, work, grouped, ranges, vals,
                                                                   rec, out, pairs);
    return cudaGetLastError();
}

cudaError_t launch_composite_full(const CompositeParams& p, int32_t nv, const uint2* ranges,
                                  const uint32_t* vals, const float4* rec, float* Mm,
                                  unsigned long long* pairs, cudaStream_t s) {
    const int nthr = p.tile_w * p.tile_h;
    const size_t smem = size_t(nthr) * (2 * sizeof(float4) + sizeof(float));
    const int64_t blocks = int64_t(nv) * p.ntiles;
    composite_full_kernel<<<unsigned(blocks), nthr, smem, s>>>(p, ranges, vals, rec, Mm, pairs);
    return cudaGetLastError();
}

cudaError_t launch_interweave(int32_t w, int32_t h, int32_t nv, const uint16_t* V, const float* Mm,
                              float* out, cudaStream_t s) {
    (void)nv;
    const int64_t total = 3 * int64_t(w) * h;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    interweave_kernel<<<unsigned(grid), 256, 0, s>>>(w, h, V, Mm, out);
    return cudaGetLastError();
}

}  // namespace dl
