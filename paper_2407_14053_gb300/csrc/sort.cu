// Device-wide exclusive scan and a stable LSD radix sort of (u64 key, u32
// value) pairs, used to order tile keys by (view, tile, depth) (the depth sort
// of Sec. 3.3 / Sec. 7 step 3) and rays by compositing tile.
//
// Radix sort, per 8-bit digit pass, over a fixed grid of G blocks that each
// own one contiguous chunk of the input:
//   upsweep   -- per-block digit histogram, written digit-major [256][G];
//   scan      -- one block turns the histogram into global start offsets;
//   downsweep -- each block walks its chunk in tiles of 256 x ITEMS keys,
//                ranks keys stably inside the tile (warp match + per-warp
//                digit counters), stages the tile digit-sorted in shared
//                memory and writes each digit's run contiguously.
#include "dl_internal.cuh"

namespace dl {

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over a block of up to 1024 threads.
// Returns the exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t x = lane < nw ? s_w[lane] : 0;
        const uint32_t xi = warp_incl_scan(x);
        if (lane < nw) s_w[lane] = xi - x;
        if (lane == 31) s_total = xi;  // inclusive sum over every warp
    }
    __syncthreads();
    const uint32_t res = s_w[wid] + inc - v;
    if (total) *total = s_total;
    __syncthreads();
    return res;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                   uint32_t* __restrict__ bsum) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile;
    uint32_t s = 0;
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in one block; writes the grand total.
__global__ void scan_blocks_kernel(uint32_t* __restrict__ bsum, int64_t nb,
                                   uint32_t* __restrict__ d_total) {
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b0; i < b0 + per && i < nb; ++i) s += bsum[i];
    uint32_t tot;
    uint32_t run = block_excl_scan(s, &tot);
    for (int64_t i = b0; i < b0 + per && i < nb; ++i) {
        const uint32_t v = bsum[i];
        bsum[i] = run;
        run += v;
    }
    if (threadIdx.x == 0 && d_total) *d_total = tot;
}

__global__ void scan_apply_kernel(const uint32_t* __restrict__ in, int64_t n,
                                  const uint32_t* __restrict__ bsum, uint32_t* __restrict__ out) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        v[j] = i < n ? in[i] : 0;
        s += v[j];
    }
    uint32_t run = block_excl_scan(s, nullptr) + bsum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}

// ---------------------------------------------------------------- radix ----
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 12;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kBins = 256;

__global__ void __launch_bounds__(kRadixThreads)
radix_upsweep_kernel(const unsigned long long* __restrict__ keys, int64_t n, int64_t chunk,
                     int shift, uint32_t mask, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRadixWarps][kBins];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * kBins; i += kRadixThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t beg = int64_t(blockIdx.x) * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    for (int64_t i0 = beg; i0 < end; i0 += kRadixThreads) {
        const int64_t i = i0 + threadIdx.x;
        const bool ok = i < end;
        const uint32_t d = ok ? uint32_t(keys[i] >> shift) & mask : 0xFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & ((1u << lane) - 1)) == 0) atomicAdd(&h[wid][d], __popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kRadixThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) s += h[w][d];
        hist[int64_t(d) * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void radix_scan_kernel(uint32_t* __restrict__ hist, int64_t total) {
    const int64_t per = (total + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b0; i < b0 + per && i < total; ++i) s += hist[i];
    uint32_t run = block_excl_scan(s, nullptr);
    for (int64_t i = b0; i < b0 + per && i < total; ++i) {
        const uint32_t v = hist[i];
        hist[i] = run;
        run += v;
    }
}

struct RadixSmem {
    uint32_t wcnt[kRadixWarps][kBins];
    uint32_t lbase[kBins];
    uint32_t gbase[kBins];
    uint32_t tot[kBins];
    unsigned long long k[kRadixTile];
    uint32_t v[kRadixTile];
};

__global__ void __launch_bounds__(kRadixThreads)
radix_downsweep_kernel(const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
                       unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout,
                       int64_t n, int64_t chunk, int shift, uint32_t mask,
                       const uint32_t* __restrict__ hist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RadixSmem& S = *reinterpret_cast<RadixSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1;
    for (int d = threadIdx.x; d < kBins; d += kRadixThreads)
        S.gbase[d] = hist[int64_t(d) * gridDim.x + blockIdx.x];
    const int64_t beg = int64_t(blockIdx.x) * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    for (int64_t t0 = beg; t0 < end; t0 += kRadixTile) {
        const int cnt = int(end - t0 < kRadixTile ? end - t0 : kRadixTile);
        for (int d = lane; d < kBins; d += 32) S.wcnt[wid][d] = 0;
        __syncwarp();
        unsigned long long k[kRadixItems];
        uint32_t v[kRadixItems], rk[kRadixItems];
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            const int idx = wid * (32 * kRadixItems) + j * 32 + lane;
            const bool ok = idx < cnt;
            k[j] = ok ? kin[t0 + idx] : 0ull;
            v[j] = ok ? vin[t0 + idx] : 0u;
            const uint32_t d = ok ? uint32_t(k[j] >> shift) & mask : 0xFFFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t base = ok ? S.wcnt[wid][d] : 0u;
            __syncwarp();
            if (ok && (peers & lt_mask) == 0) S.wcnt[wid][d] = base + __popc(peers);
            __syncwarp();
            rk[j] = base + __popc(peers & lt_mask);
        }
        __syncthreads();
        {   // per digit: warp-exclusive prefixes and tile total
            const int d = threadIdx.x;  // kRadixThreads == kBins
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) {
                const uint32_t c = S.wcnt[w][d];
                S.wcnt[w][d] = s;
                s += c;
            }
            S.tot[d] = s;
            const uint32_t lb = block_excl_scan(s, nullptr);
            S.lbase[d] = lb;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRadixItems; ++j) {
            const int idx = wid * (32 * kRadixItems) + j * 32 + lane;
            if (idx < cnt) {
                const uint32_t d = uint32_t(k[j] >> shift) & mask;
                const uint32_t pos = S.lbase[d] + S.wcnt[wid][d] + rk[j];
                S.k[pos] = k[j];
                S.v[pos] = v[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
            const unsigned long long key = S.k[i];
            const uint32_t d = uint32_t(key >> shift) & mask;
            const int64_t g = int64_t(S.gbase[d]) + (i - int64_t(S.lbase[d]));
            kout[g] = key;
            vout[g] = S.v[i];
        }
        __syncthreads();
        S.gbase[threadIdx.x] += S.tot[threadIdx.x];
        __syncthreads();
    }
}

__global__ void key_ranges_kernel(const unsigned long long* __restrict__ keys, int64_t n,
                                  int shift, uint2* __restrict__ ranges, int64_t n_groups) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long g = keys[i] >> shift;
        if (g >= (unsigned long long)n_groups) continue;  // never produced; not followed
        if (i == 0 || (keys[i - 1] >> shift) != g) ranges[g].x = uint32_t(i);
        if (i == n - 1 || (keys[i + 1] >> shift) != g) ranges[g].y = uint32_t(i + 1);
    }
}

int radix_grid(int64_t n, int64_t* chunk) {
    const int64_t tiles = (n + kRadixTile - 1) / kRadixTile;
    int64_t G = int64_t(num_sms()) * 4;
    if (G > tiles) G = tiles;
    if (G < 1) G = 1;
    const int64_t tiles_per = (tiles + G - 1) / G;
    *chunk = tiles_per * kRadixTile;
    G = (n + *chunk - 1) / *chunk;
    return int(G < 1 ? 1 : G);
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    return size_t(nb + 1) * sizeof(uint32_t) + 256;
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                                  void* tmp, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    uint32_t* bsum = static_cast<uint32_t*>(tmp);
    scan_reduce_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, bsum);
    scan_blocks_kernel<<<1, 1024, 0, s>>>(bsum, nb, d_total);
    scan_apply_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, bsum, out);
    return cudaGetLastError();
}

size_t radix_tmp_bytes(int64_t n) {
    int64_t chunk;
    const int G = radix_grid(n > 0 ? n : 1, &chunk);
    return size_t(kBins) * G * sizeof(uint32_t) + 256;
}

cudaError_t radix_sort_pairs(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* tmp,
                             int* result_in_alt, cudaStream_t s) {
    *result_in_alt = 0;
    if (n <= 1 || bits <= 0) return cudaSuccess;
    static bool attr_set = false;
    const size_t smem = sizeof(RadixSmem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(radix_downsweep_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int64_t chunk;
    const int G = radix_grid(n, &chunk);
    uint32_t* hist = static_cast<uint32_t*>(tmp);
    unsigned long long *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    int flips = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        const int nb = bits - shift < 8 ? bits - shift : 8;
        const uint32_t mask = (1u << nb) - 1u;
        radix_upsweep_kernel<<<G, kRadixThreads, 0, s>>>(ki, n, chunk, shift, mask, hist);
        radix_scan_kernel<<<1, 1024, 0, s>>>(hist, int64_t(kBins) * G);
        radix_downsweep_kernel<<<G, kRadixThreads, smem, s>>>(ki, vi, ko, vo, n, chunk, shift, mask,
                                                               hist);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
        flips ^= 1;
    }
    *result_in_alt = flips;
    return cudaSuccess;
}

cudaError_t launch_key_ranges(const unsigned long long* keys, int64_t n, int shift, uint2* ranges,
                              int64_t n_groups, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    key_ranges_kernel<<<unsigned(grid), 256, 0, s>>>(keys, n, shift, ranges, n_groups);
    return cudaGetLastError();
}

}  // namespace dl
