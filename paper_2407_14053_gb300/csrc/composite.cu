// Front-to-back alpha compositing (Sec. 3.2 Eq. (5), Sec. 3.3 Eq. (10)) and
// the standard paradigm's interweave (Alg. 1).
//
// Both compositing kernels stream one (view, tile) list of depth-sorted
// Gaussian records through shared memory in batches.  Each warp first tests
// 32 records at a time against the bounding box of its own rays (one ballot)
// and then composites only the records whose alpha >= 1/255 box touches it,
// in list order, so the per-ray sequence of composited Gaussians is exactly
// the depth-sorted one.  A block stops once every ray's transmittance would
// fall below 1e-4 (block-wide vote).
//  - composite_rays_kernel (DirectL): one block per work item, i.e. up to
//    kRayThreads required rays of one (view, tile), ordered along a Morton
//    curve so that a warp's rays are close together; each ray writes its
//    colour, and reorder_kernel gathers the encoded image by the ray table
//    (Sec. 4 step (3): the channel reorder by precomputed indices).
//  - composite_full_kernel (standard paradigm): one block per (view, tile),
//    one thread per pixel, every pixel of every view into M_m.
#include <climits>

#include "dl_internal.cuh"

namespace dl {
namespace {

constexpr int kRayThreads = 128;
constexpr float kLog2MinAlpha = -7.99435343685886f;  // log2(1/255)

struct Acc {
    float T, c0, c1, c2;
    uint32_t blended;
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Asynchronous 16-byte global -> shared copies (Ampere-and-later cp.async),
// used to fetch the next batch of records while the current one is blended.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// log2 alpha = A dx^2 + B dx dy + C dy^2 + log2 o at pixel offset (dx, dy)
// from the record's mean.  Every caller evaluates exactly this expression, so
// a pre-test and the blend below always agree bit for bit.
__device__ __forceinline__ float log2_alpha(float px, float py, float u, float v, float A, float B,
                                            float C, float L) {
    const float dx = px - u, dy = py - v;
    return fmaf(dx, fmaf(A, dx, B * dy), fmaf(C * dy, dy, L));
}

// One record against one ray.  Returns false once the ray is finished.
// alpha = min(0.99, 2^log2_alpha); skip alpha < 1/255 (CHECK_L2: tested
// first on log2 alpha, which spares the ex2 for records that miss the ray,
// then on alpha itself); stop before T (1 - alpha) = T - alpha T would drop
// below 1e-4.  After the log2 test the steps are selects, not branches: a
// skipped record adds 0 alpha T = 0 to the colour and leaves T (>= 1e-4) as
// it is.  COUNT keeps the composited-pair statistic.  The colour is
// (q1.z, q1.w, b): kernels that load a batch thread by thread decode the
// packed colour once per record when they store it in shared memory (the
// standard paradigm blends tens of times per record); blend_rec below takes
// a record as stored.
template <bool CHECK_L2 = true, bool COUNT = true>
__device__ __forceinline__ bool blend(Acc& a, float px, float py, const float4& q0,
                                      const float4& q1, float b) {
    const float l2 = log2_alpha(px, py, q0.x, q0.y, q0.z, q0.w, q1.x, q1.y);
    if (CHECK_L2 && l2 < kLog2MinAlpha) return true;
    float alpha = fminf(0.99f, ex2_approx(l2));
    alpha = alpha < (1.0f / 255.0f) ? 0.f : alpha;
    const float w0 = alpha * a.T;
    const float Tn = a.T - w0;
    const bool go = Tn >= 1e-4f;
    const float w = go ? w0 : 0.f;
    a.c0 = fmaf(w, q1.z, a.c0);
    a.c1 = fmaf(w, q1.w, a.c1);
    a.c2 = fmaf(w, b, a.c2);
    a.T = go ? Tn : a.T;
    if (COUNT && go && alpha > 0.f) ++a.blended;
    return go;
}

// blend() on a record as the projection stored it (packed colour).
template <bool CHECK_L2 = true, bool COUNT = true>
__device__ __forceinline__ bool blend_rec(Acc& a, float px, float py, const float4& q0,
                                          const float4& q1) {
    float r, g, b;
    unpack_rgb(q1.z, q1.w, r, g, b);
    return blend<CHECK_L2, COUNT>(a, px, py, q0, make_float4(q1.x, q1.y, r, g), b);
}

// blend() of two candidates in list order, their alphas formed together
// (`two` false: the second is none).  The arithmetic and its order are
// blend()'s on each candidate in turn; false once the ray is finished.
template <bool COUNT>
__device__ __forceinline__ bool blend2(Acc& a, float px, float py, const float4& p0,
                                       const float4& p1, float pb, const float4& q0,
                                       const float4& q1, float qb, bool two) {
    const float la = log2_alpha(px, py, p0.x, p0.y, p0.z, p0.w, p1.x, p1.y);
    const float lb = log2_alpha(px, py, q0.x, q0.y, q0.z, q0.w, q1.x, q1.y);
    float alpha_a = fminf(0.99f, ex2_approx(la));
    float alpha_b = fminf(0.99f, ex2_approx(lb));
    alpha_a = alpha_a < (1.0f / 255.0f) ? 0.f : alpha_a;
    alpha_b = (alpha_b < (1.0f / 255.0f) || !two) ? 0.f : alpha_b;
    const float wa0 = alpha_a * a.T;
    const float Ta = a.T - wa0;
    const bool goa = Ta >= 1e-4f;
    const float wa = goa ? wa0 : 0.f;
    a.c0 = fmaf(wa, p1.z, a.c0);
    a.c1 = fmaf(wa, p1.w, a.c1);
    a.c2 = fmaf(wa, pb, a.c2);
    a.T = goa ? Ta : a.T;
    const float wb0 = alpha_b * a.T;
    const float Tb = a.T - wb0;
    const bool gob = goa && Tb >= 1e-4f;
    const float wb = gob ? wb0 : 0.f;
    a.c0 = fmaf(wb, q1.z, a.c0);
    a.c1 = fmaf(wb, q1.w, a.c1);
    a.c2 = fmaf(wb, qb, a.c2);
    a.T = gob ? Tb : a.T;
    if (COUNT) a.blended += (goa && alpha_a > 0.f) + (gob && alpha_b > 0.f);
    return gob;
}

// A record and its pixel box in the shared-memory layout of the batch
// loaders: s0 = (u, v, A, B), s1 = (C, L, r, g), s2 = (b, -, rect_c, rect_r).
__device__ __forceinline__ void store_decoded(const float4& q0, const float4& q1, uint2 rect,
                                              float4& s0, float4& s1, float4& s2) {
    float r, g, b;
    unpack_rgb(q1.z, q1.w, r, g, b);
    s0 = q0;
    s1 = make_float4(q1.x, q1.y, r, g);
    s2 = make_float4(b, 0.f, __uint_as_float(rect.x), __uint_as_float(rect.y));
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

// Transposed evaluation of up to 32 records (indices wbuf[0..n)) for the
// warp's rays: each lane holds one record, tests it against every ray that is
// still compositing (ray position by shuffle, one ballot per ray), and keeps
// the mask of records that may reach alpha >= 1/255 for its own ray.  Then
// every lane blends its own candidates in list order.  Finished rays drop out
// of the ray loop, so they cost nothing.
__device__ __forceinline__ void warp_group(Acc& a, bool& done, uint32_t& evals, float px, float py,
                                           const int* wbuf, int n, const float4* s0,
                                           const float4* s1, const float4* s2) {
    const int lane = threadIdx.x & 31;
    const int j = lane < n ? wbuf[lane] : -1;
    float u = 0.f, v = 0.f, A = 0.f, B = 0.f, C = 0.f, L = -1e30f;
    if (j >= 0) {
        const float4 q0 = s0[j];
        const float2 q1 = *reinterpret_cast<const float2*>(s1 + j);
        u = q0.x; v = q0.y; A = q0.z; B = q0.w; C = q1.x; L = q1.y;
    }
    unsigned act = __ballot_sync(0xffffffffu, !done);
    unsigned mine = 0;
    while (act) {
        const int r = __ffs(act) - 1;
        act &= act - 1;
        const float rx = __shfl_sync(0xffffffffu, px, r);
        const float ry = __shfl_sync(0xffffffffu, py, r);
        const bool pass = log2_alpha(rx, ry, u, v, A, B, C, L) >= kLog2MinAlpha;
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (lane == r) mine = m;
    }
    if (!done) evals += uint32_t(n);
    while (mine && !done) {
        const int sidx = __ffs(mine) - 1;
        mine &= mine - 1;
        const int jj = wbuf[sidx];
        if (!blend(a, px, py, s0[jj], s1[jj], s2[jj].x)) done = true;
    }
}

// Composites a shared-memory batch of nb records for this lane's ray.  Records
// whose pixel box misses the warp's box [bx0,bx1] x [by0,by1] are dropped; the
// rest are compacted, in list order, into the warp's buffer (64 ints) and
// evaluated 32 at a time.
__device__ __forceinline__ void warp_batch(Acc& a, bool& done, uint32_t& evals, float px, float py,
                                           int bx0, int bx1, int by0, int by1, const float4* s0,
                                           const float4* s1, const float4* s2, int nb, int* wbuf) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1;
    int cnt = 0;
    for (int j0 = 0; j0 < nb; j0 += 32) {
        if (__all_sync(0xffffffffu, done)) return;
        bool hit = false;
        if (j0 + lane < nb) {
            const float4 q2 = s2[j0 + lane];
            const uint32_t rc = __float_as_uint(q2.z), rr = __float_as_uint(q2.w);
            hit = int(rc & 0xFFFFu) <= bx1 && int(rc >> 16) >= bx0 && int(rr & 0xFFFFu) <= by1 &&
                  int(rr >> 16) >= by0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) wbuf[cnt + __popc(m & lt)] = j0 + lane;
        cnt += __popc(m);
        __syncwarp();
        if (cnt >= 32) {
            warp_group(a, done, evals, px, py, wbuf, 32, s0, s1, s2);
            __syncwarp();
            const int rest = cnt - 32;
            const int t = lane < rest ? wbuf[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) wbuf[lane] = t;
            __syncwarp();
            cnt = rest;
        }
    }
    if (cnt > 0 && !__all_sync(0xffffffffu, done)) {
        warp_group(a, done, evals, px, py, wbuf, cnt, s0, s1, s2);
    }
    __syncwarp();
}

// Direct evaluation: every lane walks the culled records in list order and
// evaluates each one for its own ray (record fields by shared-memory broadcast).
__device__ __forceinline__ void warp_batch_direct(Acc& a, bool& done, uint32_t& evals, float px,
                                                  float py, int bx0, int bx1, int by0, int by1,
                                                  const float4* s0, const float4* s1,
                                                  const float4* s2, int nb) {
    const int lane = threadIdx.x & 31;
    for (int j0 = 0; j0 < nb; j0 += 32) {
        if (__all_sync(0xffffffffu, done)) return;
        bool hit = false;
        if (j0 + lane < nb) {
            const float4 q2 = s2[j0 + lane];
            const uint32_t rc = __float_as_uint(q2.z), rr = __float_as_uint(q2.w);
            hit = int(rc & 0xFFFFu) <= bx1 && int(rc >> 16) >= bx0 && int(rr & 0xFFFFu) <= by1 &&
                  int(rr >> 16) >= by0;
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        while (m) {
            const int j = j0 + __ffs(m) - 1;
            m &= m - 1;
            if (!done) {
                ++evals;
                if (!blend(a, px, py, s0[j], s1[j], s2[j].x)) done = true;
            }
        }
    }
}

template <bool TRANSPOSED>
__device__ __forceinline__ void eval_batch(Acc& a, bool& done, uint32_t& evals, float px, float py,
                                           int bx0, int bx1, int by0, int by1, const float4* s0,
                                           const float4* s1, const float4* s2, int nb, int* wbuf) {
    if (TRANSPOSED)
        warp_batch(a, done, evals, px, py, bx0, bx1, by0, by1, s0, s1, s2, nb, wbuf);
    else
        warp_batch_direct(a, done, evals, px, py, bx0, bx1, by0, by1, s0, s1, s2, nb);
}

__device__ __forceinline__ void warp_box(bool active, int col, int row, int& bx0, int& bx1, int& by0,
                                         int& by1) {
    bx0 = __reduce_min_sync(0xffffffffu, active ? col : INT_MAX);
    bx1 = __reduce_max_sync(0xffffffffu, active ? col : INT_MIN);
    by0 = __reduce_min_sync(0xffffffffu, active ? row : INT_MAX);
    by1 = __reduce_max_sync(0xffffffffu, active ? row : INT_MIN);
}

__global__ void __launch_bounds__(kRayThreads)
composite_rays_kernel(CompositeParams p, const int4* __restrict__ work,
                      const int2* __restrict__ grouped, const uint2* __restrict__ ranges,
                      const uint32_t* __restrict__ vals, const float4* __restrict__ rec,
                      float* __restrict__ raycol, unsigned long long* __restrict__ pairs) {
    __shared__ float4 s0[kRayThreads];
    __shared__ float4 s1[kRayThreads];
    __shared__ float4 s2[kRayThreads];
    const int4 wi = work[blockIdx.x];
    const int v = wi.x / p.ntiles;
    const int rid = wi.y + int(threadIdx.x);
    const bool active = rid < wi.z;
    const int2 ray = active ? grouped[rid] : make_int2(0, -1);
    const int col = int(uint32_t(ray.x) & 0xFFFFu), row = int(uint32_t(ray.x) >> 16);
    const float px = float(col) - p.half_w;
    const float py = float(row) - p.half_h;
    int bx0, bx1, by0, by1;
    warp_box(active, col, row, bx0, bx1, by0, by1);
    const uint2 rg = ranges[wi.x];
    const int64_t vbase = int64_t(v) * p.n;
    Acc a{1.f, 0.f, 0.f, 0.f, 0u};
    uint32_t evals = 0;
    bool done = !active;
    for (uint32_t b = rg.x; b < rg.y; b += kRayThreads) {
        const uint32_t i = b + threadIdx.x;
        if (i < rg.y) {
            const int64_t e = vbase + vals[i];
            const float4 q0 = rec[kRecordFloat4 * e], q1 = rec[kRecordFloat4 * e + 1];
            const uint4 m = p.meta[e];
            store_decoded(q0, q1, make_uint2(m.x, m.y), s0[threadIdx.x], s1[threadIdx.x],
                          s2[threadIdx.x]);
        }
        __syncthreads();
        const int nb = int(rg.y - b < kRayThreads ? rg.y - b : kRayThreads);
        warp_batch_direct(a, done, evals, px, py, bx0, bx1, by0, by1, s0, s1, s2, nb);
        if (__syncthreads_count(done) == int(blockDim.x)) break;
    }
    if (pairs) count_pairs(pairs, evals, a.blended);
    if (active) {
        float* o = raycol + 3 * int64_t(rid);  // grouped order
        o[0] = a.c0;
        o[1] = a.c1;
        o[2] = a.c2;
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
    float4* s2 = sm + 2 * nthr;
    const int group = blockIdx.x;
    const int v = group / p.ntiles;
    const int tile = group - v * p.ntiles;
    const int tx = tile % p.ntx, ty = tile / p.ntx;
    const int col = tx * p.tile_w + int(threadIdx.x) % p.tile_w;
    const int row = ty * p.tile_h + int(threadIdx.x) / p.tile_w;
    const bool inside = col < p.width && row < p.height;
    const float px = float(col) - p.half_w, py = float(row) - p.half_h;
    int bx0, bx1, by0, by1;
    warp_box(inside, col, row, bx0, bx1, by0, by1);
    const uint2 rg = ranges[group];
    const int64_t vbase = int64_t(v) * p.n;
    Acc a{1.f, 0.f, 0.f, 0.f, 0u};
    uint32_t evals = 0;
    bool done = !inside;
    for (uint32_t b = rg.x; b < rg.y; b += nthr) {
        const uint32_t i = b + threadIdx.x;
        if (i < rg.y) {
            const int64_t e = vbase + vals[i];
            const float4 q0 = rec[kRecordFloat4 * e], q1 = rec[kRecordFloat4 * e + 1];
            const uint4 m = p.meta[e];
            store_decoded(q0, q1, make_uint2(m.x, m.y), s0[threadIdx.x], s1[threadIdx.x],
                          s2[threadIdx.x]);
        }
        __syncthreads();
        const int nb = int(rg.y - b < uint32_t(nthr) ? rg.y - b : uint32_t(nthr));
        warp_batch_direct(a, done, evals, px, py, bx0, bx1, by0, by1, s0, s1, s2, nb);
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

// ---------------------------------------------------------- binned path ---
// Ascending bitonic sort of P (a power of two) unique keys in shared memory.
__device__ void bitonic_sort(unsigned long long* s, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
                const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const int hi = lo + j;
                const bool up = (lo & k) == 0;
                const unsigned long long a = s[lo], b = s[hi];
                if ((a > b) == up) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Exclusive scan, in place, of n <= blockDim.x * 64 counters in shared memory.
__device__ void block_scan_counts(uint32_t* c, int n) {
    __shared__ uint32_t s_w[32];
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int per = (n + nthr - 1) / nthr;
    const int b0 = tid * per;
    uint32_t sum = 0;
    for (int i = b0; i < b0 + per && i < n; ++i) sum += c[i];
    const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t x = lane < nw ? s_w[lane] : 0;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) s_w[lane] = xi - x;
    }
    __syncthreads();
    uint32_t run = s_w[wid] + inc - sum;
    for (int i = b0; i < b0 + per && i < n; ++i) {
        const uint32_t v = c[i];
        c[i] = run;
        run += v;
    }
    __syncthreads();
}

// largest bucket sorted inside its list (by one thread in the block sort, by
// odd-even phases in the warp sort); a larger one sends the list to a bitonic sort
constexpr int kBucketSortLimit = 64;

// Sorts the group's keys (depth << 32 | Gaussian, all distinct) into sk:
// a counting sort on the depth bucket floor((d - dmin) NB / (dmax - dmin + 1))
// (monotone in d), then an insertion sort inside every bucket.  If a bucket
// holds more than kBucketSortLimit keys (many equal depths), the whole list
// is bitonic-sorted instead.  KPT > 0: the block holds the keys in registers
// (len <= KPT * blockDim.x, one coalesced load); KPT == 0: the keys are read
// from global memory once per pass.  sk holds next_pow2(len) keys; cnt holds
// cap + 2 counters, cap >= len being the class capacity (a power of two).
template <int KPT>
__device__ void block_sort(const unsigned long long* __restrict__ keys, uint32_t start, int len,
                           int cap, unsigned long long* sk, uint32_t* cnt) {
    __shared__ uint32_t s_lo, s_hi, s_big;
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr int R = KPT > 0 ? KPT : 1;
    unsigned long long kr[R];
    if (tid == 0) {
        s_lo = 0xFFFFFFFFu;
        s_hi = 0u;
        s_big = 0u;
    }
    __syncthreads();
    if (len <= 1) {
        if (len == 1 && tid == 0) sk[0] = keys[start];
        __syncthreads();
        return;
    }
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    if (KPT > 0) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = j * nthr + tid;
            kr[j] = i < len ? keys[start + i] : ~0ull;
            if (i < len) {
                lo = min(lo, uint32_t(kr[j] >> 32));
                hi = max(hi, uint32_t(kr[j] >> 32));
            }
        }
    } else {
        for (int i = tid; i < len; i += nthr) {
            const uint32_t d = uint32_t(keys[start + i] >> 32);
            lo = min(lo, d);
            hi = max(hi, d);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((tid & 31) == 0) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    int NB = 1;
    while (NB < len) NB <<= 1;
    NB = NB >> 1;
    if (NB > cap / 2) NB = cap / 2;
    if (NB < 1) NB = 1;
    uint32_t* bstart = cnt;               // NB + 1
    uint32_t* bfill = cnt + cap / 2 + 1;  // NB
    for (int i = tid; i <= NB; i += nthr) bstart[i] = 0u;
    for (int i = tid; i < NB; i += nthr) bfill[i] = 0u;
    __syncthreads();
    const uint32_t dmin = s_lo;
    const float scale = float(NB) / (float(s_hi - s_lo) + 1.0f);
    auto bucket = [&](unsigned long long k) {
        return min(NB - 1, int(float(uint32_t(k >> 32) - dmin) * scale));
    };
    if (KPT > 0) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (j * nthr + tid < len) atomicAdd(&bstart[bucket(kr[j])], 1u);
    } else {
        for (int i = tid; i < len; i += nthr) atomicAdd(&bstart[bucket(keys[start + i])], 1u);
    }
    __syncthreads();
    block_scan_counts(bstart, NB);
    if (tid == 0) bstart[NB] = uint32_t(len);
    __syncthreads();
    if (KPT > 0) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            if (j * nthr + tid < len) {
                const int b = bucket(kr[j]);
                sk[bstart[b] + atomicAdd(&bfill[b], 1u)] = kr[j];
            }
    } else {
        for (int i = tid; i < len; i += nthr) {
            const unsigned long long k = keys[start + i];
            const int b = bucket(k);
            sk[bstart[b] + atomicAdd(&bfill[b], 1u)] = k;
        }
    }
    __syncthreads();
    for (int b = tid; b < NB; b += nthr)
        if (bstart[b + 1] - bstart[b] > uint32_t(kBucketSortLimit)) s_big = 1u;
    __syncthreads();
    if (s_big) {
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = len + tid; i < P; i += nthr) sk[i] = ~0ull;
        __syncthreads();
        bitonic_sort(sk, P);
    } else {
        for (int b = tid; b < NB; b += nthr) {
            const int b0 = int(bstart[b]), b1 = int(bstart[b + 1]);
            for (int i = b0 + 1; i < b1; ++i) {
                const unsigned long long k = sk[i];
                int j = i - 1;
                while (j >= b0 && sk[j] > k) {
                    sk[j + 1] = sk[j];
                    --j;
                }
                sk[j + 1] = k;
            }
        }
        __syncthreads();
    }
}

// Streams the sorted list's records through two shared-memory batches of
// blockDim.x records (cp.async prefetch of batch b+1 while batch b is
// blended) until every ray of the block is finished.
template <bool TRANSPOSED>
__device__ __forceinline__ void stream_list(const CompositeParams& p, const unsigned long long* sk,
                                            int len, int64_t vbase, const float4* __restrict__ rec,
                                            float4* buf, int* wbuf, Acc& a, bool& done,
                                            uint32_t& evals, float px, float py, int bx0, int bx1,
                                            int by0, int by1) {
    const int nthr = blockDim.x, t = threadIdx.x;
    // single shared batch: load (the record and, from the tile metadata, its
    // pixel box), barrier, blend, vote
    for (int b = 0; b < len; b += nthr) {
        const int i = b + t;
        if (i < len) {
            const int64_t e = vbase + (uint32_t(sk[i]) >> 4);
            const float4 q0 = rec[kRecordFloat4 * e], q1 = rec[kRecordFloat4 * e + 1];
            const uint4 m = p.meta[e];
            store_decoded(q0, q1, make_uint2(m.x, m.y), buf[t], buf[nthr + t], buf[2 * nthr + t]);
        }
        __syncthreads();
        const int nb = len - b < nthr ? len - b : nthr;
        eval_batch<TRANSPOSED>(a, done, evals, px, py, bx0, bx1, by0, by1, buf, buf + nthr,
                               buf + 2 * nthr, nb, wbuf);
        if (__syncthreads_count(done) == nthr) break;
    }
}

// Shared memory of a binned block: keys (cap), bucket counters (cap + 2),
// a record batch (3 x nthr float4), compaction buffers (64 ints per warp).
struct BinnedSmem {
    unsigned long long* sk;
    uint32_t* cnt;
    float4* buf;
    int* wbuf;
};

// Bytes of the key array (cap keys) and the bucket counters (cap + 2) of
// block_sort, rounded up to 16.
__host__ __device__ __forceinline__ size_t block_sort_bytes(int cap) {
    return (8 * size_t(cap) + 4 * size_t(cap + 2) + 15) & ~size_t(15);
}

__device__ __forceinline__ BinnedSmem carve_binned(unsigned char* base, int cap, int nthr) {
    BinnedSmem m;
    m.sk = reinterpret_cast<unsigned long long*>(base);
    m.cnt = reinterpret_cast<uint32_t*>(base + 8 * size_t(cap));
    const size_t off = (8 * size_t(cap) + 4 * size_t(cap + 2) + 15) & ~size_t(15);
    m.buf = reinterpret_cast<float4*>(base + off);
    m.wbuf = reinterpret_cast<int*>(m.buf + 3 * nthr) + 64 * (threadIdx.x >> 5);
    return m;
}

template <bool TRANSPOSED, int KPT>
__global__ void __launch_bounds__(kBinnedThreads)
composite_rays_binned_kernel(CompositeParams p, const int4* __restrict__ gwork,
                             const int32_t* __restrict__ list, int cap,
                             const int2* __restrict__ grouped, const uint32_t* __restrict__ gstart,
                             const unsigned long long* __restrict__ keys,
                             const float4* __restrict__ rec, float* __restrict__ raycol,
                             unsigned long long* __restrict__ pairs) {
    extern __shared__ __align__(16) unsigned char smb[];
    const int nthr = blockDim.x;
    const BinnedSmem S = carve_binned(smb, cap, nthr);
    const int4 wi = gwork[list[blockIdx.x]];
    const int v = wi.x / p.ntiles;
    const uint32_t start = gstart[wi.x];
    const int len = int(gstart[wi.x + 1] - start);
    block_sort<KPT>(keys, start, len, cap, S.sk, S.cnt);
    const int64_t vbase = int64_t(v) * p.n;
    uint32_t evals = 0, blended = 0;
    for (int r0 = wi.y; r0 < wi.z; r0 += nthr) {
        const int rid = r0 + int(threadIdx.x);
        const bool active = rid < wi.z;
        const int2 ray = active ? grouped[rid] : make_int2(0, -1);
        const int col = int(uint32_t(ray.x) & 0xFFFFu), row = int(uint32_t(ray.x) >> 16);
        const float px = float(col) - p.half_w, py = float(row) - p.half_h;
        int bx0, bx1, by0, by1;
        warp_box(active, col, row, bx0, bx1, by0, by1);
        Acc a{1.f, 0.f, 0.f, 0.f, 0u};
        bool done = !active;
        stream_list<TRANSPOSED>(p, S.sk, len, vbase, rec, S.buf, S.wbuf, a, done, evals, px, py,
                                bx0, bx1, by0, by1);
        if (active) {
            float* o = raycol + 3 * int64_t(rid);  // grouped order
            o[0] = a.c0;
            o[1] = a.c1;
            o[2] = a.c2;
        }
        blended += a.blended;
    }
    if (pairs) count_pairs(pairs, evals, blended);
}

// Direct evaluation at 32 registers a thread: the standard paradigm's blocks
// (a thread per pixel, 256 for its 16 x 16 tiles) then run eight to an SM,
// which its latency-bound per-pixel blend loop needs
template <bool TRANSPOSED, int KPT>
__global__ void __launch_bounds__(1024, TRANSPOSED ? 1 : 2)
composite_full_binned_kernel(CompositeParams p, const int32_t* __restrict__ list, int cap,
                             const uint32_t* __restrict__ gstart,
                             const unsigned long long* __restrict__ keys,
                             const float4* __restrict__ rec, float* __restrict__ Mm,
                             unsigned long long* __restrict__ pairs) {
    extern __shared__ __align__(16) unsigned char smb[];
    const int nthr = blockDim.x;
    const BinnedSmem S = carve_binned(smb, cap, nthr);
    const int group = list[blockIdx.x];
    const int v = group / p.ntiles;
    const int tile = group - v * p.ntiles;
    const int tx = tile % p.ntx, ty = tile / p.ntx;
    const int col = tx * p.tile_w + int(threadIdx.x) % p.tile_w;
    const int row = ty * p.tile_h + int(threadIdx.x) / p.tile_w;
    const bool inside = col < p.width && row < p.height;
    const float px = float(col) - p.half_w, py = float(row) - p.half_h;
    const uint32_t start = gstart[group];
    const int len = int(gstart[group + 1] - start);
    block_sort<KPT>(keys, start, len, cap, S.sk, S.cnt);
    int bx0, bx1, by0, by1;
    warp_box(inside, col, row, bx0, bx1, by0, by1);
    const int64_t vbase = int64_t(v) * p.n;
    Acc a{1.f, 0.f, 0.f, 0.f, 0u};
    uint32_t evals = 0;
    bool done = !inside;
    stream_list<TRANSPOSED>(p, S.sk, len, vbase, rec, S.buf, S.wbuf, a, done, evals, px, py, bx0,
                            bx1, by0, by1);
    if (pairs) count_pairs(pairs, evals, a.blended);
    if (inside) {
        float* o = Mm + ((int64_t(v) * p.height + row) * p.width + col) * 3;
        o[0] = a.c0;
        o[1] = a.c1;
        o[2] = a.c2;
    }
}

// ------------------------------------------------- one warp per tile ----
// DirectL tiles hold few rays (tens) and a few hundred Gaussians, so each
// warp owns one (view, tile) group: it sorts the group's keys in its own
// shared memory (warp-level bucket sort), streams the records in batches of
// 32 with cp.async (up to three batches ahead), and evaluates them transposed
// against its rays.  Only __syncwarp is used, so warps never wait on each
// other.
constexpr int kWarpsPerBlock = 4;

// Positions of the warp's rays about their box centre (x, y), written per
// ray chunk, the per-ray candidate masks of one batch and the third colour
// channel of its records (the other two are decoded in place).  Coordinates
// are stored apart, so four rays' x (or y) are one 16-byte read.
struct RayTable {
    float4 x[8], y[8];
    uint4 mask[8];
    float blue[32];
};

// A warp's shared memory holds its group's keys while it sorts them and,
// once sorted, only their low words (Gaussian index << 4 | quadrant nibble)
// beside the record batches and the ray table: the two phases share the
// space, which keeps the 1024-key class at six blocks per SM.
template <int CAP>
struct WarpSort {
    // at least one bucket a key up to 384 (or 320) keys: the passes that
    // order keys inside buckets grow with the most crowded bucket, and depths
    // cluster; for CAP = 512 the buckets fill the space the stream phase
    // needs anyway, for CAP = 1024 the sort phase sets the size (six blocks
    // per SM)
    static constexpr int kBuckets = CAP <= 512 ? 384 : 320;
    unsigned long long sk[CAP];
    uint32_t bstart[kBuckets];  // bucket sizes, starts, then (after the scatter) ends
};
template <int CAP>
struct WarpStream {
    // record batch slots (one being composited, the rest in flight): as many
    // 32-record batches of 32-byte records as fit in the space the sort phase
    // needs anyway (the 512-key class at eight blocks per SM, the 1024-key
    // class at six)
    static constexpr int kSlots = CAP <= 512 ? 3 : 4;
    uint32_t idx[CAP];
    float4 buf[kSlots][kRecordFloat4][32];
    RayTable rays;
};
template <int CAP>
union WarpSmem {
    WarpSort<CAP> s;
    WarpStream<CAP> c;
};
static_assert(sizeof(WarpSort<512>) <= sizeof(WarpStream<512>), "sort phase fits the stream's space");
static_assert(sizeof(WarpStream<1024>) <= sizeof(WarpSort<1024>), "stream phase fits the sort's space");
// blocks of kWarpsPerBlock warps per SM: eight (512-key class, 64
// registers a thread) and six (1024-key class, 80 registers); 228 KB of
// shared memory an SM, 1 KB of it reserved per block
template <int CAP>
constexpr int warp_class_blocks() { return CAP <= 512 ? 8 : 6; }
static_assert(warp_class_blocks<1024>() * (kWarpsPerBlock * sizeof(WarpSmem<1024>) + 1024) <=
                  228 * 1024, "1024-key class: 6 blocks");
static_assert(warp_class_blocks<512>() * (kWarpsPerBlock * sizeof(WarpSmem<512>) + 1024) <=
                  228 * 1024, "512-key class: 8 blocks");

// Warp-level version of block_sort (len <= CAP).  The first KPL * 32 keys
// (256 in the 512-key class, whose registers are held to 64 for eight blocks
// per SM; 512 in the 1024-key class) are held in registers; the rest of a
// longer list is re-read from global memory (L2) per pass.
template <int CAP>
__device__ void warp_sort(const unsigned long long* __restrict__ keys, uint32_t start, int len,
                          WarpSort<CAP>& W) {
    const int lane = threadIdx.x & 31;
    constexpr int kWarpBuckets = WarpSort<CAP>::kBuckets;
    constexpr int KPL = CAP <= 512 ? 8 : 16;
    unsigned long long kr[KPL];
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    const bool in_regs = len <= KPL * 32;
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
        const int i = j * 32 + lane;
        kr[j] = i < len ? keys[start + i] : ~0ull;
        if (i < len) {
            lo = min(lo, uint32_t(kr[j] >> 32));
            hi = max(hi, uint32_t(kr[j] >> 32));
        }
    }
    for (int i = KPL * 32 + lane; i < len; i += 32) {
        lo = min(lo, uint32_t(keys[start + i] >> 32));
        hi = max(hi, uint32_t(keys[start + i] >> 32));
    }
    if (len <= 1) {
        if (len == 1 && lane == 0) W.sk[0] = kr[0];
        __syncwarp();
        return;
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    int NB = 1;
    while (NB < len) NB <<= 1;
    if (NB > kWarpBuckets) NB = kWarpBuckets;
    // Depths cluster (a dense core in front of a sparse background), so
    // buckets spread evenly over [lo, hi] crowd where the keys are.  With 64
    // buckets or more the mapping is equi-depth at a coarse grain: a first
    // count over kCoarse even bins of [lo, hi] gives bin c a share of the
    // buckets in proportion to its keys (at least one when it has any), and
    // a key takes the bucket of its position within its bin.  The bucket is
    // non-decreasing in the depth word (t is; so is the bin; within a bin so
    // are t - c, exact, and its scaled integer part; the bins' bucket ranges
    // are disjoint and in order), which is all the phases below need.  The
    // bins' table takes the last kCoarse bucket words.
    constexpr int kCoarse = 32;
    const bool equi = NB >= 2 * kCoarse;
    if (equi && NB > kWarpBuckets - kCoarse) NB = kWarpBuckets - kCoarse;
    uint32_t* const table = W.bstart + (kWarpBuckets - kCoarse);
    for (int b = lane; b < NB; b += 32) W.bstart[b] = 0u;
    const float scale = float(equi ? kCoarse : NB) / (float(hi - lo) + 1.0f);
    if (equi) {
        auto bin = [&](unsigned long long k) {
            return min(kCoarse - 1, int(float(uint32_t(k >> 32) - lo) * scale));
        };
        table[lane] = 0u;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < KPL; ++j)
            if (j * 32 + lane < len) atomicAdd(&table[bin(kr[j])], 1u);
        if (!in_regs)
            for (int i = KPL * 32 + lane; i < len; i += 32) atomicAdd(&table[bin(keys[start + i])], 1u);
        __syncwarp();
        const uint32_t nc = table[lane];  // keys in bin `lane`
        const uint32_t nb = nc * uint32_t(NB - kCoarse) / uint32_t(len) + (nc ? 1u : 0u);
        uint32_t inc = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        __syncwarp();
        table[lane] = (inc - nb) | (nb << 16);  // first bucket | buckets << 16
    }
    __syncwarp();
    auto bucket = [&](unsigned long long k) {
        const float t = float(uint32_t(k >> 32) - lo) * scale;
        if (!equi) return min(NB - 1, int(t));
        const int c = min(kCoarse - 1, int(t));
        const uint32_t q = table[c];
        const int nb = int(q >> 16);
        return int(q & 0xFFFFu) + min(nb - 1, int((t - float(c)) * float(nb)));
    };
    // the first KPL * 32 keys are in registers, the rest are re-read
#pragma unroll
    for (int j = 0; j < KPL; ++j)
        if (j * 32 + lane < len) atomicAdd(&W.bstart[bucket(kr[j])], 1u);
    if (!in_regs)
        for (int i = KPL * 32 + lane; i < len; i += 32)
            atomicAdd(&W.bstart[bucket(keys[start + i])], 1u);
    __syncwarp();
    uint32_t most = 0u;  // the most crowded bucket's size
    {  // exclusive scan of bstart[0..NB)
        const int per = (NB + 31) / 32, b0 = lane * per;
        uint32_t sum = 0;
        for (int b = b0; b < b0 + per && b < NB; ++b) {
            const uint32_t c = W.bstart[b];
            sum += c;
            most = max(most, c);
        }
        most = __reduce_max_sync(0xffffffffu, most);
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        uint32_t run = inc - sum;
        __syncwarp();
        for (int b = b0; b < b0 + per && b < NB; ++b) {
            const uint32_t c = W.bstart[b];
            W.bstart[b] = run;
            run += c;
        }
    }
    __syncwarp();
    // scatter: bstart[b] serves as bucket b's cursor, so afterwards it holds
    // the bucket's end (= the start of bucket b + 1)
#pragma unroll
    for (int j = 0; j < KPL; ++j)
        if (j * 32 + lane < len) W.sk[atomicAdd(&W.bstart[bucket(kr[j])], 1u)] = kr[j];
    if (!in_regs)
        for (int i = KPL * 32 + lane; i < len; i += 32) {
            const unsigned long long k = keys[start + i];
            W.sk[atomicAdd(&W.bstart[bucket(k)], 1u)] = k;
        }
    __syncwarp();
    if (most > uint32_t(kBucketSortLimit)) {
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = len + lane; i < P; i += 32) W.sk[i] = ~0ull;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < (P >> 1); i += 32) {
                    const int a = ((i & ~(jj - 1)) << 1) | (i & (jj - 1));
                    const int c = a + jj;
                    const bool up = (a & k) == 0;
                    const unsigned long long x = W.sk[a], y = W.sk[c];
                    if ((x > y) == up) {
                        W.sk[a] = y;
                        W.sk[c] = x;
                    }
                }
                __syncwarp();
            }
    } else {
        // The buckets are in order, so only keys within a bucket are out of
        // place, and no compared pair that straddles two buckets is ever
        // swapped: odd-even transposition phases over the whole list (even
        // pairs (2i, 2i + 1) as one 16-byte access, odd pairs (2i + 1,
        // 2i + 2)) sort every bucket at once, and s phases sort s keys
        // whichever phase comes first, so the most crowded bucket's size is
        // the phase count (none when every bucket holds at most one key).
        // Every lane has work in every phase, unlike a lane-per-bucket
        // insertion sort, where the warp waits for the most crowded of each
        // 32 buckets.
        ulonglong2* const pairs = reinterpret_cast<ulonglong2*>(W.sk);
        for (uint32_t ph = 0; ph < most; ++ph) {
            if ((ph & 1u) == 0u) {
                for (int i = lane; 2 * i + 1 < len; i += 32) {
                    const ulonglong2 q = pairs[i];
                    if (q.x > q.y) pairs[i] = make_ulonglong2(q.y, q.x);
                }
            } else {
                for (int i = 2 * lane + 1; i + 1 < len; i += 64) {
                    const unsigned long long x = W.sk[i], y = W.sk[i + 1];
                    if (x > y) {
                        W.sk[i] = y;
                        W.sk[i + 1] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Keeps the low words of the warp's sorted keys (Gaussian index << 4 |
// nibble) in place of the keys: chunk by chunk, each chunk read whole before
// it is written, and a chunk's 32 words land on keys already read (the words
// of chunk c take bytes [128 c, 128 c + 128), below the chunk's own keys).
template <int CAP>
__device__ __forceinline__ void narrow_keys(WarpSmem<CAP>& W, int len) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < len; base += 32) {
        const int i = base + lane;
        const uint32_t lo = i < len ? uint32_t(W.s.sk[i]) : 0u;
        __syncwarp();
        if (i < len) W.c.idx[i] = lo;
        __syncwarp();
    }
}

// Margin of the batch test below: the expanded quadratic is rounded
// differently from log2_alpha, by less than 0.05 for tiles up to 256 x 256
// pixels (its terms are bounded by lambda_max(conic) <= 1/0.3 times the
// squared distance from the box centre), so a pair passes the test whenever
// log2_alpha reaches the threshold; blend() then decides exactly.
constexpr float kTestMargin = 0.05f;

// Transposed evaluation of a batch of n <= 32 records held in shared memory
// (c0, c1: the two halves of each record) for the warp's rays: lane j holds
// record j's conic (u, v, A, B, C, L) and packed colour (pc, pd) when `hit`
// (j < n).  The lane decodes the colour once for every ray that will blend
// the record (r, g over the packed words, b into T.blue), then expands the
// quadratic about the box centre (ox, oy) into
// l2(x, y) = x (A x + B y + D) + y (C y + E) + F and tests it against every
// ray (5 FMAs per pair, ray positions from the table), four rays per step
// with the FMAs paired over two rays (packed FP32x2 FMA: per component the
// same rounding as fmaf); ray r's mask of candidate records goes to
// T.mask[r].  Then every lane blends its candidates in list order.
template <bool COUNT>
__device__ __forceinline__ void eval32(const float4* c0, float4* c1, int n, bool hit, float u,
                                       float v, float A, float B, float C, float L, float pc,
                                       float pd, Acc& a, bool& done, uint32_t& evals, float px,
                                       float py, RayTable& T, float ox, float oy) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(0xffffffffu, hit)) return;
    if (hit) {
        float r, g, b;
        unpack_rgb(pc, pd, r, g, b);
        reinterpret_cast<float2*>(c1 + lane)[1] = make_float2(r, g);
        T.blue[lane] = b;
    }
    const unsigned act = __ballot_sync(0xffffffffu, !done);
    const float du = u - ox, dv = v - oy;
    const float D = -fmaf(2.f * A, du, B * dv);
    const float E = -fmaf(2.f * C, dv, B * du);
    const float F = hit ? fmaf(du, fmaf(A, du, B * dv), fmaf(C * dv, dv, L)) + kTestMargin : -1e30f;
    const float2 A2 = make_float2(A, A), B2 = make_float2(B, B), C2 = make_float2(C, C);
    const float2 D2 = make_float2(D, D), E2 = make_float2(E, E), F2 = make_float2(F, F);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        if (!((act >> (4 * g)) & 0xFu)) continue;
        const float4 qx = T.x[g], qy = T.y[g];
        unsigned m[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 x = h ? make_float2(qx.z, qx.w) : make_float2(qx.x, qx.y);
            const float2 y = h ? make_float2(qy.z, qy.w) : make_float2(qy.x, qy.y);
            const float2 t1 = __ffma2_rn(A2, x, __ffma2_rn(B2, y, D2));
            const float2 l2 = __ffma2_rn(x, t1, __ffma2_rn(y, __ffma2_rn(C2, y, E2), F2));
            m[2 * h] = __ballot_sync(0xffffffffu, l2.x >= kLog2MinAlpha);
            m[2 * h + 1] = __ballot_sync(0xffffffffu, l2.y >= kLog2MinAlpha);
        }
        if (lane == 0) T.mask[g] = make_uint4(m[0], m[1], m[2], m[3]);
    }
    __syncwarp();
    unsigned mine = (act >> lane) & 1u ? reinterpret_cast<const unsigned*>(T.mask)[lane] : 0u;
    if (COUNT && !done) evals += uint32_t(n);
    while (mine && !done) {  // candidates passed the (widened) test: alpha decides
        const int s1 = __ffs(mine) - 1;
        mine &= mine - 1;
        const bool two = mine != 0u;
        const int s2 = two ? __ffs(mine) - 1 : s1;
        mine &= mine - 1u;
        if (!blend2<COUNT>(a, px, py, c0[s1], c1[s1], T.blue[s1], c0[s2], c1[s2], T.blue[s2], two))
            done = true;
    }
    __syncwarp();
}

// Fills the ray table for the warp's current rays (box centre (ox, oy)).
__device__ __forceinline__ void ray_table(RayTable& T, bool active, float px, float py, float& ox,
                                          float& oy, int bx0, int bx1, int by0, int by1,
                                          float half_w, float half_h) {
    const int lane = threadIdx.x & 31;
    ox = 0.5f * float(bx0 + bx1) - half_w;
    oy = 0.5f * float(by0 + by1) - half_h;
    reinterpret_cast<float*>(T.x)[lane] = active ? px - ox : 1e18f;
    reinterpret_cast<float*>(T.y)[lane] = active ? py - oy : 1e18f;
    __syncwarp();
}

// Lane's record of a shared-memory batch: loads its conic and packed colour
// into registers (lanes past the batch hold a conic that no ray passes).  A
// tile list holds only records whose pixel box meets the tile, and the
// warp's rays spread over the tile, so no box pre-test is made: the widened
// test below sorts the records out at a few FMAs per pair.
__device__ __forceinline__ bool batch_conic(const float4* c0, const float4* c1, int n, float& u,
                                            float& v, float& A, float& B, float& C, float& L,
                                            float& pc, float& pd) {
    const int lane = threadIdx.x & 31;
    u = 0.f; v = 0.f; A = 0.f; B = 0.f; C = 0.f; L = -1e30f; pc = 0.f; pd = 0.f;
    if (lane >= n) return false;
    const float4 q0 = c0[lane];
    const float4 q1 = c1[lane];
    u = q0.x; v = q0.y; A = q0.z; B = q0.w; C = q1.x; L = q1.y; pc = q1.z; pd = q1.w;
    return true;
}

// Streams the warp's sorted list in batches of 32 records (cp.async, up to
// three batches ahead) and composites them, transposed, for the warp's rays.
template <int CAP, bool COUNT>
__device__ __forceinline__ void warp_stream(WarpSmem<CAP>& W, int len, int64_t vbase,
                                            const float4* __restrict__ rec, Acc& a, bool& done,
                                            uint32_t& evals, float px, float py, int bx0, int bx1,
                                            int by0, int by1, float ox, float oy) {
    const int lane = threadIdx.x & 31;
    const int nbatch = (len + 31) / 32;
    if (nbatch == 0) return;
    constexpr int S = WarpStream<CAP>::kSlots;
    // batch b goes to slot b mod S; S - 1 batches are in flight ahead of the
    // one being composited (one cp.async group per batch, empty past the end)
    auto issue = [&](int b, int slot) {
        const int i = b * 32 + lane;
        if (b < nbatch && i < len) {
            const int64_t e = vbase + (W.c.idx[i] >> 4);
            cp_async16(&W.c.buf[slot][0][lane], rec + kRecordFloat4 * e);
            cp_async16(&W.c.buf[slot][1][lane], rec + kRecordFloat4 * e + 1);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) issue(k, k);
    int slot = 0;  // b mod S
    for (int b = 0; b < nbatch; ++b) {
        issue(b + S - 1, slot == 0 ? S - 1 : slot - 1);
        cp_async_wait<S - 1>();
        __syncwarp();
        const float4* c0 = W.c.buf[slot][0];
        float4* c1 = W.c.buf[slot][1];
        slot = slot + 1 == S ? 0 : slot + 1;
        const int n = len - b * 32 < 32 ? len - b * 32 : 32;
        float u, v, A, B, C, L, pc, pd;
        const bool hit = batch_conic(c0, c1, n, u, v, A, B, C, L, pc, pd);
        eval32<COUNT>(c0, c1, n, hit, u, v, A, B, C, L, pc, pd, a, done, evals, px, py, W.c.rays,
                      ox, oy);
        if (__all_sync(0xffffffffu, done)) break;
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Per-warp shared memory of the quadrant block kernel: list positions
// selected for the warp's quadrant and not yet batched, and two batches of 32
// records in flight (cp.async double buffering).
struct QuadPipe {
    int stage[64];
    int idx[2][32];
    float4 buf[2][kRecordFloat4][32];
    RayTable rays;
};

// Streams the records of a block-sorted list whose key marks quadrant `q`
// (bit q of the key's low nibble) for the warp's rays, in list order: the
// selected positions are compacted 32 at a time and their records fetched
// with cp.async one batch ahead of the batch being evaluated (as in
// warp_stream).
__device__ void quadrant_stream(const unsigned long long* sk, int len, int q, int64_t vbase,
                                const float4* __restrict__ rec, QuadPipe& Q, Acc& a, bool& done,
                                uint32_t& evals, float px, float py, int bx0, int bx1, int by0,
                                int by1, float ox, float oy) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int pos = 0, cnt = 0;  // scan position, staged positions (uniform)
    // next batch of up to 32 selected positions into Q.idx[slot], its records
    // requested; returns its size
    auto produce = [&](int slot) -> int {
        while (cnt < 32 && pos < len) {
            const int i = pos + lane;
            const bool sel = i < len && ((uint32_t(sk[i]) >> q) & 1u);
            const unsigned m = __ballot_sync(0xffffffffu, sel);
            if (sel) Q.stage[cnt + __popc(m & lt)] = i;
            cnt += __popc(m);
            pos += 32;
            __syncwarp();
        }
        const int n = cnt < 32 ? cnt : 32;
        const int mine = lane < n ? Q.stage[lane] : 0;
        const int rest = lane + 32 < cnt ? Q.stage[lane + 32] : 0;
        __syncwarp();
        if (lane + 32 < cnt) Q.stage[lane] = rest;
        Q.idx[slot][lane] = mine;
        cnt -= n;
        if (lane < n) {
            const int64_t e = vbase + (uint32_t(sk[mine]) >> 4);
            cp_async16(&Q.buf[slot][0][lane], rec + kRecordFloat4 * e);
            cp_async16(&Q.buf[slot][1][lane], rec + kRecordFloat4 * e + 1);
        }
        cp_async_commit();
        __syncwarp();
        return n;
    };
    int slot = 0;
    int n_cur = produce(0);
    while (n_cur > 0) {
        const int n_next = __all_sync(0xffffffffu, done) ? 0 : produce(slot ^ 1);
        if (n_next > 0) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncwarp();
        const float4* c0 = Q.buf[slot][0];
        float4* c1 = Q.buf[slot][1];
        float u, v, A, B, C, L, pc, pd;
        const bool hit = batch_conic(c0, c1, n_cur, u, v, A, B, C, L, pc, pd);
        eval32<true>(c0, c1, n_cur, hit, u, v, A, B, C, L, pc, pd, a, done, evals, px, py, Q.rays,
                     ox, oy);
        slot ^= 1;
        n_cur = __all_sync(0xffffffffu, done) ? 0 : n_next;
    }
    cp_async_wait<0>();
    __syncwarp();
}


// Index of the frame whose class range holds item i: the last f with
// prefix[f] <= i (prefix ascending, prefix[0] = 0).
__device__ __forceinline__ int frame_of(const int64_t* __restrict__ prefix, int n_frames, int64_t i) {
    int lo = 0, hi = n_frames - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Item i of class cls (0: front of items, 1: back of items) across frames.
__device__ __forceinline__ int4 batch_item(const FrameDesc* __restrict__ F,
                                           const int64_t* __restrict__ prefix, int n_frames, int cls,
                                           int64_t i, int& f) {
    f = frame_of(prefix, n_frames, i);
    const int64_t j = i - __ldg(prefix + f);
    const int4* items = F[f].items;
    return cls == 0 ? items[j] : items[F[f].n_work - 1 - j];
}

// Persistent: resident warps take items until none is left (the first
// n_warps by warp id, the rest claimed from *cursor: groups differ widely in
// cost); an item is {group, first key, first ray, rays << 16 | keys} of
// frame f.  The next item is claimed and loaded before the current one is
// composited.  (Prefetching its keys and rays into L2 as well measured
// slower once eight blocks of the 512-key class were resident.)
template <int CAP, bool COUNT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, warp_class_blocks<CAP>())
composite_rays_warp_kernel(const FrameDesc* __restrict__ F, const int64_t* __restrict__ prefix,
                           int n_frames, int cls, uint32_t* __restrict__ cursor,
                           unsigned long long* __restrict__ pairs) {
    extern __shared__ __align__(16) unsigned char wsm_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP>& W = reinterpret_cast<WarpSmem<CAP>*>(wsm_raw)[warp];
    const int64_t n_items = __ldg(prefix + n_frames);
    const int64_t n_warps = int64_t(gridDim.x) * kWarpsPerBlock;
    int64_t item = int64_t(blockIdx.x) * kWarpsPerBlock + warp;
    uint32_t evals = 0, blended = 0;
    int fcur = 0;
    int4 cur = item < n_items ? batch_item(F, prefix, n_frames, cls, item, fcur) : make_int4(0, 0, 0, 0);
    while (item < n_items) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(cursor, 1u);
        const int64_t nxt = n_warps + int64_t(__shfl_sync(0xffffffffu, c, 0));
        int fnxt = 0;
        const int4 next = nxt < n_items ? batch_item(F, prefix, n_frames, cls, nxt, fnxt)
                                        : make_int4(0, 0, 0, 0);
        const FrameDesc& d = F[fcur];
        const int2* __restrict__ grouped = d.grouped;
        const float4* __restrict__ rec = d.rec;
        float* __restrict__ raycol = d.raycol;
        const int group = cur.x;
        const uint32_t start = uint32_t(cur.y);
        const int rbeg = cur.z, nrays = int(uint32_t(cur.w) >> 16), len = cur.w & 0xFFFF;
        const int v = group / d.cp.ntiles;
        const float half_w = d.cp.half_w, half_h = d.cp.half_h;
        warp_sort<CAP>(d.keys, start, len, W.s);
        narrow_keys<CAP>(W, len);
        const int64_t vbase = int64_t(v) * d.cp.n;
        for (int r0 = 0; r0 < nrays; r0 += 32) {
            const int rid = r0 + lane;
            const bool active = rid < nrays;
            const int2 ray = active ? grouped[rbeg + rid] : make_int2(0, -1);
            const int col = int(uint32_t(ray.x) & 0xFFFFu), row = int(uint32_t(ray.x) >> 16);
            const float px = float(col) - half_w, py = float(row) - half_h;
            int bx0, bx1, by0, by1;
            warp_box(active, col, row, bx0, bx1, by0, by1);
            float ox, oy;
            ray_table(W.c.rays, active, px, py, ox, oy, bx0, bx1, by0, by1, half_w, half_h);
            Acc a{1.f, 0.f, 0.f, 0.f, 0u};
            bool done = !active;
            warp_stream<CAP, COUNT>(W, len, vbase, rec, a, done, evals, px, py, bx0, bx1, by0, by1,
                                    ox, oy);
            if (active) {
                float* o = raycol + 3 * (int64_t(rbeg) + rid);  // grouped order
                o[0] = a.c0;
                o[1] = a.c1;
                o[2] = a.c2;
            }
            blended += a.blended;
        }
        item = nxt;
        cur = next;
        fcur = fnxt;
    }
    if (COUNT) count_pairs(pairs, evals, blended);
}

// Block class across frames: one block of four warps per group list too long
// for a warp (sorted together in shared memory up to `cap` keys); warp q then
// composites the group's rays in quadrant q of the tile (x half + 2 * y half)
// over the records whose key marks that quadrant, so every warp has work and
// each streams only about half of the list.  Persistent like the warp
// classes.
__global__ void __launch_bounds__(kBinnedThreads)
composite_rays_block_kernel(const FrameDesc* __restrict__ F, const int64_t* __restrict__ prefix,
                            int n_frames, int cap, uint32_t* __restrict__ cursor,
                            unsigned long long* __restrict__ pairs) {
    extern __shared__ __align__(16) unsigned char smb[];
    __shared__ int64_t s_item;
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(smb);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smb + 8 * size_t(cap));
    QuadPipe* pipes = reinterpret_cast<QuadPipe*>(smb + block_sort_bytes(cap));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_items = __ldg(prefix + n_frames);
    uint32_t evals = 0, blended = 0;
    int64_t item = blockIdx.x;
    while (item < n_items) {
        const int f = frame_of(prefix, n_frames, item);
        const FrameDesc& d = F[f];
        const int4 bi = d.block_items[item - __ldg(prefix + f)];
        const int4 wi = d.gwork[bi.z];
        const uint32_t start = uint32_t(bi.y);
        const int len = bi.w;
        if (len > cap) {
            if (threadIdx.x == 0) atomicOr(d.status, 2u);
        } else {
            const int v = wi.x / d.cp.ntiles;
            const int tile = wi.x - v * d.cp.ntiles;
            const int xm = (tile % d.cp.ntx) * d.cp.tile_w + (d.cp.tile_w >> 1);
            const int ym = (tile / d.cp.ntx) * d.cp.tile_h + (d.cp.tile_h >> 1);
            const int qx = warp & 1, qy = warp >> 1;
            // the keys carry the quadrant bits (bit q: the record's pixel
            // box overlaps quadrant q, x half + 2 * y half, of the tile)
            block_sort<0>(d.keys, start, len, cap, sk, cnt);
            __syncthreads();
            const int64_t vbase = int64_t(v) * d.cp.n;
            for (int r0 = wi.y; r0 < wi.z; r0 += 32) {
                const int rid = r0 + lane;
                const int2 ray = rid < wi.z ? d.grouped[rid] : make_int2(0, -1);
                const int col = int(uint32_t(ray.x) & 0xFFFFu), row = int(uint32_t(ray.x) >> 16);
                const bool mine = rid < wi.z && int(col >= xm) == qx && int(row >= ym) == qy;
                if (!__any_sync(0xffffffffu, mine)) continue;
                const float px = float(col) - d.cp.half_w, py = float(row) - d.cp.half_h;
                int bx0, bx1, by0, by1;
                warp_box(mine, col, row, bx0, bx1, by0, by1);
                float ox, oy;
                ray_table(pipes[warp].rays, mine, px, py, ox, oy, bx0, bx1, by0, by1, d.cp.half_w,
                          d.cp.half_h);
                Acc a{1.f, 0.f, 0.f, 0.f, 0u};
                bool done = !mine;
                quadrant_stream(sk, len, warp, vbase, d.rec, pipes[warp], a, done, evals, px, py,
                                bx0, bx1, by0, by1, ox, oy);
                if (mine) {
                    float* o = d.raycol + 3 * int64_t(rid);  // grouped order
                    o[0] = a.c0;
                    o[1] = a.c1;
                    o[2] = a.c2;
                }
                blended += a.blended;
            }
        }
        __syncthreads();  // shared memory reused by the next item
        if (threadIdx.x == 0) s_item = int64_t(gridDim.x) + int64_t(atomicAdd(cursor, 1u));
        __syncthreads();
        item = s_item;
    }
    if (pairs) count_pairs(pairs, evals, blended);
}

__global__ void batch_prefix_kernel(const FrameDesc* __restrict__ F, int n_frames,
                                    int64_t* __restrict__ prefix) {
    if (threadIdx.x != 0) return;
    int64_t a = 0, b = 0, c = 0;
    const int stride = n_frames + 1;
    for (int f = 0; f < n_frames; ++f) {
        prefix[f] = a;
        prefix[stride + f] = b;
        prefix[2 * stride + f] = c;
        a += F[f].meta[0];
        b += F[f].meta[4];
        c += F[f].meta[1];
    }
    prefix[n_frames] = a;
    prefix[stride + n_frames] = b;
    prefix[2 * stride + n_frames] = c;
}

// Items of the warp classes: DirectL groups with fewer than 65536 rays and
// at most cap1 keys become self-contained items at the front of `items`,
// those with cap1 < keys <= cap2 at the back (cap2 = 0: no second class); the
// rest become block items {group, first key, gwork index, keys}.
// meta = {n_items1, n_block, max keys, -, n_items2}.  Nothing is written
// when the frame's keys were not all emitted (*total_keys > key_cap, or
// status bit 0 already set).
__global__ void partition_warp_kernel(const int4* __restrict__ gwork, int64_t n_work,
                                      GroupSlices S, uint32_t cap1, uint32_t cap2,
                                      int4* __restrict__ items, int4* __restrict__ block_items,
                                      uint32_t* __restrict__ meta,
                                      const uint32_t* __restrict__ total_keys, uint32_t key_cap,
                                      uint32_t* __restrict__ status) {
    if (total_keys && *total_keys > key_cap) {  // keys were not emitted
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1u);
        return;
    }
    if (status && (*status & 1u)) return;
    const uint32_t* __restrict__ first = S.use_alt && *S.use_alt ? S.start_alt : S.start;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    // one counter atomic a warp and class: the warp's items of a class stay
    // together and in group order (consecutive items share records in L2)
    auto slot = [&](unsigned am, bool mine, uint32_t* counter) -> uint32_t {
        const unsigned m = __ballot_sync(am, mine);
        uint32_t base = 0u;
        if (m) {
            const int leader = __ffs(m) - 1;
            if (int(threadIdx.x & 31) == leader) base = atomicAdd(counter, uint32_t(__popc(m)));
            base = __shfl_sync(am, base, leader);
        }
        return base + uint32_t(__popc(m & lt));
    };
    for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < n_work;
         w += int64_t(gridDim.x) * blockDim.x) {
        const unsigned am = __activemask();
        const int4 wi = gwork[w];
        const uint32_t st = first[wi.x];
        const uint32_t len = (S.cursor ? S.cursor[wi.x] : S.start[wi.x + 1]) - st;
        const uint32_t nr = uint32_t(wi.z - wi.y);
        const int4 it = make_int4(wi.x, int(st), wi.y, int((nr << 16) | len));
        const int cls = nr < 65536u && len <= cap1 ? 0 : (nr < 65536u && len <= cap2 ? 1 : 2);
        const uint32_t s0 = slot(am, cls == 0, meta);
        const uint32_t s1 = slot(am, cls == 1, meta + 4);
        const uint32_t s2 = slot(am, cls == 2, meta + 1);
        if (cls == 0)
            items[s0] = it;
        else if (cls == 1)
            items[n_work - 1 - int64_t(s1)] = it;
        else
            block_items[s2] = make_int4(wi.x, int(st), int(w), int(len));
        const uint32_t longest = __reduce_max_sync(am, len);
        if (int(threadIdx.x & 31) == __ffs(am) - 1) atomicMax(meta + 2, longest);
    }
}

__global__ void partition_kernel(const int4* __restrict__ gwork, int64_t n_work,
                                 const uint32_t* __restrict__ gstart, uint32_t small_cap,
                                 int32_t* __restrict__ small_list, int32_t* __restrict__ large_list,
                                 uint32_t* __restrict__ meta) {
    for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < n_work;
         w += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = gwork ? gwork[w].x : w;
        const uint32_t len = gstart[g + 1] - gstart[g];
        if (len <= small_cap) small_list[atomicAdd(meta, 1u)] = int32_t(w);
        else large_list[atomicAdd(meta + 1, 1u)] = int32_t(w);
        atomicMax(meta + 2, len);
    }
}

// subpixels [first, n)
__global__ void reorder_kernel(const uint32_t* __restrict__ ray_of, const float* __restrict__ raycol,
                               int64_t first, int64_t n, float* __restrict__ out,
                               const uint32_t* __restrict__ skip) {
    if (skip && *skip) return;  // the frame was not composited
    for (int64_t i = first + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        out[i] = raycol[3 * int64_t(ray_of[i]) + (i % 3)];
}

// The same, four subpixels a thread (16-byte index loads and stores, four
// gathers in flight) over subpixels [0, 4 n4).
__global__ void reorder4_kernel(const uint4* __restrict__ ray_of, const float* __restrict__ raycol,
                                int64_t n4, float4* __restrict__ out,
                                const uint32_t* __restrict__ skip) {
    if (skip && *skip) return;  // the frame was not composited
    for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n4;
         q += int64_t(gridDim.x) * blockDim.x) {
        const uint4 r = ray_of[q];
        const uint32_t k = uint32_t((4 * q) % 3);  // channel of the first; then k+1, k+2, k
        const uint32_t k1 = k == 2u ? 0u : k + 1u, k2 = k == 0u ? 2u : k - 1u;
        float4 o;
        o.x = raycol[3 * int64_t(r.x) + k];
        o.y = raycol[3 * int64_t(r.y) + k1];
        o.z = raycol[3 * int64_t(r.z) + k2];
        o.w = raycol[3 * int64_t(r.w) + k];
        out[q] = o;
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

// The paper's "HR w SR" assembly: subpixel (x, y, k) takes channel k of view
// V(x, 3y + k) at its repurposed source pixel src = (x' << 16 | y') (Sec. 5)
// rather than at (x, y); a source outside the panel (never produced by the
// repurposing) reads the subpixel's own pixel.
__global__ void repurposed_interweave_kernel(int32_t w, int32_t h, const uint16_t* __restrict__ V,
                                             const uint32_t* __restrict__ src,
                                             const float* __restrict__ Mm,
                                             float* __restrict__ out) {
    const int64_t total = 3 * int64_t(w) * h;
    const int64_t plane = int64_t(h) * w * 3;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t sp = src[i];
        const uint32_t sr = sp >> 16, sc = sp & 0xFFFFu;
        const int64_t p = (sr < uint32_t(h) && sc < uint32_t(w)) ? int64_t(sr) * w + sc : i / 3;
        out[i] = Mm[int64_t(V[i]) * plane + 3 * p + (i - 3 * (i / 3))];
    }
}

// Alg. 1 with views rendered at rw x rh and upsampled while interweaving:
// subpixel (x, y, k) takes channel k of view V(x, 3y + k) bilinearly at
// column y rw / w, row x rh / h of that view (pixel (r, c) of a view samples
// its image point (c, r) about the principal point, so the panel's and the
// view's pixel grids share the corner), clamped at the border.  Positions
// are split into integer and fractional parts exactly.
__global__ void resize_interweave_kernel(int32_t w, int32_t h, int32_t rw, int32_t rh,
                                         const uint16_t* __restrict__ V,
                                         const float* __restrict__ Mm, float* __restrict__ out) {
    const int64_t n = 3 * int64_t(w) * h;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = i / (3 * int64_t(w));
        const int64_t s = i - row * 3 * int64_t(w);
        const int64_t col = s / 3;
        const int k = int(s - col * 3);
        const int v = V[i];
        const int64_t nx = col * rw, ny = row * rh;
        const int x0 = int(nx / w), y0 = int(ny / h);
        const float fx = float(nx - int64_t(x0) * w) / float(w);
        const float fy = float(ny - int64_t(y0) * h) / float(h);
        const int x1 = min(x0 + 1, rw - 1), y1 = min(y0 + 1, rh - 1);
        const float* img = Mm + int64_t(v) * rh * rw * 3 + k;
        const float a = img[(int64_t(y0) * rw + x0) * 3], b = img[(int64_t(y0) * rw + x1) * 3];
        const float c = img[(int64_t(y1) * rw + x0) * 3], d = img[(int64_t(y1) * rw + x1) * 3];
        out[i] = (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
    }
}

}  // namespace

cudaError_t launch_composite_rays(const CompositeParams& p, const int4* work, int64_t n_work,
                                  const int2* grouped, const uint2* ranges, const uint32_t* vals,
                                  const float4* rec, float* raycol, unsigned long long* pairs,
                                  cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    composite_rays_kernel<<<unsigned(n_work), kRayThreads, 0, s>>>(p, work, grouped, ranges, vals,
                                                                   rec, raycol, pairs);
    return cudaGetLastError();
}

cudaError_t launch_composite_full(const CompositeParams& p, int32_t nv, const uint2* ranges,
                                  const uint32_t* vals, const float4* rec, float* Mm,
                                  unsigned long long* pairs, cudaStream_t s) {
    const int nthr = p.tile_w * p.tile_h;
    const size_t smem = size_t(nthr) * 3 * sizeof(float4) + size_t(nthr / 32) * 64 * sizeof(int);
    const int64_t blocks = int64_t(nv) * p.ntiles;
    composite_full_kernel<<<unsigned(blocks), nthr, smem, s>>>(p, ranges, vals, rec, Mm, pairs);
    return cudaGetLastError();
}

size_t block_smem_bytes(int cap) {
    return block_sort_bytes(cap) + (kBinnedThreads / 32) * sizeof(QuadPipe);
}

size_t binned_smem_bytes(int cap, int nthr) {
    const size_t off = (8 * size_t(cap) + 4 * size_t(cap + 2) + 15) & ~size_t(15);
    return off + size_t(nthr) * 3 * sizeof(float4) + size_t(nthr / 32) * 64 * sizeof(int);
}

cudaError_t launch_composite_rays_binned(const CompositeParams& p, const int4* gwork,
                                         const int32_t* list, int64_t n_list, int cap,
                                         const int2* grouped, const uint32_t* gstart,
                                         const unsigned long long* keys, const float4* rec,
                                         float* raycol, unsigned long long* pairs, int transposed,
                                         cudaStream_t s) {
    if (n_list <= 0) return cudaSuccess;
    const int nthr = kBinnedThreads;
    const size_t smem = binned_smem_bytes(cap, nthr);
    const bool regs = false;
    auto go = [&](auto kernel) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        kernel<<<unsigned(n_list), nthr, smem, s>>>(p, gwork, list, cap, grouped, gstart, keys, rec,
                                                    raycol, pairs);
        return cudaGetLastError();
    };
    if (transposed) return regs ? go(composite_rays_binned_kernel<true, 8>)
                                : go(composite_rays_binned_kernel<true, 0>);
    return regs ? go(composite_rays_binned_kernel<false, 8>) : go(composite_rays_binned_kernel<false, 0>);
}

cudaError_t launch_composite_full_binned(const CompositeParams& p, const int32_t* list,
                                         int64_t n_list, int cap, const uint32_t* gstart,
                                         const unsigned long long* keys, const float4* rec,
                                         float* Mm, unsigned long long* pairs, int transposed,
                                         cudaStream_t s) {
    if (n_list <= 0) return cudaSuccess;
    const int nthr = p.tile_w * p.tile_h;
    const size_t smem = binned_smem_bytes(cap, nthr);
    const bool regs = false;
    auto go = [&](auto kernel) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        kernel<<<unsigned(n_list), nthr, smem, s>>>(p, list, cap, gstart, keys, rec, Mm, pairs);
        return cudaGetLastError();
    };
    if (transposed) return regs ? go(composite_full_binned_kernel<true, 4>)
                                : go(composite_full_binned_kernel<true, 0>);
    return regs ? go(composite_full_binned_kernel<false, 4>) : go(composite_full_binned_kernel<false, 0>);
}

namespace {
template <class K>
cudaError_t launch_persistent(K kernel, int threads, size_t smem, int64_t max_blocks,
                              const FrameDesc* frames, const int64_t* prefix, int32_t n_frames,
                              int extra, uint32_t* cursor, unsigned long long* pairs, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = int64_t(num_sms()) * (per_sm > 0 ? per_sm : 1);
    if (blocks > max_blocks) blocks = max_blocks;
    kernel<<<unsigned(blocks), threads, smem, s>>>(frames, prefix, n_frames, extra, cursor, pairs);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_batch_prefix(const FrameDesc* frames, int32_t n_frames, int64_t* prefix,
                                cudaStream_t s) {
    batch_prefix_kernel<<<1, 32, 0, s>>>(frames, n_frames, prefix);
    return cudaGetLastError();
}

cudaError_t launch_composite_rays_warp(int cap, int cls, const FrameDesc* frames,
                                       const int64_t* prefix, int32_t n_frames, int64_t max_items,
                                       uint32_t* cursor, unsigned long long* pairs, cudaStream_t s) {
    if (max_items <= 0 || n_frames <= 0) return cudaSuccess;
    const int64_t need = (max_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t* pc = prefix + int64_t(cls) * (n_frames + 1);
    const int t = kWarpsPerBlock * 32;
    const size_t s1 = kWarpsPerBlock * sizeof(WarpSmem<512>), s2 = kWarpsPerBlock * sizeof(WarpSmem<1024>);
    if (cap == 1024)
        return pairs ? launch_persistent(composite_rays_warp_kernel<1024, true>, t, s2, need, frames,
                                         pc, n_frames, cls, cursor, pairs, s)
                     : launch_persistent(composite_rays_warp_kernel<1024, false>, t, s2, need, frames,
                                         pc, n_frames, cls, cursor, pairs, s);
    return pairs ? launch_persistent(composite_rays_warp_kernel<512, true>, t, s1, need, frames, pc,
                                     n_frames, cls, cursor, pairs, s)
                 : launch_persistent(composite_rays_warp_kernel<512, false>, t, s1, need, frames, pc,
                                     n_frames, cls, cursor, pairs, s);
}

cudaError_t launch_composite_rays_block(int block_cap, const FrameDesc* frames,
                                        const int64_t* prefix, int32_t n_frames, int64_t max_items,
                                        uint32_t* cursor, unsigned long long* pairs, cudaStream_t s) {
    if (max_items <= 0 || n_frames <= 0) return cudaSuccess;
    const size_t smem = block_smem_bytes(block_cap);
    return launch_persistent(composite_rays_block_kernel, kBinnedThreads, smem, max_items, frames,
                             prefix + 2 * (n_frames + 1), n_frames, block_cap, cursor, pairs, s);
}

cudaError_t launch_partition_warp(const int4* gwork, int64_t n_work, const GroupSlices& slices,
                                  uint32_t cap1, uint32_t cap2, int4* items, int4* block_items,
                                  uint32_t* meta, const uint32_t* total_keys, uint32_t key_cap,
                                  uint32_t* status, cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    int64_t grid = (n_work + 255) / 256;
    const int64_t lim = int64_t(num_sms()) * 16;
    if (grid > lim) grid = lim;
    partition_warp_kernel<<<unsigned(grid), 256, 0, s>>>(gwork, n_work, slices, cap1, cap2, items,
                                                         block_items, meta, total_keys, key_cap,
                                                         status);
    return cudaGetLastError();
}

cudaError_t launch_partition(const int4* gwork, int64_t n_work, const uint32_t* gstart,
                             uint32_t small_cap, int32_t* small_list, int32_t* large_list,
                             uint32_t* meta, cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    int64_t grid = (n_work + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 16;
    if (grid > cap) grid = cap;
    partition_kernel<<<unsigned(grid), 256, 0, s>>>(gwork, n_work, gstart, small_cap, small_list,
                                                    large_list, meta);
    return cudaGetLastError();
}

int reorder_launches(const uint32_t* ray_of, int64_t n, const float* out) {
    if (n <= 0) return 0;
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(ray_of) & 15u) == 0;
    if (!vec) return 1;
    return (n / 4 > 0 ? 1 : 0) + (n % 4 != 0 ? 1 : 0);
}

cudaError_t launch_reorder(const uint32_t* ray_of, const float* raycol, int64_t n, float* out,
                           const uint32_t* skip, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t cap = int64_t(num_sms()) * 32;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0 && (reinterpret_cast<uintptr_t>(ray_of) & 15u) == 0) {
        const int64_t n4 = n / 4;
        if (n4 > 0) {
            int64_t grid = (n4 + 255) / 256;
            if (grid > cap) grid = cap;
            reorder4_kernel<<<unsigned(grid), 256, 0, s>>>(reinterpret_cast<const uint4*>(ray_of),
                                                           raycol, n4, reinterpret_cast<float4*>(out),
                                                           skip);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        done = 4 * n4;
    }
    if (done < n) {  // the tail, or everything for unaligned buffers
        int64_t grid = (n - done + 255) / 256;
        if (grid > cap) grid = cap;
        reorder_kernel<<<unsigned(grid), 256, 0, s>>>(ray_of, raycol, done, n, out, skip);
    }
    return cudaGetLastError();
}

cudaError_t launch_resize_interweave(int32_t w, int32_t h, int32_t rw, int32_t rh,
                                     const uint16_t* V, const float* Mm, float* out,
                                     cudaStream_t s) {
    const int64_t n = 3 * int64_t(w) * h;
    int64_t grid = (n + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    resize_interweave_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(w, h, rw, rh, V, Mm, out);
    return cudaGetLastError();
}

cudaError_t launch_repurposed_interweave(int32_t w, int32_t h, const uint16_t* V, const uint32_t* src,
                                        const float* Mm, float* out, cudaStream_t s) {
    const int64_t total = 3 * int64_t(w) * h;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    repurposed_interweave_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(w, h, V, src, Mm, out);
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
