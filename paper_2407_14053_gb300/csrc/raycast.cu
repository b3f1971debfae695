// Ray-order 3DGS (Sec. 7, Alg. 3): every required ray is cast through the
// scene, one thread per ray.  Per ray, each Gaussian it meets gives its point
// of highest density t_j = (mu - o)^T S^-1 d / (d^T S^-1 d) (Eq. (16)) and
// alpha_j = o_j G(o + t_j d) (Eq. (17)); the c_h nearest are kept (Alg. 3
// keeps them in a max-heap of capacity c_h; here an ascending list of the
// same capacity, which needs no sort at the end) and blended front to back
// with the SH colour at the ray direction.  The ray meets a Gaussian when
// alpha_j >= 1/255 and t_j > 0.2 (the near plane of the rasteriser); the
// list orders by (t, index), so the image does not depend on the traversal
// order.
//
// Acceleration (Sec. 7: a compact 8-wide bounding-volume hierarchy built with
// the surface area heuristic): every Gaussian is bounded by the box of its
// alpha >= 1/255 ellipsoid.  A binary tree is built top down over the
// scene's stored order (a 3D Morton curve of the means), so every node holds
// a contiguous run of Gaussians; each node is split at the position of the
// run that minimises the SAH cost A(left) n(left) + A(right) n(right) over
// every split position (prefix and suffix boxes of the run), down to leaves
// of at most four Gaussians.  The binary tree is then collapsed into 8-wide
// nodes: a wide node starts from a binary node's two children and
// repeatedly opens the child with the largest surface area until it has
// eight.  Children are visited nearest first, and once the list is full a
// node whose box starts beyond the list's farthest entry is skipped: a
// Gaussian's highest-density point lies inside its ellipsoid, hence inside
// every box above it.
#include <cfloat>

#include "dl_internal.cuh"
#include "sh.cuh"

namespace dl {
namespace {

constexpr float kNearT = 0.2f;
constexpr float kMinAlpha = 1.0f / 255.0f;

// Per Gaussian: a = (mean, opacity), b = (S00, S01, S02, S11), c = (S12, S22)
// of S = Sigma^-1 = R diag(s^-2) R^T; box of the alpha >= 1/255 ellipsoid.
template <typename T>
__global__ void rc_prepare_kernel(GaussiansView<T> G, int64_t n, float4* __restrict__ gauss,
                                  float4* __restrict__ box) {
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n;
         g += int64_t(gridDim.x) * blockDim.x) {
        float qw = to_f(G.rot[4 * g]), qx = to_f(G.rot[4 * g + 1]);
        float qy = to_f(G.rot[4 * g + 2]), qz = to_f(G.rot[4 * g + 3]);
        const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw *= qn; qx *= qn; qy *= qn; qz *= qn;
        const float R[3][3] = {
            {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
            {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
            {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
        float s2[3], is2[3];
        for (int k = 0; k < 3; ++k) {
            const float ls = to_f(G.log_scale[3 * g + k]);
            s2[k] = __expf(2.f * ls);
            is2[k] = __expf(-2.f * ls);
        }
        auto inv = [&](int i, int j) {
            return R[i][0] * R[j][0] * is2[0] + R[i][1] * R[j][1] * is2[1] + R[i][2] * R[j][2] * is2[2];
        };
        const float op = 1.f / (1.f + __expf(-to_f(G.opacity_logit[g])));
        const float mx = G.mean[3 * g], my = G.mean[3 * g + 1], mz = G.mean[3 * g + 2];
        gauss[3 * g] = make_float4(mx, my, mz, op);
        gauss[3 * g + 1] = make_float4(inv(0, 0), inv(0, 1), inv(0, 2), inv(1, 1));
        gauss[3 * g + 2] = make_float4(inv(1, 2), inv(2, 2), 0.f, 0.f);
        // alpha >= 1/255 inside (x - mu)^T S (x - mu) <= K = 2 ln(255 o); the
        // ellipsoid's half extent along axis i is sqrt(K Sigma_ii) (+0.1 %)
        float4 lo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), hi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
        if (op * 255.f > 1.f) {
            const float K = 2.f * logf(255.f * op);
            float h[3];
            for (int i = 0; i < 3; ++i)
                h[i] = sqrtf(K * (R[i][0] * R[i][0] * s2[0] + R[i][1] * R[i][1] * s2[1] +
                                  R[i][2] * R[i][2] * s2[2])) * 1.001f + 1e-6f;
            lo = make_float4(mx - h[0], my - h[1], mz - h[2], 0.f);
            hi = make_float4(mx + h[0], my + h[1], mz + h[2], 0.f);
        }
        box[2 * g] = lo;
        box[2 * g + 1] = hi;
    }
}

// ---- SAH tree ------------------------------------------------------------
constexpr int kLeafMax = 4;           // Gaussians per leaf of the binary tree
constexpr int kMedianDepth = 40;      // from this binary depth on, runs split at the middle
constexpr int kBuildThreads = 256;

__host__ __device__ inline uint32_t leaf_ref(uint32_t first, uint32_t count) {
    return kRayLeafBit | (first << 3) | (count - 1);
}

// Binary node of the build (not kept): box, children (node index or leaf
// reference), the box's surface area.
struct BinNode {
    float4 lo, hi;
    uint32_t child[2];
    float area;
    uint32_t pad;
};
// Run [a, b) of Gaussians that becomes binary node `node` at `depth`.
struct BuildTask {
    uint32_t a, b, node, depth;
};

struct Box {
    float lx, ly, lz, hx, hy, hz;
};
__device__ __forceinline__ Box box_empty() { return {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}; }
__device__ __forceinline__ Box box_join(const Box& a, const Box& b) {
    return {fminf(a.lx, b.lx), fminf(a.ly, b.ly), fminf(a.lz, b.lz),
            fmaxf(a.hx, b.hx), fmaxf(a.hy, b.hy), fmaxf(a.hz, b.hz)};
}
__device__ __forceinline__ Box box_of(const float4* __restrict__ gbox, uint32_t g) {
    const float4 l = gbox[2 * size_t(g)], h = gbox[2 * size_t(g) + 1];
    return {l.x, l.y, l.z, h.x, h.y, h.z};
}
__device__ __forceinline__ float box_area(const Box& b) {
    const float dx = b.hx - b.lx, dy = b.hy - b.ly, dz = b.hz - b.lz;
    if (!(dx >= 0.f) || !(dy >= 0.f) || !(dz >= 0.f)) return 0.f;
    return 2.f * (dx * dy + dy * dz + dz * dx);
}
__device__ __forceinline__ Box shfl_box(const Box& b, int src_delta, bool up) {
    Box r;
    if (up) {
        r.lx = __shfl_up_sync(0xffffffffu, b.lx, src_delta);
        r.ly = __shfl_up_sync(0xffffffffu, b.ly, src_delta);
        r.lz = __shfl_up_sync(0xffffffffu, b.lz, src_delta);
        r.hx = __shfl_up_sync(0xffffffffu, b.hx, src_delta);
        r.hy = __shfl_up_sync(0xffffffffu, b.hy, src_delta);
        r.hz = __shfl_up_sync(0xffffffffu, b.hz, src_delta);
    } else {
        r.lx = __shfl_down_sync(0xffffffffu, b.lx, src_delta);
        r.ly = __shfl_down_sync(0xffffffffu, b.ly, src_delta);
        r.lz = __shfl_down_sync(0xffffffffu, b.lz, src_delta);
        r.hx = __shfl_down_sync(0xffffffffu, b.hx, src_delta);
        r.hy = __shfl_down_sync(0xffffffffu, b.hy, src_delta);
        r.hz = __shfl_down_sync(0xffffffffu, b.hz, src_delta);
    }
    return r;
}

// Exclusive prefix (pre) and suffix (suf) unions of the block's per-thread
// boxes in thread order, and their total.  Every thread of the block calls it.
__device__ void block_box_scans(const Box& mine, Box& pre, Box& suf, Box& total) {
    __shared__ Box s_warp[kBuildThreads / 32], s_pre[kBuildThreads / 32], s_suf[kBuildThreads / 32];
    __shared__ Box s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Box inc = mine, rinc = mine;  // inclusive prefix / suffix inside the warp
    for (int o = 1; o < 32; o <<= 1) {
        const Box u = shfl_box(inc, o, true), d = shfl_box(rinc, o, false);
        if (lane >= o) inc = box_join(inc, u);
        if (lane + o < 32) rinc = box_join(rinc, d);
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Box run = box_empty();
        for (int w = 0; w < nw; ++w) {
            s_pre[w] = run;
            run = box_join(run, s_warp[w]);
        }
        s_total = run;
        run = box_empty();
        for (int w = nw - 1; w >= 0; --w) {
            s_suf[w] = run;
            run = box_join(run, s_warp[w]);
        }
    }
    __syncthreads();
    const Box ex_in = shfl_box(inc, 1, true);     // inclusive prefix of lane - 1
    const Box ex_rin = shfl_box(rinc, 1, false);  // inclusive suffix of lane + 1
    pre = lane > 0 ? box_join(s_pre[warp], ex_in) : s_pre[warp];
    suf = lane < 31 ? box_join(s_suf[warp], ex_rin) : s_suf[warp];
    total = s_total;
    __syncthreads();
}

// One block per task: the run [a, b) is split at the position k (a < k < b)
// minimising A([a, k)) (k - a) + A([k, b)) (b - k), over every position
// (from binary depth kMedianDepth on: the middle).  A side of at most
// kLeafMax Gaussians becomes a leaf, a longer one a new node and a task of
// the next level.  sal: one float per Gaussian of scratch.  counters[0]:
// binary nodes allocated, counters[1]: next level's tasks.
__global__ void __launch_bounds__(kBuildThreads)
sah_split_kernel(const BuildTask* __restrict__ tasks, const float4* __restrict__ gbox,
                 float* __restrict__ sal, BinNode* __restrict__ nodes, BuildTask* __restrict__ next,
                 uint32_t* __restrict__ counters) {
    __shared__ float s_cost[kBuildThreads];
    __shared__ uint32_t s_k[kBuildThreads];
    const BuildTask tk = tasks[blockIdx.x];
    const uint32_t a = tk.a, b = tk.b, m = b - a;
    const uint32_t per = (m + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = min(b, a + threadIdx.x * per), c1 = min(b, c0 + per);
    Box cb = box_empty();
    for (uint32_t g = c0; g < c1; ++g) cb = box_join(cb, box_of(gbox, g));
    Box pre, suf, total;
    block_box_scans(cb, pre, suf, total);
    // forward: sal[g] = area of [a, g + 1)
    Box L = pre;
    for (uint32_t g = c0; g < c1; ++g) {
        L = box_join(L, box_of(gbox, g));
        sal[g] = box_area(L);
    }
    __syncthreads();
    // backward: the cost of splitting at k = g, right side [g, b)
    Box R = suf;
    float best = FLT_MAX;
    uint32_t bk = a + m / 2;
    for (uint32_t g = c1; g > c0; --g) {
        R = box_join(R, box_of(gbox, g - 1));
        const uint32_t k = g - 1;
        if (k > a) {
            const float cost = sal[k - 1] * float(k - a) + box_area(R) * float(b - k);
            if (cost < best || (cost == best && k < bk)) {
                best = cost;
                bk = k;
            }
        }
    }
    s_cost[threadIdx.x] = best;
    s_k[threadIdx.x] = bk;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t k = a + m / 2;
        if (tk.depth < uint32_t(kMedianDepth)) {
            float bc = FLT_MAX;
            for (unsigned t = 0; t < blockDim.x; ++t)
                if (s_cost[t] < bc || (s_cost[t] == bc && s_k[t] < k)) {
                    bc = s_cost[t];
                    k = s_k[t];
                }
            if (!(bc < FLT_MAX)) k = a + m / 2;  // every box empty: the middle
        }
        BinNode nd;
        nd.lo = make_float4(total.lx, total.ly, total.lz, 0.f);
        nd.hi = make_float4(total.hx, total.hy, total.hz, 0.f);
        nd.area = box_area(total);
        nd.pad = 0u;
        const uint32_t ra[2] = {a, k}, rb[2] = {k, b};
        for (int side = 0; side < 2; ++side) {
            const uint32_t n = rb[side] - ra[side];
            if (n <= uint32_t(kLeafMax)) {
                nd.child[side] = leaf_ref(ra[side], n);
            } else {
                const uint32_t id = atomicAdd(counters, 1u);
                nd.child[side] = id;
                next[atomicAdd(counters + 1, 1u)] = BuildTask{ra[side], rb[side], id, tk.depth + 1};
            }
        }
        nodes[tk.node] = nd;
    }
}

// Collapse of the binary tree into 8-wide nodes, one wide node per task: the
// binary node's two children are opened, the one with the largest surface
// area first, until there are eight (or only leaves).  counters[2]: wide
// nodes allocated, [3]: next level's tasks, [4]: deepest wide level.
struct CollapseTask {
    uint32_t bin, wide, depth, pad;
};

__global__ void collapse_kernel(const CollapseTask* __restrict__ q, uint32_t nq,
                                const BinNode* __restrict__ bins, const float4* __restrict__ gbox,
                                RayNode* __restrict__ wide, CollapseTask* __restrict__ next,
                                uint32_t* __restrict__ counters) {
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nq; idx += gridDim.x * blockDim.x) {
        const CollapseTask t = q[idx];
        uint32_t ref[8];
        int c = 2;
        ref[0] = bins[t.bin].child[0];
        ref[1] = bins[t.bin].child[1];
        while (c < 8) {
            int best = -1;
            float ba = -1.f;
            for (int i = 0; i < c; ++i)
                if (!(ref[i] & kRayLeafBit) && bins[ref[i]].area > ba) {
                    ba = bins[ref[i]].area;
                    best = i;
                }
            if (best < 0) break;
            const uint32_t r = ref[best];
            ref[best] = bins[r].child[0];
            ref[c++] = bins[r].child[1];
        }
        RayNode nd;
        for (int k = 0; k < 8; ++k) {
            Box bx = box_empty();
            uint32_t ch = kRayNoChild;
            if (k < c) {
                if (ref[k] & kRayLeafBit) {
                    const uint32_t first = (ref[k] & ~kRayLeafBit) >> 3, cnt = (ref[k] & 7u) + 1u;
                    for (uint32_t g = first; g < first + cnt; ++g) bx = box_join(bx, box_of(gbox, g));
                    ch = ref[k];
                } else {
                    const BinNode& bn = bins[ref[k]];
                    bx = {bn.lo.x, bn.lo.y, bn.lo.z, bn.hi.x, bn.hi.y, bn.hi.z};
                    ch = atomicAdd(counters + 2, 1u);
                    next[atomicAdd(counters + 3, 1u)] = CollapseTask{ref[k], ch, t.depth + 1, 0u};
                }
            }
            nd.lox[k] = bx.lx; nd.loy[k] = bx.ly; nd.loz[k] = bx.lz;
            nd.hix[k] = bx.hx; nd.hiy[k] = bx.hy; nd.hiz[k] = bx.hz;
            nd.child[k] = ch;
            nd.pad[k] = 0u;
        }
        wide[t.wide] = nd;
        atomicMax(counters + 4, t.depth);
    }
}

// A scene of at most kLeafMax Gaussians: the root holds one leaf.
__global__ void leaf_root_kernel(const float4* __restrict__ gbox, uint32_t n, RayNode* __restrict__ wide) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    RayNode nd;
    for (int k = 0; k < 8; ++k) {
        Box bx = box_empty();
        uint32_t ch = kRayNoChild;
        if (k == 0 && n > 0) {
            for (uint32_t g = 0; g < n; ++g) bx = box_join(bx, box_of(gbox, g));
            ch = leaf_ref(0u, n);
        }
        nd.lox[k] = bx.lx; nd.loy[k] = bx.ly; nd.loz[k] = bx.lz;
        nd.hix[k] = bx.hx; nd.hiy[k] = bx.hy; nd.hiz[k] = bx.hz;
        nd.child[k] = ch;
        nd.pad[k] = 0u;
    }
    wide[0] = nd;
}

// Highest-density point and alpha of Gaussian g along the ray.
__device__ __forceinline__ float rc_alpha(const float4* __restrict__ gauss, int64_t g, float ox,
                                          float oy, float oz, float dx, float dy, float dz, float& t) {
    const float4 a = gauss[3 * g], b = gauss[3 * g + 1], c = gauss[3 * g + 2];
    // S d and d^T S d, S = [[b.x b.y b.z] [b.y b.w c.x] [b.z c.x c.y]]
    const float sx = b.x * dx + b.y * dy + b.z * dz;
    const float sy = b.y * dx + b.w * dy + c.x * dz;
    const float sz = b.z * dx + c.x * dy + c.y * dz;
    const float den = dx * sx + dy * sy + dz * sz;
    const float mx = a.x - ox, my = a.y - oy, mz = a.z - oz;
    t = (mx * sx + my * sy + mz * sz) / den;
    const float px = t * dx - mx, py = t * dy - my, pz = t * dz - mz;
    const float q = b.x * px * px + b.w * py * py + c.y * pz * pz +
                    2.f * (b.y * px * py + b.z * px * pz + c.x * py * pz);
    return fminf(0.99f, a.w * __expf(-0.5f * q));
}

constexpr int kTraceThreads = 128;
constexpr int kTraceWarps = kTraceThreads / 32;
constexpr int kListHead = 16;  // list slots 0..15 (the 16 nearest) in shared memory

// A ray's entry into a box (+inf when it misses the box or the box lies
// behind the near plane).
__device__ __forceinline__ float slab_enter(const float4& lo, const float4& hi, float ox, float oy,
                                            float oz, float ix, float iy, float iz) {
    const float tx0 = (lo.x - ox) * ix, tx1 = (hi.x - ox) * ix;
    const float ty0 = (lo.y - oy) * iy, ty1 = (hi.y - oy) * iy;
    const float tz0 = (lo.z - oz) * iz, tz1 = (hi.z - oz) * iz;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return (tn <= tf && tf > kNearT) ? tn : INFINITY;
}

// A ray's ascending list of its c_h nearest intersections: slots below
// kListHead in shared memory, the rest in the thread's local memory.
struct RayList {
    unsigned long long* head;  // slot k < kListHead at head[32 k]
    unsigned long long* rest;  // slot k >= kListHead at rest[k - kListHead]
    __device__ __forceinline__ unsigned long long get(int k) const {
        return k < kListHead ? head[32 * k] : rest[k - kListHead];
    }
    __device__ __forceinline__ void set(int k, unsigned long long v) const {
        if (k < kListHead) head[32 * k] = v;
        else rest[k - kListHead] = v;
    }
};

// Traversal of the 8-wide tree is by the whole warp: its rays share a camera
// centre and nearly a direction, so they need nearly the same nodes.  A
// warp-shared stack holds {node or leaf reference, the lanes whose ray hit
// its box}; a popped node is loaded once for the warp, every lane tests its
// ray against the eight child boxes (a child beyond the lane's full list does
// not count as hit), and the children hit by any lane are pushed farthest
// first by their nearest entry over those lanes.  A leaf is tested by the
// lanes that hit it.  At most 7 entries a level plus 8 are pending (the
// tree's depth is checked against kMaxWideDepth when it is built; the guard
// only keeps the stack in bounds).  Every lane reaches every warp-wide
// synchronisation point: the loop's trip count and the branch between leaf
// and node are the same for the whole warp.
template <typename T, int DEG>
__global__ void __launch_bounds__(kTraceThreads)
rc_trace_kernel(const float4* __restrict__ gauss, const RayNode* __restrict__ nodes,
                int64_t n, const T* __restrict__ sh, const uint32_t* __restrict__ ray_view,
                const uint32_t* __restrict__ ray_pix, const int2* __restrict__ order,
                int64_t n_rays, const Cam* __restrict__ cams, float focal, float half_w,
                float half_h, int heap_cap, float* __restrict__ raycol) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    __shared__ uint32_t s_ref[kTraceWarps][kRayStack];
    __shared__ uint32_t s_lanes[kTraceWarps][kRayStack];
    __shared__ unsigned long long s_head[kTraceWarps][kListHead][32];  // [slot][lane]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const bool valid = i0 < n_rays;
    const int64_t i = valid ? i0 : n_rays - 1;  // lanes past the end follow the last ray, unwritten
    // thread i casts ray order[i].y: the rays grouped by (view, tile) and
    // Morton-ordered inside a tile
    const int64_t r = order ? int64_t(order[i].y) : i;
    const uint32_t px = ray_pix[r];
    const Cam& cam = cams[ray_view[r]];
    // direction: camera ray ((c - w/2 - shift)/f, (r - h/2)/f, 1) to world
    const float cx = (float(px & 0xFFFFu) - half_w - cam.shift) / focal;
    const float cy = (float(px >> 16) - half_h) / focal;
    float dx = cam.r[0] * cx + cam.r[3] * cy + cam.r[6];
    float dy = cam.r[1] * cx + cam.r[4] * cy + cam.r[7];
    float dz = cam.r[2] * cx + cam.r[5] * cy + cam.r[8];
    const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dn; dy *= dn; dz *= dn;
    const float ox = cam.c[0], oy = cam.c[1], oz = cam.c[2];
    const float ix = 1.f / dx, iy = 1.f / dy, iz = 1.f / dz;
    // list entries packed as t's FP32 bits << 32 | Gaussian index: t > 0, so
    // the integer order of the packed key is the (t, index) order
    unsigned long long rest[kMaxHeap - kListHead];
    const RayList hl{&s_head[warp][0][lane], rest};
    int hn = 0;
    // Transmittance bound: tb is set once the intersections found so far
    // (every one at t <= tmax) multiply T below 5e-5.  Sorted, they alone
    // take T below 1e-4 by t = tmax, so blending stops at or before tmax and
    // nothing beyond tb can be blended; the walk skips it.  (5e-5, not
    // 1e-4: the product is formed in another order than the blend's.)
    float prodT = 1.f, tmax = 0.f, tb = INFINITY;
    uint32_t* const st_ref = s_ref[warp];
    uint32_t* const st_lanes = s_lanes[warp];
    const unsigned all = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) {
        st_ref[0] = 0u;  // the root
        st_lanes[0] = all;
    }
    int sp = all ? 1 : 0;
    __syncwarp();
    while (sp > 0) {
        --sp;
        const uint32_t e = st_ref[sp];
        const bool mine = (st_lanes[sp] >> lane) & 1u;
        __syncwarp();
        const float bound = fminf(
            tb, hn == heap_cap ? __uint_as_float(uint32_t(hl.get(hn - 1) >> 32)) : INFINITY);
        if (e & kRayLeafBit) {  // leaf: Gaussians first .. first + count - 1
            if (mine) {
                const uint32_t first = (e & ~kRayLeafBit) >> 3, cnt = (e & 7u) + 1u;
                // the leaf's Gaussians evaluated together (their loads in
                // flight at once), then taken in order
                for (uint32_t base = 0; base < cnt; base += kLeafMax) {
                    float al[kLeafMax], tl[kLeafMax];
#pragma unroll
                    for (int q = 0; q < kLeafMax; ++q) {
                        al[q] = 0.f;
                        tl[q] = 0.f;
                        if (base + q < cnt)
                            al[q] = rc_alpha(gauss, first + base + q, ox, oy, oz, dx, dy, dz, tl[q]);
                    }
#pragma unroll
                    for (int q = 0; q < kLeafMax; ++q) {
                        if (base + q >= cnt) break;
                        const uint32_t g = first + base + q;
                        const float a = al[q], t = tl[q];
                        if (!(a >= kMinAlpha) || !(t > kNearT) || t > tb) continue;
                        if (tb == INFINITY) {
                            prodT *= 1.f - a;
                            tmax = fmaxf(tmax, t);
                            if (prodT < 5e-5f) tb = tmax;
                        }
                        const unsigned long long key =
                            (static_cast<unsigned long long>(__float_as_uint(t)) << 32) | g;
                        if (hn == heap_cap) {  // full: drop the farthest if this one is nearer
                            if (!(key < hl.get(hn - 1))) continue;
                            --hn;
                        }
                        // insert into the ascending list: rays find their
                        // intersections nearly in order, so few entries move
                        int k = hn++;
                        while (k > 0) {
                            const unsigned long long vp = hl.get(k - 1);
                            if (!(key < vp)) break;
                            hl.set(k, vp);
                            --k;
                        }
                        hl.set(k, key);
                    }
                }
            }
        } else {  // wide node: its children, nearest first
            const float4* nf = reinterpret_cast<const float4*>(nodes + e);
            float te[8];
            uint32_t chv[8];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float4 a0 = __ldg(nf + q), a1 = __ldg(nf + 2 + q), a2 = __ldg(nf + 4 + q);
                const float4 a3 = __ldg(nf + 6 + q), a4 = __ldg(nf + 8 + q), a5 = __ldg(nf + 10 + q);
                const uint4 c4 = __ldg(reinterpret_cast<const uint4*>(nf + 12 + q));
                const float lxa[4] = {a0.x, a0.y, a0.z, a0.w}, lya[4] = {a1.x, a1.y, a1.z, a1.w};
                const float lza[4] = {a2.x, a2.y, a2.z, a2.w}, hxa[4] = {a3.x, a3.y, a3.z, a3.w};
                const float hya[4] = {a4.x, a4.y, a4.z, a4.w}, hza[4] = {a5.x, a5.y, a5.z, a5.w};
                const uint32_t ca[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    chv[4 * q + k] = ca[k];
                    float t = INFINITY;
                    if (mine && ca[k] != kRayNoChild) {
                        t = slab_enter(make_float4(lxa[k], lya[k], lza[k], 0.f),
                                       make_float4(hxa[k], hya[k], hza[k], 0.f), ox, oy, oz, ix, iy,
                                       iz);
                        if (t > bound) t = INFINITY;  // beyond a full list
                    }
                    te[4 * q + k] = t;
                }
            }
            // children hit by any lane, with their nearest entry (t >= 0:
            // the bits order like the values)
            uint32_t hit[8], near[8];
            int m = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const bool h = te[c] < INFINITY;
                hit[c] = __ballot_sync(0xffffffffu, h);
                near[c] = __reduce_min_sync(0xffffffffu,
                                            h ? __float_as_uint(fmaxf(te[c], 0.f)) : 0xFFFFFFFFu);
                m += hit[c] ? 1 : 0;
            }
            if (sp + m > kRayStack) m = 0;  // cannot happen (depth checked); keeps the stack in bounds
            if (lane < 8 && m > 0) {
                // farthest first: lane c places child c by its rank in
                // descending entry (ties by child position)
                uint32_t my_hit = 0u, my_near = 0u, my_ref = 0u;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (c == lane) {
                        my_hit = hit[c];
                        my_near = near[c];
                        my_ref = chv[c];
                    }
                }
                if (my_hit) {
                    int rank = 0;
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        rank += (hit[c] && (near[c] > my_near || (near[c] == my_near && c < lane)));
                    st_ref[sp + rank] = my_ref;
                    st_lanes[sp + rank] = my_hit;
                }
            }
            sp += m;
            __syncwarp();
        }
    }
    if (valid) {
        // blend front to back, colour from the SH at the ray direction
        float Y[16];
        sh_basis<DEG>(dx, dy, dz, Y);
        float tr = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;  // transmittance, colour
        for (int k = 0; k < hn; ++k) {
            float t;
            const int64_t g = int64_t(uint32_t(hl.get(k)));
            const float a = rc_alpha(gauss, g, ox, oy, oz, dx, dy, dz, t);
            const float tn = tr * (1.f - a);
            if (tn < 1e-4f) break;
            float col[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NC; ++j) acc = fmaf(Y[j], to_f(sh[(g * NC + j) * 3 + ch]), acc);
                col[ch] = fmaxf(acc + 0.5f, 0.f);
            }
            const float w = a * tr;
            c0 = fmaf(w, col[0], c0);
            c1 = fmaf(w, col[1], c1);
            c2 = fmaf(w, col[2], c2);
            tr = tn;
        }
        // colours in thread order: the grouped order when `order` is given
        raycol[3 * i] = c0;
        raycol[3 * i + 1] = c1;
        raycol[3 * i + 2] = c2;
    }
}

int grid_of(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = int64_t(num_sms()) * 64;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_raycast_prepare(int dtype, const void* const* attrs, int64_t n, float4* gauss,
                                   float4* gbox, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_of(n, 256);
    if (dtype == 1) {
        GaussiansView<__nv_bfloat16> G{static_cast<const float*>(attrs[0]),
                                       static_cast<const __nv_bfloat16*>(attrs[1]),
                                       static_cast<const __nv_bfloat16*>(attrs[2]),
                                       static_cast<const __nv_bfloat16*>(attrs[3]),
                                       static_cast<const __nv_bfloat16*>(attrs[4])};
        rc_prepare_kernel<<<grid, 256, 0, s>>>(G, n, gauss, gbox);
    } else if (dtype == 2) {
        GaussiansView<__half> G{static_cast<const float*>(attrs[0]), static_cast<const __half*>(attrs[1]),
                                static_cast<const __half*>(attrs[2]), static_cast<const __half*>(attrs[3]),
                                static_cast<const __half*>(attrs[4])};
        rc_prepare_kernel<<<grid, 256, 0, s>>>(G, n, gauss, gbox);
    } else {
        GaussiansView<float> G{static_cast<const float*>(attrs[0]), static_cast<const float*>(attrs[1]),
                               static_cast<const float*>(attrs[2]), static_cast<const float*>(attrs[3]),
                               static_cast<const float*>(attrs[4])};
        rc_prepare_kernel<<<grid, 256, 0, s>>>(G, n, gauss, gbox);
    }
    return cudaGetLastError();
}

// Build scratch: binary nodes, two task lists, the SAH sweep's areas, the
// counters and two collapse queues.
struct BuildScratch {
    BinNode* bins;
    BuildTask* tasks[2];
    float* sal;
    uint32_t* counters;
    CollapseTask* queue[2];
};
static size_t task_cap(int64_t n) { return size_t(n / (kLeafMax + 1) + 2); }
static BuildScratch carve_build(void* tmp, int64_t n) {
    BuildScratch b;
    char* p = static_cast<char*>(tmp);
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~size_t(255);
        return q;
    };
    b.bins = reinterpret_cast<BinNode*>(take(sizeof(BinNode) * size_t(n + 1)));
    b.tasks[0] = reinterpret_cast<BuildTask*>(take(sizeof(BuildTask) * task_cap(n)));
    b.tasks[1] = reinterpret_cast<BuildTask*>(take(sizeof(BuildTask) * task_cap(n)));
    b.sal = reinterpret_cast<float*>(take(sizeof(float) * size_t(n + 1)));
    b.counters = reinterpret_cast<uint32_t*>(take(64));
    b.queue[0] = reinterpret_cast<CollapseTask*>(take(sizeof(CollapseTask) * size_t(n + 1)));
    b.queue[1] = reinterpret_cast<CollapseTask*>(take(sizeof(CollapseTask) * size_t(n + 1)));
    return b;
}

size_t raycast_build_tmp_bytes(int64_t n) {
    const size_t r = 255;
    auto up = [&](size_t x) { return (x + r) & ~r; };
    return up(sizeof(BinNode) * size_t(n + 1)) + 2 * up(sizeof(BuildTask) * task_cap(n)) +
           up(sizeof(float) * size_t(n + 1)) + up(64) + 2 * up(sizeof(CollapseTask) * size_t(n + 1));
}

cudaError_t raycast_build_binary(const float4* gbox, int64_t n, void* tmp, int64_t* n_bin,
                                 cudaStream_t s) {
    *n_bin = 0;
    if (n <= kLeafMax) return cudaSuccess;
    BuildScratch b = carve_build(tmp, n);
    uint32_t h[16] = {1u, 0u};  // the root is node 0
    cudaError_t e = cudaMemcpyAsync(b.counters, h, sizeof(h), cudaMemcpyHostToDevice, s);
    const BuildTask root{0u, uint32_t(n), 0u, 0u};
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.tasks[0], &root, sizeof(root), cudaMemcpyHostToDevice, s);
    uint32_t n_tasks = 1;
    int cur = 0;
    while (e == cudaSuccess && n_tasks > 0) {
        sah_split_kernel<<<n_tasks, kBuildThreads, 0, s>>>(b.tasks[cur], gbox, b.sal, b.bins,
                                                           b.tasks[cur ^ 1], b.counters);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, b.counters, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.counters + 1, 0, 4, s);
        n_tasks = h[1];
        cur ^= 1;
    }
    *n_bin = int64_t(h[0]);
    return e;
}

cudaError_t raycast_collapse(const float4* gbox, int64_t n, void* tmp, int64_t n_bin,
                             RayNode* nodes, int64_t* n_wide, int* depth, cudaStream_t s) {
    *n_wide = 1;
    *depth = 0;
    if (n_bin == 0) {
        leaf_root_kernel<<<1, 32, 0, s>>>(gbox, uint32_t(n > 0 ? n : 0), nodes);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    BuildScratch b = carve_build(tmp, n);
    uint32_t h[16] = {0u};
    h[2] = 1u;  // the wide root is node 0
    cudaError_t e = cudaMemcpyAsync(b.counters, h, sizeof(h), cudaMemcpyHostToDevice, s);
    const CollapseTask root{0u, 0u, 0u, 0u};
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.queue[0], &root, sizeof(root), cudaMemcpyHostToDevice, s);
    uint32_t nq = 1;
    int cur = 0;
    while (e == cudaSuccess && nq > 0) {
        collapse_kernel<<<grid_of(nq, 128), 128, 0, s>>>(b.queue[cur], nq, b.bins, gbox, nodes,
                                                         b.queue[cur ^ 1], b.counters);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, b.counters, 32, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b.counters + 3, 0, 4, s);
        nq = h[3];
        cur ^= 1;
    }
    *n_wide = int64_t(h[2]);
    *depth = int(h[4]);
    return e;
}

cudaError_t launch_raycast(int dtype, int sh_degree, const float4* gauss, const RayNode* nodes,
                           int64_t n, const void* sh, const uint32_t* ray_view,
                           const uint32_t* ray_pix, const int2* order, int64_t n_rays,
                           const Cam* cams, float focal, float half_w, float half_h, int heap_cap,
                           float* raycol, cudaStream_t s) {
    if (n_rays <= 0) return cudaSuccess;
    const unsigned grid = unsigned((n_rays + kTraceThreads - 1) / kTraceThreads);
#define DL_RC(T, D)                                                                          \
    rc_trace_kernel<T, D><<<grid, kTraceThreads, 0, s>>>(gauss, nodes, n, static_cast<const T*>(sh),   \
                                               ray_view, ray_pix, order, n_rays, cams, focal,  \
                                               half_w, half_h, heap_cap, raycol)
#define DL_RC_DEG(T)                  \
    switch (sh_degree) {              \
        case 0: DL_RC(T, 0); break;   \
        case 1: DL_RC(T, 1); break;   \
        case 2: DL_RC(T, 2); break;   \
        default: DL_RC(T, 3); break;  \
    }
    if (dtype == 1) {
        DL_RC_DEG(__nv_bfloat16)
    } else if (dtype == 2) {
        DL_RC_DEG(__half)
    } else {
        DL_RC_DEG(float)
    }
#undef DL_RC_DEG
#undef DL_RC
    return cudaGetLastError();
}

}  // namespace dl
