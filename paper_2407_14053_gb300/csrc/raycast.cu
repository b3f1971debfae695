// Ray-order 3DGS (Sec. 7, Alg. 3): every required ray is cast through the
// scene, one thread per ray.  Per ray, each Gaussian it meets gives its point
// of highest density t_j = (mu - o)^T S^-1 d / (d^T S^-1 d) (Eq. (16)) and
// alpha_j = o_j G(o + t_j d) (Eq. (17)); a max-heap of capacity c_h keeps the
// c_h nearest; they are sorted by t and blended front to back with the SH
// colour at the ray direction.  The ray meets a Gaussian when alpha_j >= 1/255
// and t_j > 0.2 (the near plane of the rasteriser); the heap orders by
// (t, index), so the image does not depend on the traversal order.
//
// Acceleration: an implicit 8-wide bounding-volume tree over the scene's
// stored order (a 3D Morton curve of the means): leaf node i bounds Gaussians
// 8i..8i+7 (each by the box of its alpha >= 1/255 ellipsoid), node i of level
// k > 0 bounds nodes 8i..8i+7 of level k-1.  Children are visited nearest
// first, and once the heap is full a node whose box starts beyond the heap's
// farthest entry is skipped: a Gaussian's highest-density point lies inside
// its ellipsoid, hence inside every box above it.
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

// Node i bounds children 8i..8i+7 (< n_child) of the level below.
__global__ void rc_level_kernel(const float4* __restrict__ child, int64_t n_child,
                                float4* __restrict__ node, int64_t n_node) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_node;
         i += int64_t(gridDim.x) * blockDim.x) {
        float4 lo = make_float4(FLT_MAX, FLT_MAX, FLT_MAX, 0.f), hi = make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f);
        for (int64_t c = 8 * i; c < 8 * i + 8 && c < n_child; ++c) {
            const float4 a = child[2 * c], b = child[2 * c + 1];
            lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
            hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
        }
        node[2 * i] = lo;
        node[2 * i + 1] = hi;
    }
}

// Ray-box slab test: entry distance, or +inf when the ray misses the box
// (or the box lies behind the near plane).
__device__ __forceinline__ float slab_enter(const float4& lo, const float4& hi, float ox, float oy,
                                            float oz, float ix, float iy, float iz) {
    const float tx0 = (lo.x - ox) * ix, tx1 = (hi.x - ox) * ix;
    const float ty0 = (lo.y - oy) * iy, ty1 = (hi.y - oy) * iy;
    const float tz0 = (lo.z - oz) * iz, tz1 = (hi.z - oz) * iz;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    return (tn <= tf && tf > kNearT) ? tn : INFINITY;
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

template <typename T, int DEG>
__global__ void __launch_bounds__(128)
rc_trace_kernel(const float4* __restrict__ gauss, const float4* __restrict__ nodes,
                const int64_t* __restrict__ level_off, int n_levels, const int64_t* __restrict__ level_n,
                int64_t n, const T* __restrict__ sh, const uint32_t* __restrict__ ray_view,
                const uint32_t* __restrict__ ray_pix, const int2* __restrict__ order,
                int64_t n_rays, const Cam* __restrict__ cams, float focal, float half_w,
                float half_h, int heap_cap, float* __restrict__ raycol) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n_rays) return;
    // thread i casts ray order[i].y: the rays grouped by (view, tile) and
    // Morton-ordered inside a tile, so a warp's rays share a camera centre and
    // nearly share a direction, and traverse the tree alike
    const int64_t r = order ? int64_t(order[i].y) : i;
    // heap entries packed as t's FP32 bits << 32 | Gaussian index: t > 0, so
    // the integer order of the packed key is the (t, index) order
    unsigned long long hk[kMaxHeap];
    int hn = 0;
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
    // traversal: stack entries level << 28 | node; depth-first with <= 8
    // children pushed per node holds at most 7 (levels - 1) + 8 <= kRayStack
    uint32_t stack[kRayStack];
    int sp = 0;
    stack[sp++] = uint32_t(n_levels - 1) << 28;
    while (sp > 0) {
        const uint32_t e = stack[--sp];
        const int lv = int(e >> 28);
        const int64_t i = int64_t(e & 0x0FFFFFFFu);
        const float bound = hn == heap_cap ? __uint_as_float(uint32_t(hk[0] >> 32)) : INFINITY;
        if (lv == 0) {  // leaf: Gaussians 8i..8i+7
            for (int64_t g = 8 * i; g < 8 * i + 8 && g < n; ++g) {
                float t;
                const float a = rc_alpha(gauss, g, ox, oy, oz, dx, dy, dz, t);
                if (!(a >= kMinAlpha) || !(t > kNearT)) continue;
                const unsigned long long key =
                    (static_cast<unsigned long long>(__float_as_uint(t)) << 32) | uint32_t(g);
                if (hn < heap_cap) {  // insert and sift up
                    int k = hn++;
                    while (k > 0) {
                        const int p = (k - 1) >> 1;
                        if (!(hk[p] < key)) break;
                        hk[k] = hk[p];
                        k = p;
                    }
                    hk[k] = key;
                } else if (key < hk[0]) {  // replace the farthest
                    int k = 0;
                    for (;;) {
                        int c = 2 * k + 1;
                        if (c >= hn) break;
                        if (c + 1 < hn && hk[c] < hk[c + 1]) ++c;
                        if (!(key < hk[c])) break;
                        hk[k] = hk[c];
                        k = c;
                    }
                    hk[k] = key;
                }
            }
        } else {  // children 8i..8i+7 of the level below, nearest first
            const float4* child = nodes + 2 * level_off[lv - 1];
            const int64_t nc = level_n[lv - 1];
            float ct[8];
            uint32_t ce[8];
            int m = 0;
            for (int64_t c = 8 * i; c < 8 * i + 8 && c < nc; ++c) {
                const float te = slab_enter(child[2 * c], child[2 * c + 1], ox, oy, oz, ix, iy, iz);
                if (!(te < INFINITY) || te > bound) continue;  // misses, or beyond a full heap
                int k = m++;
                while (k > 0 && ct[k - 1] < te) {  // descending: nearest pushed last
                    ct[k] = ct[k - 1];
                    ce[k] = ce[k - 1];
                    --k;
                }
                ct[k] = te;
                ce[k] = (uint32_t(lv - 1) << 28) | uint32_t(c);
            }
            for (int k = 0; k < m; ++k) stack[sp++] = ce[k];
        }
    }
    // pop the heap from its farthest entry: list in ascending (t, index)
    for (int k = hn - 1; k > 0; --k) {
        const unsigned long long top = hk[0], last = hk[k];
        int j = 0;
        for (;;) {
            int c = 2 * j + 1;
            if (c >= k) break;
            if (c + 1 < k && hk[c] < hk[c + 1]) ++c;
            if (!(last < hk[c])) break;
            hk[j] = hk[c];
            j = c;
        }
        hk[j] = last;
        hk[k] = top;
    }
    // blend front to back, colour from the SH at the ray direction
    float Y[16];
    sh_basis<DEG>(dx, dy, dz, Y);
    float tr = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;  // transmittance, colour
    for (int k = 0; k < hn; ++k) {
        float t;
        const int64_t g = int64_t(uint32_t(hk[k]));
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
    raycol[3 * r] = c0;
    raycol[3 * r + 1] = c1;
    raycol[3 * r + 2] = c2;
}

int grid_of(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = int64_t(num_sms()) * 64;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

}  // namespace

size_t raycast_bvh_nodes(int64_t n, int64_t* level_n, int* n_levels) {
    int64_t cnt = (n + 7) / 8, total = 0;
    int lv = 0;
    for (;;) {
        level_n[lv++] = cnt;
        total += cnt;
        if (cnt == 1) break;
        cnt = (cnt + 7) / 8;
    }
    *n_levels = lv;
    return size_t(total);
}

cudaError_t launch_raycast_prepare(int dtype, const void* const* attrs, int64_t n, float4* gauss,
                                   float4* gbox, float4* nodes, const int64_t* level_off,
                                   const int64_t* level_n, int n_levels, cudaStream_t s) {
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
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float4* below = gbox;
    int64_t n_below = n;
    for (int lv = 0; lv < n_levels; ++lv) {
        float4* out = nodes + 2 * level_off[lv];
        rc_level_kernel<<<grid_of(level_n[lv], 256), 256, 0, s>>>(below, n_below, out, level_n[lv]);
        below = out;
        n_below = level_n[lv];
    }
    return cudaGetLastError();
}

cudaError_t launch_raycast(int dtype, int sh_degree, const float4* gauss, const float4* nodes,
                           const int64_t* level_off_dev, const int64_t* level_n_dev, int n_levels,
                           int64_t n, const void* sh, const uint32_t* ray_view,
                           const uint32_t* ray_pix, const int2* order, int64_t n_rays,
                           const Cam* cams, float focal, float half_w, float half_h, int heap_cap,
                           float* raycol, cudaStream_t s) {
    if (n_rays <= 0) return cudaSuccess;
    const unsigned grid = unsigned((n_rays + 127) / 128);
#define DL_RC(T, D)                                                                          \
    rc_trace_kernel<T, D><<<grid, 128, 0, s>>>(gauss, nodes, level_off_dev, n_levels,         \
                                               level_n_dev, n, static_cast<const T*>(sh),      \
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
