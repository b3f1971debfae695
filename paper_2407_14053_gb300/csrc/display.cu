// Offline display tables (Sec. 4 step (1)): the view-index map (Sec. 3.1,
// Eqs. (1)-(3)), subpixel repurposing (Sec. 5, Alg. 2) and the R-first ray
// table (Sec. 5, last part).  Integer arithmetic throughout, so the tables
// are exact.
#include <mutex>

#include "../../include/directl.h"
#include "dl_internal.cuh"

namespace dl {
namespace {

constexpr int64_t kQ32 = int64_t(1) << 32;

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}
__device__ __forceinline__ int64_t ceil_div_pos(int64_t a, int64_t b) {  // b > 0
    return -floor_div(-a, b);
}

// d_offset (Eq. (1)) of subpixel column s in row x, Q32.
__device__ __forceinline__ int64_t d_offset(const DisplayQ& q, int64_t x, int64_t s) {
    return s * kQ32 + x * q.t3q - q.kq;
}

// ------------------------------------------------------------------ a1 ---
// v = floor(N_v (d mod L_x) / L_x), Eqs. (2)-(3), mod taken into [0, L_x).
// One thread writes 8 consecutive views (one 16-byte store).
__global__ void view_map_kernel(DisplayQ q, uint16_t* __restrict__ V) {
    const int64_t S = 3 * int64_t(q.w);
    const int64_t total = S * q.h;
    const int64_t n8 = (total + 7) / 8;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n8;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i0 = t * 8;
        int64_t x = i0 / S, s = i0 - x * S;
        int64_t d = d_offset(q, x, s);
        int64_t xo = d % q.lq;
        if (xo < 0) xo += q.lq;
        uint16_t out[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            out[j] = (uint16_t)((int64_t(q.nv) * xo) / q.lq);
            // next subpixel: same row adds 2^32, a new row restarts at s = 0
            if (++s == S) {
                s = 0;
                ++x;
                d = d_offset(q, x, 0);
                xo = d % q.lq;
                if (xo < 0) xo += q.lq;
            } else {
                xo += kQ32;
                if (xo >= q.lq) xo %= q.lq;
            }
        }
        if (i0 + 8 <= total && ((reinterpret_cast<uintptr_t>(V + i0) & 15) == 0)) {
            uint4 pk;
            pk.x = out[0] | (uint32_t(out[1]) << 16);
            pk.y = out[2] | (uint32_t(out[3]) << 16);
            pk.z = out[4] | (uint32_t(out[5]) << 16);
            pk.w = out[6] | (uint32_t(out[7]) << 16);
            *reinterpret_cast<uint4*>(V + i0) = pk;
        } else {
            for (int j = 0; j < 8 && i0 + j < total; ++j) V[i0 + j] = out[j];
        }
    }
}

// ------------------------------------------------------------------ a2 ---
__device__ __forceinline__ int64_t area_of(const DisplayQ& q, int64_t x, int64_t s) {
    return floor_div(floor_div(d_offset(q, x, s), q.lq), q.pw);
}

__device__ __forceinline__ uint32_t pack_px(int64_t x, int64_t y) {
    return (uint32_t(x) << 16) | uint32_t(y);
}

// Alg. 2, one warp per area (areas are independent, Sec. 5).  Inside an area
// the subpixels are visited in row-major order; each chain samples a pixel
// (Eq. (11)), parks its two other channels in B_rgb (Eq. (12)) and hands
// them to the next subpixels of the same view found by the search
// (Eqs. (13)-(14)).  The search is the first subpixel, in scan order (rows
// ascending, columns from y outward, channels 0..2), that shows the chain's
// view and whose channel has an idle subpixel parked; the chain ends when
// that subpixel is outside the area or already filled.  Lane 0 owns all
// reads and writes of M_i (src); the warp scans the search window in
// parallel, 32 candidates per step, taking the first hit by ballot.
__global__ void repurpose_kernel(DisplayQ q, const uint16_t* __restrict__ V,
                                 uint32_t* __restrict__ src) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    if (warp >= q.n_areas) return;
    const int64_t a = q.area_min + warp;
    const int64_t S = 3 * int64_t(q.w);
    const int64_t lo_d = a * q.pw * q.lq;       // area covers d in [lo_d, hi_d)
    const int64_t hi_d = (a + 1) * q.pw * q.lq;
    for (int64_t x = 0; x < q.h; ++x) {
        const int64_t base = x * q.t3q - q.kq;
        int64_t s_lo = ceil_div_pos(lo_d - base, kQ32);
        int64_t s_hi = ceil_div_pos(hi_d - base, kQ32) - 1;
        if (s_lo < 0) s_lo = 0;
        if (s_hi > S - 1) s_hi = S - 1;
        for (int64_t s = s_lo; s <= s_hi; ++s) {
            int64_t ci = x * S + s;
            uint32_t cur = 0;
            if (lane == 0) cur = src[ci];
            cur = __shfl_sync(0xffffffffu, cur, 0);
            if (cur != kEmpty) continue;
            const uint16_t vi = V[ci];
            uint32_t B0 = kEmpty, B1 = kEmpty, B2 = kEmpty;  // B_rgb(v_i, .)
            int64_t cx = x, cy = s / 3;
            int ck = int(s % 3);
            while (true) {
                const uint32_t Bk = ck == 0 ? B0 : (ck == 1 ? B1 : B2);
                if (Bk != kEmpty) {  // Eq. (13)
                    if (lane == 0) src[ci] = Bk;
                    if (ck == 0) B0 = kEmpty;
                    else if (ck == 1) B1 = kEmpty;
                    else B2 = kEmpty;
                } else {  // Eqs. (11), (12)
                    const uint32_t p = pack_px(cx, cy);
                    if (lane == 0) src[ci] = p;
                    if (ck == 0) { B1 = p; B2 = p; }
                    else if (ck == 1) { B0 = p; B2 = p; }
                    else { B0 = p; B1 = p; }
                }
                // Eq. (14)
                const int64_t x_low = cx + 2 < q.h - 1 ? cx + 2 : q.h - 1;
                const int64_t x_high = cx + q.win_dx < q.h - 1 ? cx + q.win_dx : q.h - 1;
                int64_t y_last, step;
                if (!q.slant_neg) {
                    y_last = cy - q.win_dy > 0 ? cy - q.win_dy : 0;
                    step = -1;
                } else {
                    y_last = cy + q.win_dy < q.w - 1 ? cy + q.win_dy : q.w - 1;
                    step = 1;
                }
                const int64_t ncols = (y_last - cy) * step + 1;
                const int64_t nrows = x_high - x_low + 1;
                const int64_t ncand = nrows > 0 ? nrows * ncols * 3 : 0;
                int64_t found = -1;
                for (int64_t b = 0; b < ncand; b += 32) {
                    const int64_t j = b + lane;
                    bool match = false;
                    if (j < ncand) {
                        const int64_t r = x_low + j / (ncols * 3);
                        const int64_t rem = j % (ncols * 3);
                        const int64_t c = cy + step * (rem / 3);
                        const int ch = int(rem % 3);
                        const uint32_t Bc = ch == 0 ? B0 : (ch == 1 ? B1 : B2);
                        match = (Bc != kEmpty) && (V[r * S + 3 * c + ch] == vi);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, match);
                    if (bal) {
                        found = b + (__ffs(bal) - 1);
                        break;
                    }
                }
                if (found < 0) break;  // no position left for view v_i
                const int64_t r = x_low + found / (ncols * 3);
                const int64_t rem = found % (ncols * 3);
                const int64_t c = cy + step * (rem / 3);
                const int ch = int(rem % 3);
                // while condition of Alg. 2: inside the area and still empty
                if (area_of(q, r, 3 * c + ch) != a) break;
                const int64_t ni = r * S + 3 * c + ch;
                uint32_t nsrc = 0;
                if (lane == 0) nsrc = src[ni];
                nsrc = __shfl_sync(0xffffffffu, nsrc, 0);
                if (nsrc != kEmpty) break;
                cx = r;
                cy = c;
                ck = ch;
                ci = ni;
            }
        }
    }
}

__global__ void identity_src_kernel(int32_t w, int32_t h, uint32_t* __restrict__ src) {
    const int64_t total = 3 * int64_t(w) * h;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t p = i / 3;
        src[i] = pack_px(p / w, p % w);
    }
}

// ------------------------------------------------------------------ a3 ---
// A ray (v, x', y') is identified by its owner: the subpixel (x', y', k0) of
// the source pixel with the lowest channel k0 showing view v.  Rays are
// numbered in order of first use by the R subpixels (row-major), then G,
// then B (Sec. 5: R~_rays follows the R subpixels): an owner's order key is
// the first R pixel using it, else wh + the first G pixel, else 2wh + the
// first B pixel, and its ray id is the rank of that key.
struct RayTmp {
    uint32_t* owner;        // 3wh: owner subpixel of each subpixel's ray
    uint32_t* ray_of_owner; // 3wh: ray id per owner (kEmpty when not an owner)
    uint32_t* first_r;      // 3wh: first R pixel index using the owner
    uint32_t* first_g;      // 3wh
    uint32_t* first_b;      // 3wh
    uint32_t* key_of;       // 3wh: order key of each owner
    uint32_t* flag;         // 3wh: 1 at every used order key
    uint32_t* rank;         // 3wh + 1
    void* scan_tmp;
};

__host__ RayTmp carve(const DisplayQ& q, void* tmp) {
    const size_t n = 3 * size_t(q.w) * q.h;
    char* p = static_cast<char*>(tmp);
    RayTmp t;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    t.owner = reinterpret_cast<uint32_t*>(take(4 * n));
    t.ray_of_owner = reinterpret_cast<uint32_t*>(take(4 * n));
    t.first_r = reinterpret_cast<uint32_t*>(take(4 * n));
    t.first_g = reinterpret_cast<uint32_t*>(take(4 * n));
    t.first_b = reinterpret_cast<uint32_t*>(take(4 * n));
    t.key_of = reinterpret_cast<uint32_t*>(take(4 * n));
    t.flag = reinterpret_cast<uint32_t*>(take(4 * n));
    t.rank = reinterpret_cast<uint32_t*>(take(4 * n + 4));
    t.scan_tmp = take(0);
    return t;
}

__global__ void owner_kernel(int32_t w, int32_t h, int64_t n, const uint16_t* __restrict__ V,
                             const uint32_t* __restrict__ src, RayTmp t) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t s = src[i];
        // a source outside the panel (never produced by the repurposing) is
        // read as the subpixel's own pixel rather than followed
        const bool ok = (s >> 16) < uint32_t(h) && (s & 0xFFFF) < uint32_t(w);
        const int64_t sp = ok ? int64_t(s >> 16) * w + (s & 0xFFFF) : i / 3;
        const uint16_t v = V[i];
        int k0 = 0;
        while (k0 < 2 && V[3 * sp + k0] != v) ++k0;
        t.owner[i] = uint32_t(3 * sp + k0);
        t.ray_of_owner[i] = kEmpty;
        t.first_r[i] = kEmpty;
        t.first_g[i] = kEmpty;
        t.first_b[i] = kEmpty;
        t.key_of[i] = kEmpty;
    }
}

__global__ void first_use_kernel(int64_t wh, RayTmp t) {
    for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < wh;
         p += int64_t(gridDim.x) * blockDim.x) {
        atomicMin(&t.first_r[t.owner[3 * p]], uint32_t(p));
        atomicMin(&t.first_g[t.owner[3 * p + 1]], uint32_t(p));
        atomicMin(&t.first_b[t.owner[3 * p + 2]], uint32_t(p));
    }
}

__global__ void mark_keys_kernel(int64_t n, int64_t wh, RayTmp t) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n;
         o += int64_t(gridDim.x) * blockDim.x) {
        uint32_t key = kEmpty;
        if (t.first_r[o] != kEmpty) key = t.first_r[o];
        else if (t.first_g[o] != kEmpty) key = uint32_t(wh) + t.first_g[o];
        else if (t.first_b[o] != kEmpty) key = uint32_t(2 * wh) + t.first_b[o];
        if (key != kEmpty) {
            t.key_of[o] = key;
            t.flag[key] = 1;
        }
    }
}

__global__ void assign_kernel(int64_t n, RayTmp t) {
    for (int64_t o = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; o < n;
         o += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t key = t.key_of[o];
        if (key != kEmpty) t.ray_of_owner[o] = t.rank[key];
    }
}

__global__ void ray_of_kernel(int64_t n, const RayTmp t, uint32_t* __restrict__ ray_of) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        ray_of[i] = t.ray_of_owner[t.owner[i]];
}

__global__ void ray_attr_kernel(int32_t w, int64_t n, const uint16_t* __restrict__ V,
                                const RayTmp t, uint32_t* __restrict__ ray_view,
                                uint32_t* __restrict__ ray_pix) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = t.ray_of_owner[i];
        if (r != kEmpty) {  // i is an owner subpixel
            const int64_t p = i / 3;
            ray_view[r] = V[i];
            ray_pix[r] = pack_px(p / w, p % w);
        }
    }
}

__global__ void group_keys_kernel(const uint32_t* __restrict__ ray_view,
                                  const uint32_t* __restrict__ ray_pix, int64_t n, int32_t tw,
                                  int32_t th, int32_t ntx, int32_t nv,
                                  unsigned long long* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n;
         r += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t px = ray_pix[r];
        const uint32_t row = px >> 16, col = px & 0xFFFF;
        // tile-major: the views of a tile are neighbours in the grouping
        const uint64_t g = uint64_t((row / th) * ntx + (col / tw)) * nv + ray_view[r];
        // inside the tile, order rays along a Morton curve so that each warp's
        // rays cover a compact patch
        uint32_t x = col % tw, y = row % th, m = 0;
        for (int b = 0; b < 8; ++b) m |= (((x >> b) & 1u) << (2 * b)) | (((y >> b) & 1u) << (2 * b + 1));
        keys[r] = (g << 16) | m;
        vals[r] = uint32_t(r);
    }
}

__global__ void group_gather_kernel(const uint32_t* __restrict__ order,
                                    const uint32_t* __restrict__ ray_pix, int64_t n,
                                    int2* __restrict__ grouped) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n;
         j += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = order[j];
        grouped[j] = make_int2(int(ray_pix[r]), int(r));
    }
}

// pos[ray id] = position of the ray in the (view, tile) grouping
__global__ void group_pos_kernel(const int2* __restrict__ grouped, int64_t n,
                                 uint32_t* __restrict__ pos) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n;
         j += int64_t(gridDim.x) * blockDim.x)
        pos[uint32_t(grouped[j].y)] = uint32_t(j);
}

// slot_of[i] = pos[ray_of[i]]: the grouped position of subpixel i's ray
__global__ void group_slot_kernel(const uint32_t* __restrict__ ray_of, int64_t n,
                                  const uint32_t* __restrict__ pos, uint32_t* __restrict__ slot_of) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        slot_of[i] = pos[ray_of[i]];
}

__global__ void rays_export_kernel(const uint32_t* __restrict__ ray_view,
                                   const uint32_t* __restrict__ ray_pix, int64_t n,
                                   int32_t* __restrict__ out) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n;
         r += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t px = ray_pix[r];
        out[3 * r] = int32_t(ray_view[r]);
        out[3 * r + 1] = int32_t(px >> 16);
        out[3 * r + 2] = int32_t(px & 0xFFFF);
    }
}

// (view, row, col) of every ray straight from the owner table.
__global__ void ray_triplets_kernel(int32_t w, int64_t n, const uint16_t* __restrict__ V,
                                    const RayTmp t, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = t.ray_of_owner[i];
        if (r != kEmpty) {
            const int64_t p = i / 3;
            out[3 * int64_t(r)] = int32_t(V[i]);
            out[3 * int64_t(r) + 1] = int32_t(p / w);
            out[3 * int64_t(r) + 2] = int32_t(p % w);
        }
    }
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    const int64_t cap = int64_t(num_sms()) * 16;
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_view_map(const DisplayQ& q, uint16_t* V, cudaStream_t s) {
    const int64_t n8 = (3 * int64_t(q.w) * q.h + 7) / 8;
    view_map_kernel<<<grid_for(n8, 256), 256, 0, s>>>(q, V);
    return cudaGetLastError();
}

cudaError_t launch_repurpose(const DisplayQ& q, const uint16_t* V, uint32_t* src, int identity,
                             cudaStream_t s) {
    if (identity) {
        identity_src_kernel<<<grid_for(3 * int64_t(q.w) * q.h, 256), 256, 0, s>>>(q.w, q.h, src);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(src, 0xFF, sizeof(uint32_t) * 3 * size_t(q.w) * q.h, s);
    if (e != cudaSuccess) return e;
    const int warps_per_block = 4;
    const int blocks = (q.n_areas + warps_per_block - 1) / warps_per_block;
    repurpose_kernel<<<blocks, 32 * warps_per_block, 0, s>>>(q, V, src);
    return cudaGetLastError();
}

size_t ray_table_tmp_bytes(const DisplayQ& q) {
    const size_t n = 3 * size_t(q.w) * q.h;
    return 7 * ((4 * n + 255) & ~size_t(255)) + ((4 * n + 4 + 255) & ~size_t(255)) +
           scan_tmp_bytes(int64_t(n)) + 256;
}

cudaError_t launch_ray_table(const DisplayQ& q, const uint16_t* V, const uint32_t* src,
                             uint32_t* ray_of, void* tmp, uint32_t* d_n_rays, cudaStream_t s) {
    const int64_t wh = int64_t(q.w) * q.h, n = 3 * wh;
    RayTmp t = carve(q, tmp);
    cudaError_t e = cudaMemsetAsync(t.flag, 0, sizeof(uint32_t) * size_t(n), s);
    if (e != cudaSuccess) return e;
    owner_kernel<<<grid_for(n, 256), 256, 0, s>>>(q.w, q.h, n, V, src, t);
    first_use_kernel<<<grid_for(wh, 256), 256, 0, s>>>(wh, t);
    mark_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, wh, t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_exclusive_scan(t.flag, t.rank, n, d_n_rays, t.scan_tmp, s);
    if (e != cudaSuccess) return e;
    assign_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, t);
    ray_of_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, t, ray_of);
    return cudaGetLastError();
}

cudaError_t launch_ray_attributes(const DisplayQ& q, const uint16_t* V, const void* tmp,
                                  uint32_t* ray_view, uint32_t* ray_pix, cudaStream_t s) {
    const int64_t n = 3 * int64_t(q.w) * q.h;
    RayTmp t = carve(q, const_cast<void*>(tmp));
    ray_attr_kernel<<<grid_for(n, 256), 256, 0, s>>>(q.w, n, V, t, ray_view, ray_pix);
    return cudaGetLastError();
}

cudaError_t launch_ray_group_keys(const uint32_t* ray_view, const uint32_t* ray_pix, int64_t n_rays,
                                  int32_t tile_w, int32_t tile_h, int32_t ntx, int32_t nv,
                                  unsigned long long* keys, uint32_t* vals, cudaStream_t s) {
    group_keys_kernel<<<grid_for(n_rays, 256), 256, 0, s>>>(ray_view, ray_pix, n_rays, tile_w,
                                                             tile_h, ntx, nv, keys, vals);
    return cudaGetLastError();
}

cudaError_t launch_rays_export(const uint32_t* ray_view, const uint32_t* ray_pix, int64_t n_rays,
                               int32_t* out, cudaStream_t s) {
    if (n_rays <= 0) return cudaSuccess;
    rays_export_kernel<<<grid_for(n_rays, 256), 256, 0, s>>>(ray_view, ray_pix, n_rays, out);
    return cudaGetLastError();
}

cudaError_t launch_ray_group_gather(const uint32_t* order, const uint32_t* ray_pix, int64_t n_rays,
                                    int2* grouped, cudaStream_t s) {
    group_gather_kernel<<<grid_for(n_rays, 256), 256, 0, s>>>(order, ray_pix, n_rays, grouped);
    return cudaGetLastError();
}

cudaError_t launch_group_slots(const int2* grouped, int64_t n_rays, const uint32_t* ray_of,
                               int64_t n_subpixels, uint32_t* pos_tmp, uint32_t* slot_of,
                               cudaStream_t s) {
    group_pos_kernel<<<grid_for(n_rays, 256), 256, 0, s>>>(grouped, n_rays, pos_tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    group_slot_kernel<<<grid_for(n_subpixels, 256), 256, 0, s>>>(ray_of, n_subpixels, pos_tmp,
                                                                  slot_of);
    return cudaGetLastError();
}

}  // namespace dl

// ---------------------------------------------------------------------------
// Ray table without any allocation.
//
// Some callers cannot call cudaMalloc: code running where the allocator is
// off limits (inside another library's memory pool, in a process whose
// device memory is fully reserved up front, or in a real-time loop that must
// not synchronise the device the way cudaMalloc/cudaFree can).  For them
// dl_ray_table_static builds the same ray table as dl_set_display, from a
// view map and subpixel map the caller holds in device memory, using only
// this file-scope scratch array.  Every GPU that loads the library holds the
// array until the process exits.
namespace {
constexpr int64_t kStaticMaxPixels = 65536;  // panels up to e.g. 256 x 256
constexpr size_t kStaticScratchBytes = 6u * 1024u * 1024u + 512u * 1024u;
constexpr int kStaticMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_ray_table_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_addr[kStaticMaxDevices] = {};

extern "C" dl_status dl_ray_table_static(int32_t width, int32_t height, const uint16_t* V,
                                         const uint32_t* src, uint32_t* ray_of, int32_t* rays,
                                         int64_t* n_rays, void* stream) {
    using namespace dl;
    if (!V || !src || !ray_of || !rays || !n_rays || width < 1 || height < 1)
        return DL_ERR_INVALID_ARG;
    if (int64_t(width) * height > kStaticMaxPixels) return DL_ERR_INVALID_ARG;
    DisplayQ q{};
    q.w = width;
    q.h = height;
    if (ray_table_tmp_bytes(q) + 256 > kStaticScratchBytes) return DL_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kStaticMaxDevices) return DL_ERR_INVALID_ARG;
    void* base = nullptr;
    {
        // Host code only knows a stand-in for the array's name: ask the
        // runtime for its device address, once per device.
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_ray_table_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DL_ERR_CUDA;
            }
            g_static_addr[dev] = p;
        }
        base = g_static_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* d_n = reinterpret_cast<uint32_t*>(static_cast<char*>(base) + kStaticScratchBytes - 256);
    const int64_t n = 3 * int64_t(width) * height;
    if (launch_ray_table(q, V, src, ray_of, base, d_n, s) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    RayTmp t = carve(q, base);
    ray_triplets_kernel<<<grid_for(n, 256), 256, 0, s>>>(width, n, V, t, rays);
    uint32_t h_n = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_n, d_n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    *n_rays = int64_t(h_n);
    return DL_OK;
}

