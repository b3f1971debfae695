// Multi-view 3DGS projection (Sec. 3.3, Eqs. (8)-(10)) and tile-key emission.
//
// One thread per Gaussian reads its attributes once (FP32 means; scale,
// rotation, opacity and SH in FP32/BF16/FP16), builds Sigma = R S S^T R^T once
// and then projects it into every view: camera transform, EWA 2D covariance
// Sigma' = J W Sigma W^T J^T + 0.3 I, conic, SH colour for the view's
// direction, and the tile rectangle that holds every pixel where alpha can
// reach 1/255.  All arithmetic is FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dl_internal.cuh"
#include "sh.cuh"

namespace dl {
namespace {

// Reciprocal to about one ulp (the PTX approximate reciprocal); its operands
// here are positive and well inside the normal range.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// SH coefficients of a thread's Gaussian, staged once in shared memory (its
// own column of float4, so a warp's loads are conflict-free) and read per
// visible view: this keeps them out of registers, and the kernel at 64
// registers and four blocks per SM.
template <int DEG>
constexpr int sh_float4() { return (3 * (DEG + 1) * (DEG + 1) + 3) / 4; }
constexpr int kProjectThreads = 256;

// What a Gaussian keeps across the views: its mean, Sigma = R S S^T R^T
// (Eq. (8), R from the normalised quaternion), log2 of its opacity and
// K = 2 ln(255 o), the squared Mahalanobis radius where alpha falls to 1/255.
struct GaussState {
    float mx, my, mz;
    float S00, S01, S02, S11, S12, S22;
    float log2o, K;
    bool vis;  // opacity above 1/255
};

template <typename T>
__device__ __forceinline__ GaussState load_gauss(const GaussiansView<T>& G, int64_t g) {
    GaussState s;
    s.mx = G.mean[3 * g];
    s.my = G.mean[3 * g + 1];
    s.mz = G.mean[3 * g + 2];
    float qw = to_f(G.rot[4 * g]), qx = to_f(G.rot[4 * g + 1]);
    float qy = to_f(G.rot[4 * g + 2]), qz = to_f(G.rot[4 * g + 3]);
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz),
                R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz),
                R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx),
                R22 = 1.f - 2.f * (qx * qx + qy * qy);
    const float s0 = __expf(2.f * to_f(G.log_scale[3 * g]));
    const float s1 = __expf(2.f * to_f(G.log_scale[3 * g + 1]));
    const float s2 = __expf(2.f * to_f(G.log_scale[3 * g + 2]));
    s.S00 = R00 * R00 * s0 + R01 * R01 * s1 + R02 * R02 * s2;
    s.S01 = R00 * R10 * s0 + R01 * R11 * s1 + R02 * R12 * s2;
    s.S02 = R00 * R20 * s0 + R01 * R21 * s1 + R02 * R22 * s2;
    s.S11 = R10 * R10 * s0 + R11 * R11 * s1 + R12 * R12 * s2;
    s.S12 = R10 * R20 * s0 + R11 * R21 * s1 + R12 * R22 * s2;
    s.S22 = R20 * R20 * s0 + R21 * R21 * s1 + R22 * R22 * s2;
    const float logit = to_f(G.opacity_logit[g]);
    const float opac = 1.f / (1.f + __expf(-logit));
    s.log2o = log2f(opac);
    s.vis = opac * 255.f > 1.f;
    s.K = s.vis ? 2.f * logf(255.f * opac) : 0.f;
    return s;
}

template <typename T, int DEG>
__device__ __forceinline__ void stage_sh(const GaussiansView<T>& G, int64_t g, float4* s_sh) {
    constexpr int NF = 3 * (DEG + 1) * (DEG + 1), NF4 = sh_float4<DEG>();
#pragma unroll
    for (int q = 0; q < NF4; ++q) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = 4 * q + k < NF ? to_f(G.sh[g * NF + 4 * q + k]) : 0.f;
        s_sh[q * kProjectThreads + threadIdx.x] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// A Gaussian in one view: the EWA 2D covariance (Eq. (9)), its projected
// mean and the pixel and tile rectangles that hold every pixel where alpha
// can reach 1/255.
struct Splat {
    float uc, vc, cxx, cxy, cyy, det;
    uint32_t rect_c, rect_r, dk;  // columns and rows (first | last << 16), depth key
    int tx0, tx1, ty0, ty1;
};

// False when the Gaussian is culled in this view (behind the near plane,
// alpha below 1/255, a degenerate covariance or off the screen).
__device__ __forceinline__ bool project_splat(const GaussState& s, const Cam& cam,
                                              const ProjectParams& p, Splat& o) {
    const float tx = cam.r[0] * s.mx + cam.r[1] * s.my + cam.r[2] * s.mz + cam.t[0];
    const float ty = cam.r[3] * s.mx + cam.r[4] * s.my + cam.r[5] * s.mz + cam.t[1];
    const float tz = cam.r[6] * s.mx + cam.r[7] * s.my + cam.r[8] * s.mz + cam.t[2];
    if (!(tz > 0.2f && s.vis)) return false;
    // EWA (Eq. (9)): T = J W, Sigma' = T Sigma T^T + 0.3 I
    const float iz = rcp_approx(tz);  // tz > 0.2
    // the clamp window follows a shifted principal point (off-axis views)
    const float sz = cam.shift_f;
    const float xz = fminf(fmaxf(tx * iz, -p.lim_x - sz), p.lim_x - sz);
    const float yz = fminf(fmaxf(ty * iz, -p.lim_y), p.lim_y);
    const float fz = p.focal * iz;
    const float j02 = -fz * xz, j12 = -fz * yz;
    const float T00 = fz * cam.r[0] + j02 * cam.r[6];
    const float T01 = fz * cam.r[1] + j02 * cam.r[7];
    const float T02 = fz * cam.r[2] + j02 * cam.r[8];
    const float T10 = fz * cam.r[3] + j12 * cam.r[6];
    const float T11 = fz * cam.r[4] + j12 * cam.r[7];
    const float T12 = fz * cam.r[5] + j12 * cam.r[8];
    const float a0 = T00 * s.S00 + T01 * s.S01 + T02 * s.S02;
    const float a1 = T00 * s.S01 + T01 * s.S11 + T02 * s.S12;
    const float a2 = T00 * s.S02 + T01 * s.S12 + T02 * s.S22;
    const float b0 = T10 * s.S00 + T11 * s.S01 + T12 * s.S02;
    const float b1 = T10 * s.S01 + T11 * s.S11 + T12 * s.S12;
    const float b2 = T10 * s.S02 + T11 * s.S12 + T12 * s.S22;
    o.cxx = a0 * T00 + a1 * T01 + a2 * T02 + 0.3f;
    o.cxy = a0 * T10 + a1 * T11 + a2 * T12;
    o.cyy = b0 * T10 + b1 * T11 + b2 * T12 + 0.3f;
    o.det = o.cxx * o.cyy - o.cxy * o.cxy;
    if (!(o.det > 0.f)) return false;
    o.uc = p.focal * tx * iz + cam.shift;
    o.vc = p.focal * ty * iz;
    // pixels where alpha >= 1/255 lie in the ellipse
    // d^T Sigma'^-1 d <= 2 ln(255 o); its bounding box:
    const float kx = s.K * o.cxx, ky = s.K * o.cyy;  // > 0
    const float rx = kx * rsqrtf(kx) * 1.0001f + 1e-3f;
    const float ry = ky * rsqrtf(ky) * 1.0001f + 1e-3f;
    const float c_lo = ceilf(o.uc + p.half_w - rx), c_hi = floorf(o.uc + p.half_w + rx);
    const float r_lo = ceilf(o.vc + p.half_h - ry), r_hi = floorf(o.vc + p.half_h + ry);
    if (!(c_hi >= 0.f && r_hi >= 0.f && c_lo <= float(p.width - 1) &&
          r_lo <= float(p.height - 1) && c_lo <= c_hi && r_lo <= r_hi))
        return false;
    const int ic0 = int(fmaxf(c_lo, 0.f)), ic1 = int(fminf(c_hi, float(p.width - 1)));
    const int ir0 = int(fmaxf(r_lo, 0.f)), ir1 = int(fminf(r_hi, float(p.height - 1)));
    o.tx0 = ic0 >> p.tile_sx;
    o.tx1 = ic1 >> p.tile_sx;
    o.ty0 = ir0 >> p.tile_sy;
    o.ty1 = ir1 >> p.tile_sy;
    o.rect_c = uint32_t(ic0) | (uint32_t(ic1) << 16);
    o.rect_r = uint32_t(ir0) | (uint32_t(ir1) << 16);
    const uint32_t dk = __float_as_uint(tz) - __float_as_uint(0.2f);
    o.dk = dk > 0x0FFFFFFFu ? 0x0FFFFFFFu : dk;
    return true;
}

// The 32-byte record of a Gaussian in a view: conic, log2 opacity and the
// colour of Eq. (10), SH at dir = normalise(mu - camera centre) with the
// coefficients from the thread's shared-memory column.
template <int DEG>
__device__ __forceinline__ void write_record(const GaussState& s, const Cam& cam, const Splat& o,
                                             const float4* s_sh, float4* rec) {
    constexpr int NF = 3 * (DEG + 1) * (DEG + 1), NF4 = sh_float4<DEG>();
    const float id = rcp_approx(o.det);  // det >= 0.09
    float dx = s.mx - cam.c[0], dy = s.my - cam.c[1], dz = s.mz - cam.c[2];
    const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dn; dy *= dn; dz *= dn;
    float Y[16];
    sh_basis<DEG>(dx, dy, dz, Y);
    // coefficient f = 3 i + c, in order of f: every channel sums its terms
    // in order of i
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < NF4; ++q) {
        const float4 w4 = s_sh[q * kProjectThreads + threadIdx.x];
        const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int f = 4 * q + k;
            if (f < NF) acc[f % 3] = fmaf(Y[f / 3], w[k], acc[f % 3]);
        }
    }
    float col[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) col[c] = fmaxf(acc[c] + 0.5f, 0.f);
    float clo, chi;
    pack_rgb(col[0], col[1], col[2], clo, chi);
    rec[0] = make_float4(o.uc, o.vc, -0.5f * kLog2e * o.cyy * id, kLog2e * o.cxy * id);
    rec[1] = make_float4(-0.5f * kLog2e * o.cxx * id, s.log2o, clo, chi);
}

template <typename T, int DEG>
__global__ void __launch_bounds__(kProjectThreads, 4) project_kernel(GaussiansView<T> G, ProjectParams p,
                                                      const Cam* __restrict__ cams, int32_t nv,
                                                      ProjectOut out) {
    extern __shared__ float4 s_sh[];  // [NF4][kProjectThreads]
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    unsigned long long my_total = 0;
    uint32_t my_visible = 0;
    if (g < p.n) {
        const GaussState gs = load_gauss(G, g);
        stage_sh<T, DEG>(G, g, s_sh);
        // warps start at different views (and wrap around), so warps in
        // flight add to the counters of different views' tiles
        int32_t v = int32_t((g >> 5) % nv);
        for (int32_t k = 0; k < nv; ++k, v = v + 1 == nv ? 0 : v + 1) {
            const Cam cam = load_cam(cams + v);
            const int64_t e = int64_t(v) * p.n + g;
            uint32_t cnt = 0;
            uint4 meta = make_uint4(0u, 0u, 0u, 0u);
            Splat sp;
            if (project_splat(gs, cam, p, sp)) {
                cnt = uint32_t(sp.tx1 - sp.tx0 + 1) * uint32_t(sp.ty1 - sp.ty0 + 1);
                if (out.gcount) {  // keys per (view, tile) group
                    const uint32_t vb = uint32_t(v) * uint32_t(p.ntx * p.nty);
                    const uint32_t g0 = vb + uint32_t(sp.ty0 * p.ntx + sp.tx0);
                    // the warp's Gaussians are neighbours in space: when
                    // every active lane covers the same single tile, one
                    // lane adds for all of them
                    const unsigned am = __activemask();
                    const bool single = sp.tx0 == sp.tx1 && sp.ty0 == sp.ty1;
                    const bool same = __all_sync(am, single) &&
                                      __reduce_min_sync(am, g0) == __reduce_max_sync(am, g0);
                    if (same) {
                        if ((threadIdx.x & 31) == __ffs(am) - 1) atomicAdd(out.gcount + g0, __popc(am));
                    } else {
                        for (int ty = sp.ty0; ty <= sp.ty1; ++ty)
                            for (int tx = sp.tx0; tx <= sp.tx1; ++tx)
                                atomicAdd(out.gcount + vb + uint32_t(ty * p.ntx + tx), 1u);
                    }
                }
                write_record<DEG>(gs, cam, sp, s_sh, out.rec + kRecordFloat4 * e);
                meta = make_uint4(sp.rect_c, sp.rect_r, sp.dk, cnt);
            }
            out.meta[e] = meta;
            my_total += cnt;
            my_visible += cnt ? 1u : 0u;
        }
    }
    // warp sum of the tile counts -> one 64-bit atomic per warp (no block
    // barrier: warps finish at different times)
    my_total = warp_sum(my_total);
    if ((threadIdx.x & 31) == 0 && my_total) atomicAdd(out.total, my_total);
    if (out.visible) {
        const unsigned long long vis = warp_sum((unsigned long long)my_visible);
        if ((threadIdx.x & 31) == 0 && vis) atomicAdd(out.visible, vis);
    }
}

// Key of a (view, tile, Gaussian) overlap: (view*ntiles + tile) << 28 | depth
// key, the depth key being the float bits of z minus those of 0.2 (z > 0.2,
// so the difference is positive and ordered like z; 28 bits reach z = 2^29).

// Tiles touched per (view, Gaussian), out of the metadata, for the scan that
// places the radix path's keys.
__global__ void meta_counts_kernel(const uint4* __restrict__ meta, int64_t n,
                                   uint32_t* __restrict__ count) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
         e += int64_t(gridDim.x) * blockDim.x)
        count[e] = meta[e].w;
}

__global__ void emit_keys_kernel(ProjectParams p, int32_t nv, const uint4* __restrict__ meta,
                                 const uint32_t* __restrict__ offset,
                                 unsigned long long* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
    const int64_t total = int64_t(nv) * p.n;
    const int ntiles = p.ntx * p.nty;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const uint4 m = meta[e];
        if (!m.w) continue;
        const uint32_t rx = m.x, ry = m.y, dk = m.z;
        const int tx0 = int(rx & 0xFFFF) >> p.tile_sx, tx1 = int(rx >> 16) >> p.tile_sx;
        const int ty0 = int(ry & 0xFFFF) >> p.tile_sy, ty1 = int(ry >> 16) >> p.tile_sy;
        const int64_t v = e / p.n;
        const uint32_t gidx = uint32_t(e - v * p.n);
        uint32_t o = offset[e];
        const unsigned long long vbase = (unsigned long long)(v * ntiles);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const unsigned long long grp = vbase + unsigned(ty * p.ntx + tx);
                keys[o] = (grp << 28) | dk;
                vals[o] = gidx;
                ++o;
            }
    }
}

// Binned emission: every (view, tile, Gaussian) key goes straight into its
// group's slice of the key array (slot from an atomic cursor); the order
// inside a group is fixed later by sorting the unique keys
// depth << 32 | index << 4 | quadrant bits.  Bit q of the low nibble marks
// that the Gaussian's pixel box overlaps quadrant q (x half + 2 * y half) of
// the tile, which the block class uses to split a group among its warps;
// the index is unique in a group, so the nibble never decides the order.
constexpr int kEmitRounds = 3;

// One warp's keys of one view: lane i holds a Gaussian touching cnt tiles
// (tiles [tx0, tx0 + span) x [ty0, ...), group base vb = view * tiles,
// key words khi = depth key, klo = index << 4, pixel box rect_c / rect_r).
// The warp expands its (Gaussian, tile) pairs into dense rounds of 32, so
// every lane emits a key per round and each round costs one cursor atomic
// per group it touches.  cursor[g] holds an absolute slot (it starts at the
// group's first).  CHECK: slots end at min(slice[g + 1], key_cap); a key
// past its group's end is not written and sets `over`.  Called by all 32
// lanes together.
template <bool CHECK>
__device__ __forceinline__ void warp_emit(const ProjectParams& p, uint32_t cnt, int tx0, int ty0,
                                          int span, uint32_t vb, uint32_t khi, uint32_t klo,
                                          uint32_t rect_c, uint32_t rect_r,
                                          uint32_t* __restrict__ cursor,
                                          const uint32_t* __restrict__ slice,
                                          unsigned long long* __restrict__ keys, uint32_t key_cap,
                                          bool& over) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t incl = cnt;  // inclusive scan of the pair counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t off = incl - cnt, n_pairs = __shfl_sync(0xffffffffu, incl, 31);
    if (n_pairs == 0) return;
    const float rspan = 1.0f / float(span);
    const int half_w = p.tile_w >> 1, half_h = p.tile_h >> 1;
    // pair pr -> its group and key (false past the last pair)
    auto pair_of = [&](uint32_t pr, uint32_t& grp, unsigned long long& key) {
        // owner: the last lane whose first pair is <= pr
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o2 = __shfl_sync(0xffffffffu, off, src + step);
            if (o2 <= pr) src += step;
        }
        const uint32_t k = pr - __shfl_sync(0xffffffffu, off, src);
        const int s_tx0 = __shfl_sync(0xffffffffu, tx0, src);
        const int s_ty0 = __shfl_sync(0xffffffffu, ty0, src);
        const int s_span = __shfl_sync(0xffffffffu, span, src);
        const float s_r = __shfl_sync(0xffffffffu, rspan, src);
        const uint32_t s_vb = __shfl_sync(0xffffffffu, vb, src);
        const uint32_t s_hi = __shfl_sync(0xffffffffu, khi, src);
        const uint32_t s_lo = __shfl_sync(0xffffffffu, klo, src);
        const uint32_t s_rc = __shfl_sync(0xffffffffu, rect_c, src);
        const uint32_t s_rr = __shfl_sync(0xffffffffu, rect_r, src);
        // k = dy * span + dx; the +0.5 keeps the float quotient's floor exact
        const int dy = int((float(k) + 0.5f) * s_r);
        const int dx = int(k) - dy * s_span;
        const int tx = s_tx0 + dx, ty = s_ty0 + dy;
        grp = s_vb + uint32_t(ty * p.ntx + tx);
        const int xm = tx * p.tile_w + half_w, ym = ty * p.tile_h + half_h;
        const uint32_t lo_x = int(s_rc & 0xFFFFu) < xm, hi_x = int(s_rc >> 16) >= xm;
        const uint32_t lo_y = int(s_rr & 0xFFFFu) < ym, hi_y = int(s_rr >> 16) >= ym;
        const uint32_t nib = (lo_x & lo_y) | ((hi_x & lo_y) << 1) | ((lo_x & hi_y) << 2) |
                             ((hi_x & hi_y) << 3);
        key = ((unsigned long long)s_hi << 32) | (s_lo | nib);
        return pr < n_pairs;
    };
    // kEmitRounds rounds of 32 pairs at once: their cursor atomics are in
    // flight together (the warp waits on the atomics' round trips)
    for (uint32_t r0 = 0; r0 < n_pairs; r0 += 32 * kEmitRounds) {
        uint32_t grp[kEmitRounds], base[kEmitRounds], end[kEmitRounds];
        unsigned long long key[kEmitRounds];
        unsigned peers[kEmitRounds];
        bool ok[kEmitRounds];
#pragma unroll
        for (int u = 0; u < kEmitRounds; ++u) {
            ok[u] = false;
            peers[u] = 0u;
            if (r0 + 32u * u < n_pairs) {  // warp-uniform
                ok[u] = pair_of(r0 + 32u * u + uint32_t(lane), grp[u], key[u]);
                peers[u] = __match_any_sync(0xffffffffu, ok[u] ? grp[u] : 0xFFFFFFFFu);
            }
        }
#pragma unroll
        for (int u = 0; u < kEmitRounds; ++u) {
            base[u] = 0u;
            end[u] = 0u;
            if (ok[u] && lane == __ffs(peers[u]) - 1) {
                if (CHECK) end[u] = min(__ldg(slice + grp[u] + 1), key_cap);
                base[u] = atomicAdd(cursor + grp[u], uint32_t(__popc(peers[u])));
            }
        }
#pragma unroll
        for (int u = 0; u < kEmitRounds; ++u) {
            if (r0 + 32u * u < n_pairs) {
                const int leader = __ffs(peers[u]) - 1;
                const uint32_t slot = __shfl_sync(0xffffffffu, base[u], leader) +
                                      uint32_t(__popc(peers[u] & lt));
                const uint32_t e = CHECK ? __shfl_sync(0xffffffffu, end[u], leader) : 0u;
                if (ok[u]) {
                    if (!CHECK || slot < e) keys[slot] = key[u];
                    else over = true;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256, 6) emit_binned_kernel(ProjectParams p, int32_t nv, const uint4* __restrict__ meta,
                                   uint32_t* __restrict__ cursor,
                                   unsigned long long* __restrict__ keys,
                                   const uint32_t* __restrict__ total_keys, uint32_t key_cap,
                                   uint32_t* __restrict__ status) {
    if (total_keys && *total_keys > key_cap) {  // the key slice does not fit
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 1u);
        return;
    }
    const int64_t total = int64_t(nv) * p.n;
    const int ntiles = p.ntx * p.nty;
    const float rn = 1.0f / float(p.n);
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    // each warp takes 32 consecutive records; the next iteration's metadata
    // is loaded one iteration ahead
    int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint4 m_next = make_uint4(0u, 0u, 0u, 0u);
    auto fetch = [&](int64_t ww) {
        const int64_t en = ww * 32 + lane;
        m_next = en < total ? __ldg(meta + en) : make_uint4(0u, 0u, 0u, 0u);
    };
    fetch(w);
    bool over = false;  // never set: the slices hold exactly their keys
    for (; w * 32 < total; w += warps) {
        const int64_t e = w * 32 + lane;
        const uint4 m = m_next;
        const uint32_t cnt = m.w;
        fetch(w + warps);
        int tx0 = 0, ty0 = 0, span = 1;
        uint32_t vb = 0, klo = 0;
        if (cnt) {
            tx0 = int(m.x & 0xFFFF) >> p.tile_sx;
            span = (int(m.x >> 16) >> p.tile_sx) - tx0 + 1;
            ty0 = int(m.y & 0xFFFF) >> p.tile_sy;
            // view and Gaussian of record e: a float quotient, corrected
            int64_t v = int64_t(float(e) * rn);
            int64_t gi = e - v * p.n;
            while (gi < 0) { --v; gi += p.n; }
            while (gi >= p.n) { ++v; gi -= p.n; }
            klo = uint32_t(gi) << 4;
            vb = uint32_t(v) * uint32_t(ntiles);
        }
        warp_emit<false>(p, cnt, tx0, ty0, span, vb, m.z, klo, m.x, m.y, cursor, nullptr, keys, 0u,
                         over);
    }
}

// Projection with the keys emitted in the same pass, into slices laid out
// before the frame (slice[g] .. slice[g + 1] for group g; cursor[g] starts
// at slice[g] and ends at slice[g] + the group's key count, whether or not
// every key fitted).  A key whose slice is full is not written and sets
// *overflow.  KEYS_ONLY (the pass that re-emits a frame into slices sized
// from its own counts) writes neither records nor totals, and runs only when
// *gate is set.  The Gaussian and view loops are those of project_kernel;
// every lane of a warp runs them (lanes past the last Gaussian cull every
// view), because the emission is warp-cooperative.
template <typename T, int DEG, bool KEYS_ONLY>
__global__ void __launch_bounds__(kProjectThreads, 4)
project_direct_kernel(GaussiansView<T> G, ProjectParams p, const Cam* __restrict__ cams, int32_t nv,
                      ProjectOut out) {
    if (KEYS_ONLY && *out.gate == 0u) return;
    extern __shared__ float4 s_sh[];  // [NF4][kProjectThreads]
    const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    unsigned long long my_total = 0;
    uint32_t my_visible = 0;
    GaussState gs{};
    gs.vis = false;
    if (g < p.n) {
        gs = load_gauss(G, g);
        if (!KEYS_ONLY) stage_sh<T, DEG>(G, g, s_sh);
    }
    const uint32_t ntiles = uint32_t(p.ntx * p.nty);
    bool over = false;
    // every warp walks the views in the same order, so the keys in flight
    // go to one or two views' slices, whose open ends stay in L2 (warps
    // that start at different views spread them over every view's slices:
    // 4 % slower at 4K, 4 % at 8K with 100 views)
    int32_t v = 0;
    for (int32_t k = 0; k < nv; ++k, v = v + 1 == nv ? 0 : v + 1) {
        const Cam cam = load_cam(cams + v);
        uint32_t cnt = 0;
        Splat sp;
        sp.tx0 = sp.ty0 = 0;
        sp.tx1 = sp.ty1 = 0;
        sp.rect_c = sp.rect_r = sp.dk = 0u;
        if (gs.vis && project_splat(gs, cam, p, sp)) {
            cnt = uint32_t(sp.tx1 - sp.tx0 + 1) * uint32_t(sp.ty1 - sp.ty0 + 1);
            if (!KEYS_ONLY)
                write_record<DEG>(gs, cam, sp, s_sh, out.rec + kRecordFloat4 * (int64_t(v) * p.n + g));
        }
        my_total += cnt;
        my_visible += cnt ? 1u : 0u;
        warp_emit<true>(p, cnt, sp.tx0, sp.ty0, sp.tx1 - sp.tx0 + 1, uint32_t(v) * ntiles, sp.dk,
                        uint32_t(g) << 4, sp.rect_c, sp.rect_r, out.cursor, out.slice, out.keys,
                        out.key_cap, over);
    }
    if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) atomicOr(out.overflow, 1u);
    if (!KEYS_ONLY) {
        my_total = warp_sum(my_total);
        if ((threadIdx.x & 31) == 0 && my_total) atomicAdd(out.total, my_total);
        const unsigned long long vis = warp_sum((unsigned long long)my_visible);
        if ((threadIdx.x & 31) == 0 && vis && out.visible) atomicAdd(out.visible, vis);
    }
}

// Slices for the next layout: group g gets its key count (cursor[g] -
// slice[g], or cursor[g] alone without a slice array) plus an eighth and
// 16 slots; entry n_groups is 0, so an exclusive scan of n_groups + 1
// entries ends with the total.
__global__ void pad_counts_kernel(const uint32_t* __restrict__ cursor,
                                  const uint32_t* __restrict__ slice, int64_t n_groups,
                                  uint32_t* __restrict__ padded) {
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g <= n_groups;
         g += int64_t(gridDim.x) * blockDim.x) {
        if (g == n_groups) {
            padded[g] = 0u;
        } else {
            const uint32_t c = cursor[g] - (slice ? slice[g] : 0u);
            padded[g] = c + (c >> 3) + 16u;
        }
    }
}

// cursor = start, only when *flag is set
__global__ void reset_cursor_kernel(const uint32_t* __restrict__ flag,
                                    const uint32_t* __restrict__ start, int64_t n_groups,
                                    uint32_t* __restrict__ cursor) {
    if (*flag == 0u) return;
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n_groups;
         g += int64_t(gridDim.x) * blockDim.x)
        cursor[g] = start[g];
}

__global__ void store_cams_kernel(CamBatch b, int32_t n, Cam* __restrict__ dst) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = b.cam[i];
}

}  // namespace

cudaError_t launch_store_cams(const CamBatch& b, int32_t n, Cam* dst, cudaStream_t s) {
    store_cams_kernel<<<1, kCamBatch, 0, s>>>(b, n, dst);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_project_t(const void* const* attrs, const ProjectParams& p,
                                    const Cam* cams, int32_t nv, ProjectOut out, cudaStream_t s) {
    GaussiansView<T> G;
    G.mean = static_cast<const float*>(attrs[0]);
    G.log_scale = static_cast<const T*>(attrs[1]);
    G.rot = static_cast<const T*>(attrs[2]);
    G.opacity_logit = static_cast<const T*>(attrs[3]);
    G.sh = static_cast<const T*>(attrs[4]);
    const int block = kProjectThreads;
    const int64_t grid = (p.n + block - 1) / block;
    auto smem = [](int deg) { return size_t(16) * kProjectThreads * size_t((3 * (deg + 1) * (deg + 1) + 3) / 4); };
    switch (p.sh_degree) {
        case 0: project_kernel<T, 0><<<unsigned(grid), block, smem(0), s>>>(G, p, cams, nv, out); break;
        case 1: project_kernel<T, 1><<<unsigned(grid), block, smem(1), s>>>(G, p, cams, nv, out); break;
        case 2: project_kernel<T, 2><<<unsigned(grid), block, smem(2), s>>>(G, p, cams, nv, out); break;
        default: project_kernel<T, 3><<<unsigned(grid), block, smem(3), s>>>(G, p, cams, nv, out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_project(int dtype, const void* const* attrs, const ProjectParams& p,
                           const Cam* cams, int32_t nv, ProjectOut out, cudaStream_t s) {
    if (dtype == 1) return launch_project_t<__nv_bfloat16>(attrs, p, cams, nv, out, s);
    if (dtype == 2) return launch_project_t<__half>(attrs, p, cams, nv, out, s);
    return launch_project_t<float>(attrs, p, cams, nv, out, s);
}

template <typename T>
static cudaError_t launch_project_direct_t(const void* const* attrs, const ProjectParams& p,
                                           const Cam* cams, int32_t nv, ProjectOut out,
                                           bool keys_only, cudaStream_t s) {
    GaussiansView<T> G;
    G.mean = static_cast<const float*>(attrs[0]);
    G.log_scale = static_cast<const T*>(attrs[1]);
    G.rot = static_cast<const T*>(attrs[2]);
    G.opacity_logit = static_cast<const T*>(attrs[3]);
    G.sh = static_cast<const T*>(attrs[4]);
    const int block = kProjectThreads;
    const int64_t grid = (p.n + block - 1) / block;
    if (grid <= 0) return cudaSuccess;
    auto smem = [](int deg) { return size_t(16) * kProjectThreads * size_t((3 * (deg + 1) * (deg + 1) + 3) / 4); };
    if (keys_only) {  // no colour: the SH degree does not matter
        project_direct_kernel<T, 0, true><<<unsigned(grid), block, 0, s>>>(G, p, cams, nv, out);
        return cudaGetLastError();
    }
    switch (p.sh_degree) {
        case 0: project_direct_kernel<T, 0, false><<<unsigned(grid), block, smem(0), s>>>(G, p, cams, nv, out); break;
        case 1: project_direct_kernel<T, 1, false><<<unsigned(grid), block, smem(1), s>>>(G, p, cams, nv, out); break;
        case 2: project_direct_kernel<T, 2, false><<<unsigned(grid), block, smem(2), s>>>(G, p, cams, nv, out); break;
        default: project_direct_kernel<T, 3, false><<<unsigned(grid), block, smem(3), s>>>(G, p, cams, nv, out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_project_direct(int dtype, const void* const* attrs, const ProjectParams& p,
                                  const Cam* cams, int32_t nv, ProjectOut out, bool keys_only,
                                  cudaStream_t s) {
    if (dtype == 1) return launch_project_direct_t<__nv_bfloat16>(attrs, p, cams, nv, out, keys_only, s);
    if (dtype == 2) return launch_project_direct_t<__half>(attrs, p, cams, nv, out, keys_only, s);
    return launch_project_direct_t<float>(attrs, p, cams, nv, out, keys_only, s);
}

cudaError_t launch_pad_counts(const uint32_t* cursor, const uint32_t* slice, int64_t n_groups,
                              uint32_t* padded, cudaStream_t s) {
    int64_t grid = (n_groups + 256) / 256;
    const int64_t cap = int64_t(num_sms()) * 16;
    if (grid > cap) grid = cap;
    pad_counts_kernel<<<unsigned(grid), 256, 0, s>>>(cursor, slice, n_groups, padded);
    return cudaGetLastError();
}

cudaError_t launch_reset_cursor(const uint32_t* flag, const uint32_t* start, int64_t n_groups,
                                uint32_t* cursor, cudaStream_t s) {
    int64_t grid = (n_groups + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 16;
    if (grid > cap) grid = cap;
    reset_cursor_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(flag, start, n_groups, cursor);
    return cudaGetLastError();
}

cudaError_t launch_emit_binned(const ProjectParams& p, int32_t nv, const uint4* meta,
                               uint32_t* cursor,
                               unsigned long long* keys, const uint32_t* total_keys,
                               uint32_t key_cap, uint32_t* status, cudaStream_t s) {
    const int64_t total = int64_t(nv) * p.n;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    emit_binned_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(p, nv, meta, cursor, keys,
                                                                     total_keys, key_cap, status);
    return cudaGetLastError();
}

cudaError_t launch_meta_counts(const uint4* meta, int64_t n, uint32_t* count, cudaStream_t s) {
    int64_t grid = (n + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    meta_counts_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(meta, n, count);
    return cudaGetLastError();
}

cudaError_t launch_emit_keys(const ProjectParams& p, int32_t nv, const uint4* meta,
                             const uint32_t* offset, unsigned long long* keys, uint32_t* vals,
                             cudaStream_t s) {
    const int64_t total = int64_t(nv) * p.n;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = int64_t(num_sms()) * 32;
    if (grid > cap) grid = cap;
    emit_keys_kernel<<<unsigned(grid > 0 ? grid : 1), 256, 0, s>>>(p, nv, meta, offset, keys, vals);
    return cudaGetLastError();
}

}  // namespace dl
