// Host side of the C ABI declared in include/directl.h: contexts, scenes,
// displays and the per-frame orchestration of the DirectL and standard paths.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "host.h"

using namespace dl;

namespace dl {

dl_status fail(dl_ctx* c, dl_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

dl_status cuda_fail(dl_ctx* c, cudaError_t e, const char* what) {
    const dl_status s = (e == cudaErrorMemoryAllocation) ? DL_ERR_OOM : DL_ERR_CUDA;
    return fail(c, s, "%s: %s", what, cudaGetErrorString(e));
}

int bits_for(int64_t n) {  // bits to hold values 0..n-1
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

int64_t floor_div_h(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

bool pow2_in(int32_t v, int32_t lo, int32_t hi) {
    return v >= lo && v <= hi && (v & (v - 1)) == 0;
}

// Q32 display constants (the display's exact definition) and the search
// range of Eq. (14): dx = floor(5 N_v / (2 L)), dy = ceil(N_v / (3 L)).
dl_status make_display_q(dl_ctx* ctx, const dl_display_params& p, DisplayQ* q) {
    if (p.width < 1 || p.height < 1 || p.width > 16384 || p.height > 16384)
        return fail(ctx, DL_ERR_INVALID_ARG, "panel size %dx%d out of range", p.width, p.height);
    if (p.rig != 0 && p.rig != 1) return fail(ctx, DL_ERR_INVALID_ARG, "rig %d", p.rig);
    if (p.num_views < 1 || p.num_views > 65535)
        return fail(ctx, DL_ERR_INVALID_ARG, "num_views %d out of range", p.num_views);
    if (p.p_w < 1) return fail(ctx, DL_ERR_INVALID_ARG, "p_w must be >= 1");
    if (!(p.pitch_lx > 0.0 && p.pitch_lx <= 1024.0))
        return fail(ctx, DL_ERR_INVALID_ARG, "pitch_lx out of (0, 1024]");
    if (!(std::fabs(p.tan_slant) <= 8.0) || !(std::fabs(p.offset_k) <= 1048576.0))
        return fail(ctx, DL_ERR_INVALID_ARG, "tan_slant or offset_k out of range");
    if (!(p.fov_x_deg > 0.0 && p.fov_x_deg < 179.0) || !(p.view_span_deg >= 0.0 && p.view_span_deg < 360.0))
        return fail(ctx, DL_ERR_INVALID_ARG, "fov_x_deg or view_span_deg out of range");
    const double q32 = 4294967296.0;
    q->w = p.width;
    q->h = p.height;
    q->nv = p.num_views;
    q->pw = p.p_w;
    q->t3q = int64_t(std::nearbyint(3.0 * p.tan_slant * q32));
    q->lq = int64_t(std::nearbyint(p.pitch_lx * q32));
    q->kq = int64_t(std::nearbyint(p.offset_k * q32));
    if (q->lq <= 0) return fail(ctx, DL_ERR_INVALID_ARG, "pitch_lx rounds to zero");
    q->win_dx = int32_t((5 * int64_t(p.num_views) * (int64_t(1) << 31)) / q->lq);
    q->win_dy = int32_t((int64_t(p.num_views) * (int64_t(1) << 32) + 3 * q->lq - 1) / (3 * q->lq));
    q->slant_neg = q->t3q < 0;
    // d_offset is monotone in the column and in the row, so its extremes sit
    // at the panel's corners.
    const int64_t S = 3 * int64_t(p.width);
    auto d = [&](int64_t x, int64_t s) { return s * (int64_t(1) << 32) + x * q->t3q - q->kq; };
    const int64_t dmin = std::min(d(0, 0), d(p.height - 1, 0));
    const int64_t dmax = std::max(d(0, S - 1), d(p.height - 1, S - 1));
    const int64_t amin = floor_div_h(floor_div_h(dmin, q->lq), p.p_w);
    const int64_t amax = floor_div_h(floor_div_h(dmax, q->lq), p.p_w);
    q->area_min = amin;
    q->n_areas = int32_t(amax - amin + 1);
    return DL_OK;
}

dl_status build_rayset(dl_ctx* ctx, Display& D, RaySet& R, bool identity, cudaStream_t s) {
    const DisplayQ& q = D.q;
    const size_t n = 3 * size_t(q.w) * q.h;
    DL_CK(R.src.reserve(4 * n), "alloc src");
    DL_CK(launch_repurpose(q, D.V.as<uint16_t>(), R.src.as<uint32_t>(), identity ? 1 : 0, s),
          "repurpose");
    DL_CK(R.ray_of.reserve(4 * n), "alloc ray_of");
    DevBuf tmp;
    DL_CK(tmp.reserve(ray_table_tmp_bytes(q)), "alloc ray-table scratch");
    DL_CK(ctx->ws.small.reserve(256), "alloc small");
    uint32_t* d_n = ctx->ws.small.as<uint32_t>();
    DL_CK(launch_ray_table(q, D.V.as<uint16_t>(), R.src.as<uint32_t>(), R.ray_of.as<uint32_t>(),
                           tmp.p, d_n, s),
          "ray table");
    uint32_t h_n = 0;
    DL_CK(cudaMemcpyAsync(&h_n, d_n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "copy");
    DL_CK(cudaStreamSynchronize(s), "sync");
    R.n_rays = int64_t(h_n);
    DL_CK(R.ray_view.reserve(4 * size_t(R.n_rays)), "alloc rays");
    DL_CK(R.ray_pix.reserve(4 * size_t(R.n_rays)), "alloc rays");
    DL_CK(launch_ray_attributes(q, D.V.as<uint16_t>(), tmp.p, R.ray_view.as<uint32_t>(),
                                R.ray_pix.as<uint32_t>(), s),
          "ray attributes");
    DL_CK(cudaStreamSynchronize(s), "sync");
    R.groups.clear();
    R.built = true;
    return DL_OK;
}

constexpr int kRaysPerBlock = 128;
// Tile lists of up to kSmallCap keys are sorted in a small shared-memory
// buffer; longer ones up to kLargeCap in one sized to the longest list; a
// frame with a longer list (or one whose buffer would not fit in shared
// memory) falls back to the global radix sort.
constexpr int kSmallCap = 1024;
constexpr int kLargeCap = 16384;

size_t max_smem_optin(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        cudaGetLastError();
        v = 48 * 1024;
    }
    return size_t(v);
}

// Rays of a ray set grouped by (view, tile) for one tile shape, and the work
// list of the DirectL compositing kernel (chunks of <= 128 rays).
dl_status get_groups(dl_ctx* ctx, Display& D, RaySet& R, int32_t tw, int32_t th, cudaStream_t s,
                     TileGroups** out) {
    const int64_t key = int64_t(tw) * 100000 + th;
    auto it = R.groups.find(key);
    if (it != R.groups.end()) {
        *out = it->second.get();
        return DL_OK;
    }
    auto G = std::make_unique<TileGroups>();
    G->tw = tw;
    G->th = th;
    G->ntx = (D.q.w + tw - 1) / tw;
    G->nty = (D.q.h + th - 1) / th;
    G->ntiles = G->ntx * G->nty;
    const int64_t ngroups = int64_t(D.q.nv) * G->ntiles;
    const int64_t nr = R.n_rays;
    DevBuf k0, k1, v0, v1, rtmp, ranges;
    DL_CK(k0.reserve(8 * size_t(nr)), "alloc");
    DL_CK(k1.reserve(8 * size_t(nr)), "alloc");
    DL_CK(v0.reserve(4 * size_t(nr)), "alloc");
    DL_CK(v1.reserve(4 * size_t(nr)), "alloc");
    DL_CK(rtmp.reserve(radix_tmp_bytes(nr)), "alloc");
    DL_CK(ranges.reserve(8 * size_t(ngroups)), "alloc");
    DL_CK(launch_ray_group_keys(R.ray_view.as<uint32_t>(), R.ray_pix.as<uint32_t>(), nr, tw, th,
                                G->ntx, D.q.nv, k0.as<unsigned long long>(), v0.as<uint32_t>(), s),
          "group keys");
    int alt = 0;
    DL_CK(radix_sort_pairs(k0.as<unsigned long long>(), v0.as<uint32_t>(),
                           k1.as<unsigned long long>(), v1.as<uint32_t>(), nr, bits_for(ngroups) + 16,
                           rtmp.p, &alt, s),
          "group sort");
    unsigned long long* ks = alt ? k1.as<unsigned long long>() : k0.as<unsigned long long>();
    uint32_t* vs = alt ? v1.as<uint32_t>() : v0.as<uint32_t>();
    DL_CK(cudaMemsetAsync(ranges.p, 0, 8 * size_t(ngroups), s), "memset");
    DL_CK(launch_key_ranges(ks, nr, 16, ranges.as<uint2>(), ngroups, s), "group ranges");
    DL_CK(G->grouped.reserve(8 * size_t(nr)), "alloc");
    DL_CK(launch_ray_group_gather(vs, R.ray_pix.as<uint32_t>(), nr, G->grouped.as<int2>(), s),
          "group gather");
    const int64_t nsub = 3 * int64_t(D.q.w) * D.q.h;
    DL_CK(G->slot_of.reserve(4 * size_t(nsub)), "alloc");
    DL_CK(launch_group_slots(G->grouped.as<int2>(), nr, R.ray_of.as<uint32_t>(), nsub,
                             alt ? v0.as<uint32_t>() : v1.as<uint32_t>(), G->slot_of.as<uint32_t>(),
                             s),
          "group slots");
    std::vector<uint2> h_ranges(static_cast<size_t>(ngroups));
    DL_CK(cudaMemcpyAsync(h_ranges.data(), ranges.p, 8 * size_t(ngroups), cudaMemcpyDeviceToHost, s),
          "copy");
    DL_CK(cudaStreamSynchronize(s), "sync");
    // h_ranges[tile * nv + v]: the rays of group g = v * ntiles + tile, in
    // the grouping's (tile-major) order
    const int64_t nv = D.q.nv;
    auto group_of = [&](int64_t k) { return (k % nv) * G->ntiles + k / nv; };
    std::vector<int4> work;
    work.reserve(size_t(nr / kRaysPerBlock + ngroups / 4 + 16));
    for (int64_t k = 0; k < ngroups; ++k) {
        const uint2 r = h_ranges[size_t(k)];
        const int64_t g = group_of(k);
        for (uint32_t b = r.x; b < r.y; b += kRaysPerBlock)
            work.push_back(make_int4(int(g), int(b), int(std::min<uint32_t>(b + kRaysPerBlock, r.y)), 0));
    }
    G->n_work = int64_t(work.size());
    DL_CK(G->work.reserve(16 * std::max<size_t>(work.size(), 1)), "alloc");
    if (!work.empty())
        DL_CK(cudaMemcpyAsync(G->work.p, work.data(), 16 * work.size(), cudaMemcpyHostToDevice, s),
              "copy");
    // the compositing items in view-major order: consecutive items are
    // neighbouring tiles of one view, which share records in L2 (tile-major
    // items measured 1.6 x the DRAM reads)
    std::vector<int4> gwork;
    for (int64_t g = 0; g < ngroups; ++g) {
        const int64_t k = (g % G->ntiles) * nv + g / G->ntiles;
        const uint2 r = h_ranges[size_t(k)];
        if (r.y > r.x) gwork.push_back(make_int4(int(g), int(r.x), int(r.y), 0));
    }
    G->n_gwork = int64_t(gwork.size());
    DL_CK(G->gwork.reserve(16 * std::max<size_t>(gwork.size(), 1)), "alloc");
    if (!gwork.empty())
        DL_CK(cudaMemcpyAsync(G->gwork.p, gwork.data(), 16 * gwork.size(), cudaMemcpyHostToDevice, s),
              "copy");
    DL_CK(cudaStreamSynchronize(s), "sync");
    *out = G.get();
    R.groups[key] = std::move(G);
    return DL_OK;
}

// View cameras: T_v = R_y(-theta_v) L0 (Eq. (17)); theta_v = -theta_d/2 +
// v theta_d/(N_v-1), view 0 the leftmost unless reverse_views.  Computed in
// double on the host, handed to the kernels as float world->camera matrices.
bool make_cams(const dl_display_params& p, const double L0[16], std::vector<Cam>& cams) {
    cams.resize(size_t(p.num_views));
    const double pi = 3.14159265358979323846;
    // off-axis rig: depth of the world origin in L0's camera
    const double D = -(L0[2] * L0[3] + L0[6] * L0[7] + L0[10] * L0[11]);
    const double focal = 0.5 * p.width / std::tan(0.5 * p.fov_x_deg * pi / 180.0);
    if (p.rig == 1 && !(D > 0.0)) return false;
    for (int32_t v = 0; v < p.num_views; ++v) {
        const int32_t vv = p.reverse_views ? p.num_views - 1 - v : v;
        double th = 0.0;
        if (p.num_views > 1)
            th = (-0.5 * p.view_span_deg + vv * p.view_span_deg / (p.num_views - 1)) * pi / 180.0;
        double T[3][4];
        double shift = 0.0;
        if (p.rig == 1) {  // L0 moved by D tan(theta) along its x axis
            const double xv = D * std::tan(th);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 4; ++j) T[i][j] = L0[4 * i + j] + (j == 3 ? xv * L0[4 * i] : 0.0);
            shift = focal * xv / D;
        } else {  // T_v = R_y(-theta_v) L0
            const double ph = -th, cs = std::cos(ph), sn = std::sin(ph);
            const double Ry[3][3] = {{cs, 0, sn}, {0, 1, 0}, {-sn, 0, cs}};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 4; ++j) {
                    double a = 0.0;
                    for (int k = 0; k < 3; ++k) a += Ry[i][k] * L0[4 * k + j];
                    T[i][j] = a;  // last row of L0 is (0,0,0,1): no contribution
                }
        }
        Cam& c = cams[size_t(v)];
        // world->camera: R_wc = R_cw^T, t = -R_cw^T centre
        for (int i = 0; i < 3; ++i) {
            c.c[i] = float(T[i][3]);
            double t = 0.0;
            for (int k = 0; k < 3; ++k) {
                c.r[3 * i + k] = float(T[k][i]);
                t -= T[k][i] * T[k][3];
            }
            c.t[i] = float(t);
        }
        c.shift = float(shift);
        c.shift_f = float(shift / focal);
    }
    return true;
}

dl_status upload_cams(dl_ctx* ctx, const std::vector<Cam>& cams, cudaStream_t s) {
    DL_CK(ctx->ws.cams.reserve(sizeof(Cam) * cams.size()), "alloc cams");
    Cam* dst = ctx->ws.cams.as<Cam>();
    for (size_t v0 = 0; v0 < cams.size(); v0 += kCamBatch) {
        CamBatch b;
        const int32_t n = int32_t(std::min<size_t>(kCamBatch, cams.size() - v0));
        std::memcpy(b.cam, cams.data() + v0, sizeof(Cam) * size_t(n));
        DL_CK(launch_store_cams(b, n, dst + v0, s), "store cams");
    }
    return DL_OK;
}

// Pinhole camera of Sec. 6: f = (w/2) / tan(fov_x/2), principal point (w/2,
// h/2); the Jacobian's clamp at 1.3 tan(fov/2) (3DGS practice).
ProjectParams make_project_params(const Scene& S, const Display& D, int32_t tw, int32_t th,
                                  int32_t rw, int32_t rh) {
    const int32_t w = rw > 0 ? rw : D.q.w, h = rh > 0 ? rh : D.q.h;
    const double pi = 3.14159265358979323846;
    const double focal = 0.5 * w / std::tan(0.5 * D.prm.fov_x_deg * pi / 180.0);
    ProjectParams pp{};
    pp.n = S.n;
    pp.sh_degree = S.sh_degree;
    pp.width = w;
    pp.height = h;
    pp.focal = float(focal);
    pp.half_w = 0.5f * float(w);
    pp.half_h = 0.5f * float(h);
    pp.lim_x = float(1.3 * (0.5 * w / focal));
    pp.lim_y = float(1.3 * (0.5 * h / focal));
    pp.tile_w = tw;
    pp.tile_h = th;
    pp.tile_sx = bits_for(tw);  // tw, th: powers of two
    pp.tile_sy = bits_for(th);
    pp.ntx = (w + tw - 1) / tw;
    pp.nty = (h + th - 1) / th;
    return pp;
}

dl_status check_ctx(dl_ctx* ctx) {
    if (!ctx) return DL_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return DL_OK;
}

size_t dtype_size(int32_t dt) { return dt == DL_F32 ? 4 : 2; }

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();  // leave no sticky error for the next launch check
        ms = 0.f;
    }
    return ms;
}

// Per-Gaussian data and the 8-wide SAH tree of the ray-order renderer.
dl_status build_raycast(dl_ctx* ctx, Scene& S, cudaStream_t s) {
    DL_CK(S.rc_gauss.reserve(48 * size_t(std::max<int64_t>(S.n, 1))), "alloc ray-order data");
    DL_CK(S.rc_gbox.reserve(32 * size_t(std::max<int64_t>(S.n, 1))), "alloc ray-order boxes");
    const void* attrs[5] = {S.mean.p, S.log_scale.p, S.rot.p, S.opacity.p, S.sh.p};
    DL_CK(launch_raycast_prepare(S.dtype, attrs, S.n, S.rc_gauss.as<float4>(), S.rc_gbox.as<float4>(), s),
          "ray-order preparation");
    DevBuf tmp;
    DL_CK(tmp.reserve(raycast_build_tmp_bytes(S.n)), "alloc tree build");
    int64_t n_bin = 0;
    DL_CK(raycast_build_binary(S.rc_gbox.as<float4>(), S.n, tmp.p, &n_bin, s), "SAH tree");
    DL_CK(S.rc_nodes.reserve(sizeof(RayNode) * size_t(std::max<int64_t>(n_bin, 1))), "alloc tree");
    int64_t n_wide = 0;
    int depth = 0;
    DL_CK(raycast_collapse(S.rc_gbox.as<float4>(), S.n, tmp.p, n_bin, S.rc_nodes.as<RayNode>(), &n_wide,
                           &depth, s),
          "8-wide tree");
    if (depth > kMaxWideDepth)
        return fail(ctx, DL_ERR_CAPACITY, "ray-order tree of %d wide levels (limit %d)", depth,
                    kMaxWideDepth);
    S.rc_depth = depth;
    S.rc_n_nodes = n_wide;
    S.rc_built = true;
    return DL_OK;
}

// The counter block of a frame run on device counters (copied from the
// workspace's 256-byte block: keys and visible records as u64 at bytes 0 and
// 8; at byte 64 the end of the key slices (the exact key total, or with the
// keys emitted by the projection the end of the next frame's slices) and
// the re-emission flag; the list-class words {warp items, block items,
// longest list, -, 1024-key items, cursors, status} from byte 128): fills
// the frame's statistics and resets its signature's sizing when the frame
// was dropped or used more than 85 % of a capacity.
static void apply_readback(dl_ctx* ctx, Readback& r) {
    Workspace& W = ctx->ws;
    const unsigned long long* h = r.h;
    const char* hb = reinterpret_cast<const char*>(h);
    const uint32_t* m = reinterpret_cast<const uint32_t*>(hb + 128);
    const uint32_t* t32 = reinterpret_cast<const uint32_t*>(hb + 64);
    const int64_t nkeys = int64_t(h[0]), vis = int64_t(h[1]), slice_end = int64_t(t32[0]);
    const int32_t reemitted = t32[1] != 0u ? 1 : 0;
    const int64_t lists_small = int64_t(m[0]) + int64_t(m[4]), lists_large = m[1], longest = m[2];
    const int32_t status = int32_t(m[7]);
    if (r.hint && (status != 0 || nkeys * 100 > r.hint->key_cap * 85 ||
                   slice_end * 100 > r.hint->key_cap * 85 ||
                   longest * 100 > int64_t(r.hint->block_cap) * 85))
        r.hint->sized = false;
    if (status != 0) ++W.dropped;
    for (PendingFrame& f : W.pending)
        if (f.frame == r.frame) {
            f.n_keys = nkeys;
            f.n_visible = vis;
            f.lists_small = lists_small;
            f.lists_large = lists_large;
            f.max_list = longest;
            f.status = status;
            f.reemitted = reemitted;
        }
    if (W.last_async == r.frame) {
        dl_frame_stats& fs = ctx->stats;
        fs.n_keys = nkeys;
        fs.n_visible = vis;
        fs.lists_small = lists_small;
        fs.lists_large = lists_large;
        fs.max_list = longest;
        fs.status = status;
        fs.reemitted = reemitted;
        W.last_async = -1;
    }
    r.busy = false;
}

dl_status harvest_readbacks(dl_ctx* ctx, bool wait) {
    for (Readback& r : ctx->ws.rb) {
        if (!r.busy) continue;
        if (wait) {
            DL_CK(cudaEventSynchronize(r.done), "wait for frame counters");
        } else {
            const cudaError_t e = cudaEventQuery(r.done);
            if (e == cudaErrorNotReady) {
                cudaGetLastError();
                continue;
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "frame counters");
        }
        apply_readback(ctx, r);
    }
    return DL_OK;
}

// Where a frame's last kernel writes it, by output kind: the caller's device
// buffer; the workspace frame, copied to the host on `s` (the call waits for
// it); or one of two device frames used in turn, copied to the host on the
// caller's copy stream so that the copy overlaps the next frame.  A frame
// reused by the asynchronous kind waits (on `s`) for the copy that read it two
// calls earlier.
enum OutKind : int32_t { kOutHost = 0, kOutDevice = 1, kOutHostAsync = 2 };

dl_status out_target(dl_ctx* ctx, float* out, int32_t kind, size_t bytes, cudaStream_t s,
                     float** dst) {
    Workspace& W = ctx->ws;
    if (kind == kOutDevice) {
        *dst = out;
        return DL_OK;
    }
    if (kind == kOutHost) {
        DL_CK(W.out.reserve(bytes), "alloc out");
        *dst = W.out.as<float>();
        return DL_OK;
    }
    const int k = W.aslot;
    for (int i = 0; i < 2; ++i) {
        if (!W.ev_frame[i]) DL_CK(cudaEventCreateWithFlags(&W.ev_frame[i], cudaEventDisableTiming), "event");
        if (!W.ev_copied[i]) DL_CK(cudaEventCreateWithFlags(&W.ev_copied[i], cudaEventDisableTiming), "event");
    }
    if (W.copy_pending[k]) {
        if (W.aout[k].bytes < bytes)  // the frame is replaced: its copy must have ended
            DL_CK(cudaEventSynchronize(W.ev_copied[k]), "wait for an earlier copy");
        else
            DL_CK(cudaStreamWaitEvent(s, W.ev_copied[k], 0), "order after an earlier copy");
    }
    DL_CK(W.aout[k].reserve(bytes), "alloc out");
    *dst = W.aout[k].as<float>();
    return DL_OK;
}

// After the frame's last kernel: the copy to the host (kinds kOutHost and
// kOutHostAsync); kOutHost's synchronisation is the caller's last step.
dl_status out_finish(dl_ctx* ctx, float* out, int32_t kind, const float* dst, size_t bytes,
                     cudaStream_t s, cudaStream_t cs) {
    Workspace& W = ctx->ws;
    if (kind == kOutHost) {
        DL_CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s), "copy frame");
    } else if (kind == kOutHostAsync) {
        const int k = W.aslot;
        DL_CK(cudaEventRecord(W.ev_frame[k], s), "event");
        DL_CK(cudaStreamWaitEvent(cs, W.ev_frame[k], 0), "order the copy after the frame");
        DL_CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, cs), "copy frame");
        DL_CK(cudaEventRecord(W.ev_copied[k], cs), "event");
        W.copy_pending[k] = true;
        W.aslot = k ^ 1;
    }
    return DL_OK;
}

// DL_RAYCAST frame: the DirectL rays cast through the scene (Alg. 3), then
// the ray colours gathered into the encoded image.  E: stage events (when
// stage timing is on), the unused stages recorded empty.
dl_status render_raycast(dl_ctx* ctx, Scene& S, Display& D, const double L0_c2w[16], float* out,
                         int32_t kind, cudaStream_t s, cudaStream_t cs, StageEvents* E) {
    Workspace& W = ctx->ws;
    auto mark = [&](int i) -> cudaError_t { return E ? cudaEventRecord(E->e[i], s) : cudaSuccess; };
    RaySet& R = D.rep;
    const int32_t w = D.q.w, h = D.q.h;
    std::vector<Cam> cams;
    if (!make_cams(D.prm, L0_c2w, cams))
        return fail(ctx, DL_ERR_INVALID_ARG, "off-axis rig: the world origin is not in front of L0");
    dl_status st = upload_cams(ctx, cams, s);
    if (st) return st;
    if (!S.rc_built) {
        st = build_raycast(ctx, S, s);
        if (st) return st;
    }
    // the rays in DirectL's (view, tile) grouping: coherent warps
    TileGroups* G = nullptr;
    st = get_groups(ctx, D, R, ctx->tile[DL_DIRECTL][0], ctx->tile[DL_DIRECTL][1], s, &G);
    if (st) return st;
    for (int i = 1; i <= 6; ++i) DL_CK(mark(i), "event");
    DL_CK(W.raycol.reserve(12 * size_t(R.n_rays > 0 ? R.n_rays : 1)), "alloc ray colours");
    const double pi = 3.14159265358979323846;
    const double focal = 0.5 * w / std::tan(0.5 * D.prm.fov_x_deg * pi / 180.0);
    DL_CK(launch_raycast(S.dtype, S.sh_degree, S.rc_gauss.as<float4>(), S.rc_nodes.as<RayNode>(),
                         S.n, S.sh.p, R.ray_view.as<uint32_t>(),
                         R.ray_pix.as<uint32_t>(), G->grouped.as<int2>(), R.n_rays, W.cams.as<Cam>(), float(focal),
                         0.5f * float(w), 0.5f * float(h), ctx->heap_cap, W.raycol.as<float>(), s),
          "ray-order rendering");
    DL_CK(mark(7), "event");
    const size_t out_bytes = 12 * size_t(w) * size_t(h);
    float* dst = nullptr;
    st = out_target(ctx, out, kind, out_bytes, s, &dst);
    if (st) return st;
    DL_CK(launch_reorder(G->slot_of.as<uint32_t>(), W.raycol.as<float>(), 3 * int64_t(w) * h, dst,
                         nullptr, s),
          "reorder");
    DL_CK(mark(8), "event");
    st = out_finish(ctx, out, kind, dst, out_bytes, s, cs);
    if (st) return st;
    dl_frame_stats& fs = ctx->stats;
    fs = dl_frame_stats{};
    W.last_async = -1;
    fs.n_rays = R.n_rays;
    fs.n_launches = int32_t((D.q.nv + kCamBatch - 1) / kCamBatch) + 2;
    if (E) {
        PendingFrame& pf = W.pending.back();
        pf.n_rays = fs.n_rays;
        pf.launches = fs.n_launches;
    }
    W.last_bytes = W.footprint();
    if (kind == kOutHost) DL_CK(cudaStreamSynchronize(s), "sync");
    return DL_OK;
}

// One frame of dl_render_frame / dl_render_frame_async_host (output kinds
// above; `cs` is the copy stream of kOutHostAsync).
dl_status render_frame(dl_ctx* ctx, int32_t scene_id, int32_t display_id, const double L0_c2w[16],
                       int32_t mode, float* out, int32_t kind, cudaStream_t s, cudaStream_t cs);

}  // namespace dl

extern "C" {

const char* dl_status_string(dl_status s) {
    switch (s) {
        case DL_OK: return "DL_OK";
        case DL_ERR_INVALID_ARG: return "DL_ERR_INVALID_ARG";
        case DL_ERR_OOM: return "DL_ERR_OOM";
        case DL_ERR_CUDA: return "DL_ERR_CUDA";
        case DL_ERR_NOT_FOUND: return "DL_ERR_NOT_FOUND";
        case DL_ERR_TIMEOUT: return "DL_ERR_TIMEOUT";
        case DL_ERR_DEVICE_CHECK: return "DL_ERR_DEVICE_CHECK";
        case DL_ERR_CAPACITY: return "DL_ERR_CAPACITY";
        default: return "DL_ERR_UNKNOWN";
    }
}

dl_status dl_create(dl_ctx** out, int32_t device) {
    if (!out) return DL_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DL_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
        cudaGetLastError();
        return DL_ERR_CUDA;
    }
    dl_ctx* c = new (std::nothrow) dl_ctx();
    if (!c) return DL_ERR_OOM;
    c->device = device;
    if (cudaMallocHost(&c->ws.h_total, 256) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DL_ERR_OOM;
    }
    for (dl::Readback& r : c->ws.rb) {
        if (cudaMallocHost(&r.h, 256) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return DL_ERR_OOM;
        }
    }
    *out = c;
    return DL_OK;
}

dl_status dl_destroy(dl_ctx* ctx) {
    if (!ctx) return DL_ERR_INVALID_ARG;
    if (ctx->n_batches > 0)
        return fail(ctx, DL_ERR_INVALID_ARG, "%d batch(es) still exist", ctx->n_batches);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    delete ctx;
    return DL_OK;
}

dl_status dl_last_error_detail(dl_ctx* ctx, char* buf, size_t len) {
    if (!ctx || !buf || len == 0) return DL_ERR_INVALID_ARG;
    std::snprintf(buf, len, "%s", ctx->err.c_str());
    return DL_OK;
}

dl_status dl_load_gaussians(dl_ctx* ctx, const dl_gaussians_desc* d, void* stream,
                            int32_t* scene_id) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!d || !scene_id || !d->mean || !d->log_scale || !d->rot_wxyz || !d->opacity_logit || !d->sh)
        return fail(ctx, DL_ERR_INVALID_ARG, "null argument");
    if (d->n < 1 || d->n > (int64_t(1) << 28))
        return fail(ctx, DL_ERR_INVALID_ARG, "n = %lld out of [1, 2^28]", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3)
        return fail(ctx, DL_ERR_INVALID_ARG, "sh_degree %d out of [0, 3]", d->sh_degree);
    if (d->dtype != DL_F32 && d->dtype != DL_BF16 && d->dtype != DL_F16)
        return fail(ctx, DL_ERR_INVALID_ARG, "unknown dtype %d", d->dtype);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto sc = std::make_unique<Scene>();
    sc->n = d->n;
    sc->sh_degree = d->sh_degree;
    sc->dtype = d->dtype;
    const size_t n = size_t(d->n), es = dtype_size(d->dtype);
    const size_t nc = size_t((d->sh_degree + 1) * (d->sh_degree + 1));
    const cudaMemcpyKind kind = d->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    struct {
        DevBuf* b;
        const void* src;
        size_t bytes;
    } parts[5] = {{&sc->mean, d->mean, 12 * n},
                  {&sc->log_scale, d->log_scale, 3 * es * n},
                  {&sc->rot, d->rot_wxyz, 4 * es * n},
                  {&sc->opacity, d->opacity_logit, es * n},
                  {&sc->sh, d->sh, 3 * nc * es * n}};
    for (auto& pt : parts) {
        DL_CK(pt.b->reserve(pt.bytes), "alloc scene");
        DL_CK(cudaMemcpyAsync(pt.b->p, pt.src, pt.bytes, kind, s), "copy scene");
    }
    if (sc->n > 1) {
        // Morton order of the means (see scene.cu)
        DevBuf tmp;
        DL_CK(tmp.reserve(spatial_order_tmp_bytes(sc->n)), "alloc reorder scratch");
        uint32_t* perm = nullptr;
        DL_CK(launch_spatial_order(sc->mean.as<float>(), sc->n, tmp.p, &perm, s), "spatial order");
        for (auto& pt : parts) {
            DevBuf sorted;
            DL_CK(sorted.reserve(pt.bytes), "alloc scene");
            DL_CK(launch_gather_records(pt.b->p, sorted.p, perm, sc->n, pt.bytes / n, s), "gather");
            std::swap(pt.b->p, sorted.p);
            std::swap(pt.b->bytes, sorted.bytes);
            DL_CK(cudaStreamSynchronize(s), "sync");
        }
    }
    if (!d->on_device) DL_CK(cudaStreamSynchronize(s), "sync");
    const int32_t id = ctx->next_id++;
    ctx->scenes[id] = std::move(sc);
    *scene_id = id;
    return DL_OK;
}

// Drops the capacities and key slices of the frame signatures that name a
// freed scene (field 0) or display (field 1); pending counter readbacks stop
// pointing at them.
static void drop_hints(dl_ctx* ctx, int field, int32_t id) {
    for (auto it = ctx->hints.begin(); it != ctx->hints.end();) {
        if (it->first[size_t(field)] == id) {
            for (Readback& r : ctx->ws.rb)
                if (r.hint == &it->second) r.hint = nullptr;
            it = ctx->hints.erase(it);
        } else {
            ++it;
        }
    }
}

dl_status dl_free_scene(dl_ctx* ctx, int32_t scene_id) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return fail(ctx, DL_ERR_NOT_FOUND, "scene %d", scene_id);
    if (it->second->in_use)
        return fail(ctx, DL_ERR_INVALID_ARG, "scene %d is assigned to %d batch slot(s)", scene_id,
                    it->second->in_use);
    cudaDeviceSynchronize();
    ctx->scenes.erase(it);
    drop_hints(ctx, 0, scene_id);
    return DL_OK;
}

dl_status dl_set_display(dl_ctx* ctx, const dl_display_params* params, void* stream,
                         int32_t* display_id) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!params || !display_id) return fail(ctx, DL_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto D = std::make_unique<Display>();
    D->prm = *params;
    st = make_display_q(ctx, D->prm, &D->q);
    if (st) return st;
    const size_t n = 3 * size_t(D->q.w) * D->q.h;
    DL_CK(D->V.reserve(2 * n), "alloc V");
    DL_CK(launch_view_map(D->q, D->V.as<uint16_t>(), s), "view map");
    st = build_rayset(ctx, *D, D->rep, D->prm.repurpose == 0, s);
    if (st) return st;
    TileGroups* G = nullptr;
    st = get_groups(ctx, *D, D->rep, ctx->tile[DL_DIRECTL][0], ctx->tile[DL_DIRECTL][1], s, &G);
    if (st) return st;
    const int32_t id = ctx->next_id++;
    ctx->displays[id] = std::move(D);
    *display_id = id;
    return DL_OK;
}

dl_status dl_free_display(dl_ctx* ctx, int32_t display_id) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    if (it->second->in_use)
        return fail(ctx, DL_ERR_INVALID_ARG, "display %d is assigned to %d batch slot(s)",
                    display_id, it->second->in_use);
    cudaDeviceSynchronize();
    ctx->displays.erase(it);
    drop_hints(ctx, 1, display_id);
    return DL_OK;
}

dl_status dl_display_info(dl_ctx* ctx, int32_t display_id, int64_t* n_rays, double* beta) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    const Display& D = *it->second;
    if (n_rays) *n_rays = D.rep.n_rays;
    if (beta) *beta = double(D.rep.n_rays) / (double(D.q.w) * D.q.h);
    return DL_OK;
}

static dl_status copy_out(dl_ctx* ctx, void* dst, const void* src, size_t bytes, int32_t on_device,
                          cudaStream_t s) {
    DL_CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s),
          "copy out");
    if (!on_device) DL_CK(cudaStreamSynchronize(s), "sync");
    return DL_OK;
}

dl_status dl_get_view_map(dl_ctx* ctx, int32_t display_id, uint16_t* out, int32_t out_on_device,
                          void* stream) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    if (!out) return fail(ctx, DL_ERR_INVALID_ARG, "null out");
    const Display& D = *it->second;
    return copy_out(ctx, out, D.V.p, 2 * 3 * size_t(D.q.w) * D.q.h, out_on_device,
                    static_cast<cudaStream_t>(stream));
}

dl_status dl_get_subpixel_map(dl_ctx* ctx, int32_t display_id, uint32_t* out,
                              int32_t out_on_device, void* stream) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    if (!out) return fail(ctx, DL_ERR_INVALID_ARG, "null out");
    const Display& D = *it->second;
    return copy_out(ctx, out, D.rep.src.p, 4 * 3 * size_t(D.q.w) * D.q.h, out_on_device,
                    static_cast<cudaStream_t>(stream));
}

dl_status dl_get_ray_table(dl_ctx* ctx, int32_t display_id, uint32_t* ray_of, int32_t* rays,
                           int32_t out_on_device, void* stream) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    const Display& D = *it->second;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ray_of) {
        st = copy_out(ctx, ray_of, D.rep.ray_of.p, 4 * 3 * size_t(D.q.w) * D.q.h, out_on_device, s);
        if (st) return st;
    }
    if (rays) {
        const size_t bytes = 12 * size_t(D.rep.n_rays);
        if (out_on_device) {
            DL_CK(launch_rays_export(D.rep.ray_view.as<uint32_t>(), D.rep.ray_pix.as<uint32_t>(),
                                     D.rep.n_rays, rays, s),
                  "rays export");
        } else {
            DevBuf tmp;
            DL_CK(tmp.reserve(bytes), "alloc");
            DL_CK(launch_rays_export(D.rep.ray_view.as<uint32_t>(), D.rep.ray_pix.as<uint32_t>(),
                                     D.rep.n_rays, tmp.as<int32_t>(), s),
                  "rays export");
            st = copy_out(ctx, rays, tmp.p, bytes, 0, s);
            if (st) return st;
        }
    }
    return DL_OK;
}

dl_status dl_encode_rays(dl_ctx* ctx, int32_t display_id, const float* ray_rgb, float* out,
                         void* stream) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!ray_rgb || !out) return fail(ctx, DL_ERR_INVALID_ARG, "null argument");
    auto it = ctx->displays.find(display_id);
    if (it == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    const Display& D = *it->second;
    DL_CK(launch_reorder(D.rep.ray_of.as<uint32_t>(), ray_rgb, 3 * int64_t(D.q.w) * D.q.h, out,
                         nullptr, static_cast<cudaStream_t>(stream)),
          "encode rays");
    return DL_OK;
}

dl_status dl_set_tile(dl_ctx* ctx, int32_t mode, int32_t tile_w, int32_t tile_h) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (mode == DL_STANDARD_SR) mode = DL_STANDARD;  // the same rendering
    if (mode < 0 || mode > 2) return fail(ctx, DL_ERR_INVALID_ARG, "mode %d", mode);
    if (!pow2_in(tile_w, 8, 256) || !pow2_in(tile_h, 8, 256))
        return fail(ctx, DL_ERR_INVALID_ARG, "tile %dx%d: powers of two in [8, 256]", tile_w, tile_h);
    if (mode == DL_STANDARD && tile_w * tile_h > 1024)
        return fail(ctx, DL_ERR_INVALID_ARG, "standard tiles hold at most 1024 pixels");
    ctx->tile[mode][0] = tile_w;
    ctx->tile[mode][1] = tile_h;
    return DL_OK;
}

dl_status dl_set_option(dl_ctx* ctx, int32_t option, int64_t value) {
    if (!ctx) return DL_ERR_INVALID_ARG;
    if (option == DL_OPT_SORT_MODE) {
        if (value < DL_SORT_AUTO || value > DL_SORT_BINNED)
            return fail(ctx, DL_ERR_INVALID_ARG, "sort mode %lld", (long long)value);
        ctx->sort_mode = int32_t(value);
        return DL_OK;
    }
    if (option == DL_OPT_WARP_LIST_CAP) {
        if (value != 0 && value != 512 && value != 1024)
            return fail(ctx, DL_ERR_INVALID_ARG, "warp list capacity %lld", (long long)value);
        ctx->warp_cap = int32_t(value);
        return DL_OK;
    }
    if (option == DL_OPT_KEY_EMISSION) {
        if (value < 0 || value > 2)
            return fail(ctx, DL_ERR_INVALID_ARG, "key emission %lld", (long long)value);
        ctx->key_emission = int32_t(value);
        return DL_OK;
    }
    if (option == DL_OPT_HEAP_CAPACITY) {
        if (value < 1 || value > kMaxHeap)
            return fail(ctx, DL_ERR_INVALID_ARG, "heap capacity %lld out of [1, %d]",
                        (long long)value, kMaxHeap);
        ctx->heap_cap = int32_t(value);
        return DL_OK;
    }
    if (option == DL_OPT_STANDARD_VIEW_SIZE) {
        const int64_t vw = value >> 16, vh = value & 0xFFFF;
        if (value != 0 && (vw < 1 || vw > 16384 || vh < 1 || vh > 16384))
            return fail(ctx, DL_ERR_INVALID_ARG, "standard view size %lldx%lld", (long long)vw,
                        (long long)vh);
        ctx->std_view_w = int32_t(vw);
        ctx->std_view_h = int32_t(vh);
        return DL_OK;
    }
    if (option == DL_OPT_EVAL_DIRECTL || option == DL_OPT_EVAL_STANDARD) {
        if (value != DL_EVAL_DIRECT && value != DL_EVAL_TRANSPOSED)
            return fail(ctx, DL_ERR_INVALID_ARG, "evaluation strategy %lld", (long long)value);
        if (option == DL_OPT_EVAL_DIRECTL) {
            ctx->eval_transposed[DL_DIRECTL] = int32_t(value);
            ctx->eval_transposed[DL_REQUIRED_ONLY] = int32_t(value);
        } else {
            ctx->eval_transposed[DL_STANDARD] = int32_t(value);
        }
        return DL_OK;
    }
    return fail(ctx, DL_ERR_INVALID_ARG, "unknown option %d", option);
}

dl_status dl_enable_stage_timing(dl_ctx* ctx, int32_t enable) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (enable < 0 || enable > 2) return fail(ctx, DL_ERR_INVALID_ARG, "stage timing mode %d", enable);
    if (enable == 1 && !ctx->ws.pairs.p) {
        DL_CK(ctx->ws.pairs.reserve(16), "alloc counters");
        DL_CK(cudaMemset(ctx->ws.pairs.p, 0, 16), "memset");
    }
    ctx->timing = enable != 0;
    ctx->count_pairs = enable == 1;
    return DL_OK;
}

dl_status dl_last_frame_stats(dl_ctx* ctx, dl_frame_stats* out) {
    if (!ctx || !out) return DL_ERR_INVALID_ARG;
    if (ctx->ws.last_async >= 0) {
        dl_status st = check_ctx(ctx);
        if (st) return st;
        st = harvest_readbacks(ctx, true);
        if (st) return st;
    }
    *out = ctx->stats;
    return DL_OK;
}

dl_status dl_stage_totals(dl_ctx* ctx, dl_frame_stats* sum, int32_t* n_frames) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!sum || !n_frames) return fail(ctx, DL_ERR_INVALID_ARG, "null argument");
    st = harvest_readbacks(ctx, true);
    if (st) return st;
    dl_frame_stats t{};
    t.tile_w = ctx->stats.tile_w;
    t.tile_h = ctx->stats.tile_h;
    t.sort_bits = ctx->stats.sort_bits;
    Workspace& W = ctx->ws;
    for (PendingFrame& f : W.pending) {
        DL_CK(cudaEventSynchronize(f.ev->e[kStageEvents - 1]), "event sync");
        cudaEvent_t* e = f.ev->e;
        t.ms_project += elapsed(e[0], e[1]);
        t.ms_scan += elapsed(e[1], e[2]);
        t.ms_sync += elapsed(e[2], e[3]);
        t.ms_emit += elapsed(e[3], e[4]);
        t.ms_sort += elapsed(e[4], e[5]);
        t.ms_ranges += elapsed(e[5], e[6]);
        t.ms_composite += elapsed(e[6], e[7]);
        t.ms_interweave += elapsed(e[7], e[8]);
        t.ms_total += elapsed(e[0], e[8]);
        t.n_keys += f.n_keys;
        t.n_visible += f.n_visible;
        t.n_rays += f.n_rays;
        t.n_launches += f.launches;
        t.lists_small += f.lists_small;
        t.lists_large += f.lists_large;
        t.max_list = std::max(t.max_list, f.max_list);
        t.status += f.status != 0 ? 1 : 0;
        t.reemitted += f.reemitted;
        W.ev_free.push_back(f.ev);
    }
    *n_frames = int32_t(W.pending.size());
    W.pending.clear();
    if (W.pairs.p) {
        unsigned long long h[2] = {0, 0};
        DL_CK(cudaMemcpy(h, W.pairs.p, 16, cudaMemcpyDeviceToHost), "copy counters");
        DL_CK(cudaMemset(W.pairs.p, 0, 16), "memset");
        t.pairs_evaluated = int64_t(h[0]);
        t.pairs_blended = int64_t(h[1]);
    }
    *sum = t;
    return DL_OK;
}

dl_status dl_query_footprint(dl_ctx* ctx, int32_t scene_id, int32_t display_id, int32_t mode,
                             size_t* bytes) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!bytes) return fail(ctx, DL_ERR_INVALID_ARG, "null bytes");
    auto si = ctx->scenes.find(scene_id);
    auto di = ctx->displays.find(display_id);
    if (si == ctx->scenes.end() || di == ctx->displays.end())
        return fail(ctx, DL_ERR_NOT_FOUND, "scene %d / display %d", scene_id, display_id);
    const Scene& S = *si->second;
    const Display& D = *di->second;
    const size_t ne = size_t(D.q.nv) * size_t(S.n);
    size_t b = ne * (16 * kRecordFloat4 + 16 + 8) + scan_tmp_bytes(int64_t(ne));  // records, metadata, counts, offsets
    // tile keys: about two tiles per (view, Gaussian) at the default shapes
    const size_t keys = 2 * ne;
    b += 2 * keys * 12 + radix_tmp_bytes(int64_t(keys));
    if (mode == DL_STANDARD || mode == DL_STANDARD_SR) b += size_t(D.q.nv) * D.q.w * D.q.h * 12;
    *bytes = std::max(b, ctx->ws.last_bytes);
    return DL_OK;
}

dl_status dl_render_frame(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                          const double L0_c2w[16], int32_t mode, float* out, int32_t out_on_device,
                          void* stream) {
    return render_frame(ctx, scene_id, display_id, L0_c2w, mode, out,
                        out_on_device ? kOutDevice : kOutHost, static_cast<cudaStream_t>(stream),
                        nullptr);
}

dl_status dl_render_frame_async_host(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                                     const double L0_c2w[16], int32_t mode, float* out,
                                     void* stream, void* copy_stream) {
    if (ctx && stream == copy_stream)
        return fail(ctx, DL_ERR_INVALID_ARG, "copy_stream must differ from stream");
    return render_frame(ctx, scene_id, display_id, L0_c2w, mode, out, kOutHostAsync,
                        static_cast<cudaStream_t>(stream), static_cast<cudaStream_t>(copy_stream));
}

}  // extern "C"

namespace dl {

dl_status render_frame(dl_ctx* ctx, int32_t scene_id, int32_t display_id, const double L0_c2w[16],
                       int32_t mode, float* out, int32_t kind, cudaStream_t s, cudaStream_t cs) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!L0_c2w || !out) return fail(ctx, DL_ERR_INVALID_ARG, "null argument");
    if (mode < 0 || mode > DL_STANDARD_SR) return fail(ctx, DL_ERR_INVALID_ARG, "mode %d", mode);
    auto si = ctx->scenes.find(scene_id);
    if (si == ctx->scenes.end()) return fail(ctx, DL_ERR_NOT_FOUND, "scene %d", scene_id);
    auto di = ctx->displays.find(display_id);
    if (di == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    Scene& S = *si->second;
    Display& D = *di->second;
    Workspace& W = ctx->ws;
    // counters of earlier frames that have arrived update their signatures'
    // capacities before this frame is sized
    st = harvest_readbacks(ctx, false);
    if (st) return st;
    const int64_t frame = W.frame_no++;
    const bool timing = ctx->timing;
    StageEvents* E = nullptr;
    if (timing) {
        if (W.ev_free.empty()) {
            auto* ne = new (std::nothrow) StageEvents();
            if (!ne) return fail(ctx, DL_ERR_OOM, "events");
            for (auto& e : ne->e) DL_CK(cudaEventCreate(&e), "event create");
            W.ev_free.push_back(ne);
        }
        E = W.ev_free.back();
        W.ev_free.pop_back();
        W.pending.push_back(PendingFrame{E, 0, 0, 0, 0, 0, 0, 0});
        W.pending.back().frame = frame;
    }
    auto mark = [&](int i) -> cudaError_t {
        return timing ? cudaEventRecord(E->e[i], s) : cudaSuccess;
    };
    DL_CK(mark(0), "event");
    if (mode == DL_RAYCAST) return render_raycast(ctx, S, D, L0_c2w, out, kind, s, cs, E);
    // "HR w SR" renders as DL_STANDARD (views at panel resolution) and
    // gathers each subpixel from its repurposed source pixel at the end
    const bool sr = mode == DL_STANDARD_SR;
    if (sr) mode = DL_STANDARD;

    const int32_t nv = D.q.nv, w = D.q.w, h = D.q.h;
    const int32_t tw = ctx->tile[mode][0], th = ctx->tile[mode][1];
    // the standard paradigm's views: panel resolution, or LR / MR upsampled
    // while interweaving
    const bool lowres = mode == DL_STANDARD && !sr && ctx->std_view_w > 0 &&
                        (ctx->std_view_w != w || ctx->std_view_h != h);
    const int32_t rw = lowres ? ctx->std_view_w : w, rh = lowres ? ctx->std_view_h : h;
    RaySet* R = nullptr;
    TileGroups* G = nullptr;
    if (mode != DL_STANDARD) {
        R = &D.rep;
        if (mode == DL_REQUIRED_ONLY) {
            if (D.prm.repurpose == 0) {
                R = &D.rep;
            } else {
                if (!D.ident.built) {
                    st = build_rayset(ctx, D, D.ident, true, s);
                    if (st) return st;
                }
                R = &D.ident;
            }
        }
        st = get_groups(ctx, D, *R, tw, th, s, &G);
        if (st) return st;
    }

    // ---- cameras (Eq. (17)) and projection (Eqs. (8)-(10)) ----
    std::vector<Cam> cams;
    dl_display_params view_prm = D.prm;  // the views' own resolution (focal, shifts)
    view_prm.width = rw;
    view_prm.height = rh;
    if (!make_cams(view_prm, L0_c2w, cams))
        return fail(ctx, DL_ERR_INVALID_ARG, "off-axis rig: the world origin is not in front of L0");
    st = upload_cams(ctx, cams, s);
    if (st) return st;
    const ProjectParams pp = make_project_params(S, D, tw, th, rw, rh);
    const int64_t ntiles = int64_t(pp.ntx) * pp.nty;
    const int64_t ne = int64_t(nv) * S.n;
    if (ne >= (int64_t(1) << 31)) return fail(ctx, DL_ERR_CAPACITY, "views x Gaussians >= 2^31");
    const int64_t ngroups = int64_t(nv) * ntiles;
    if (ngroups >= (int64_t(1) << 31) - 1) return fail(ctx, DL_ERR_CAPACITY, "too many tiles");
    // DirectL: lists of up to warp_cap keys become warp items, longer ones go
    // to the block kernel; standard: small / large block classes.
    const bool warp_path = mode != DL_STANDARD && ctx->warp_cap > 0;
    // Sizing: the totals are read back (one host synchronisation) until a
    // frame of this signature has been sized; later frames run on the
    // signature's capacities and device counters, and are dropped on the
    // device (status word, output untouched) when they exceed them.
    FrameHint& hint = ctx->hints[FrameSig{scene_id, display_id, mode, tw, th, rw, rh}];
    const bool on_device = warp_path && hint.sized && ctx->sort_mode != DL_SORT_RADIX;
    // keys emitted by the projection, into the slices the signature's last
    // frame laid out
    // (by default only for scenes of 131,072 Gaussians or more: a warp's
    // views run one after another, each waiting on its cursor atomics, which
    // only enough warps in flight hide)
    const bool in_projection = emit_in_projection(ctx->key_emission, S.n);
    const bool direct = on_device && in_projection && hint.slices_ready;
    DL_CK(W.rec.reserve(16 * kRecordFloat4 * size_t(ne)), "alloc records");
    if (!direct) DL_CK(W.meta.reserve(16 * size_t(ne)), "alloc tile metadata");
    DL_CK(W.gcount.reserve(4 * size_t(ngroups + 1)), "alloc group counts");
    DL_CK(W.gstart.reserve(4 * size_t(ngroups + 1)), "alloc group starts");
    DL_CK(W.gfill.reserve(4 * size_t(ngroups)), "alloc cursors");
    DL_CK(W.gscan_tmp.reserve(scan_tmp_bytes(ngroups + 1)), "alloc scan");
    DL_CK(W.small.reserve(256), "alloc");
    unsigned long long* d_total64 = W.small.as<unsigned long long>();
    uint32_t* d_total32 = reinterpret_cast<uint32_t*>(W.small.as<char>() + 64);
    uint32_t* d_redo = d_total32 + 1;  // a key found its slice full (direct emission)
    uint32_t* d_meta = reinterpret_cast<uint32_t*>(W.small.as<char>() + 128);
    uint32_t* d_status = d_meta + 7;
    DL_CK(cudaMemsetAsync(W.small.p, 0, 256, s), "memset");
    // the key buffer only grows, so its capacity covers every earlier sizing
    const uint32_t key_cap =
        on_device ? uint32_t(std::min<size_t>(W.keys[0].bytes / 8, size_t((1u << 31) - 2))) : 0u;
    const void* attrs[5] = {S.mean.p, S.log_scale.p, S.rot.p, S.opacity.p, S.sh.p};
    const int4* gwork = mode == DL_STANDARD ? nullptr : G->gwork.as<int4>();
    const int64_t n_work = mode == DL_STANDARD ? ngroups : G->n_gwork;
    const size_t nw1 = size_t(std::max<int64_t>(n_work, 1));
    DL_CK(W.lists.reserve(32 * nw1 + 16), "alloc lists");
    // warp path: items, then block items; otherwise the two class lists
    int4* items = W.lists.as<int4>();
    int4* block_items = items + nw1;
    int32_t* small_list = W.lists.as<int32_t>();
    int32_t* large_list = small_list + nw1;
    uint32_t* cursor = W.gfill.as<uint32_t>();
    if (direct) {
        DL_CK(hint.slices[hint.cur ^ 1].reserve(4 * size_t(ngroups + 1)), "alloc slices");
        const uint32_t* slice = hint.slices[hint.cur].as<uint32_t>();
        uint32_t* next = hint.slices[hint.cur ^ 1].as<uint32_t>();
        DL_CK(cudaMemcpyAsync(cursor, slice, 4 * size_t(ngroups), cudaMemcpyDeviceToDevice, s),
              "cursors");
        ProjectOut po{W.rec.as<float4>(), nullptr, d_total64, nullptr, d_total64 + 1};
        po.keys = W.keys[0].as<unsigned long long>();
        po.cursor = cursor;
        po.slice = slice;
        po.key_cap = key_cap;
        po.overflow = d_redo;
        DL_CK(launch_project_direct(S.dtype, attrs, pp, W.cams.as<Cam>(), nv, po, false, s),
              "project");
        DL_CK(mark(1), "event");
        // the next frame's slices, from this frame's counts (the scan's
        // total, at d_total32, is read back with the frame's counters)
        DL_CK(launch_pad_counts(cursor, slice, ngroups, W.gcount.as<uint32_t>(), s), "pad counts");
        DL_CK(launch_exclusive_scan(W.gcount.as<uint32_t>(), next, ngroups + 1, d_total32,
                                    W.gscan_tmp.p, s),
              "slice scan");
        // a frame that outgrew a slice emits its keys again, into those
        // slices (no key past key_cap: the frame is dropped, status bit 0)
        DL_CK(launch_reset_cursor(d_redo, next, ngroups, cursor, s), "cursors");
        ProjectOut po2 = po;
        po2.slice = next;
        po2.gate = d_redo;
        po2.overflow = d_status;
        DL_CK(launch_project_direct(S.dtype, attrs, pp, W.cams.as<Cam>(), nv, po2, true, s),
              "re-emit keys");
        GroupSlices sl;
        sl.start = slice;
        sl.start_alt = next;
        sl.use_alt = d_redo;
        sl.cursor = cursor;
        DL_CK(launch_partition_warp(gwork, n_work, sl, uint32_t(ctx->warp_cap),
                                    ctx->warp_cap < 1024 ? 1024u : 0u, items, block_items, d_meta,
                                    nullptr, key_cap, d_status, s),
              "partition");
        hint.cur ^= 1;
    } else {
        DL_CK(cudaMemsetAsync(W.gcount.p, 0, 4 * size_t(ngroups + 1), s), "memset");
        ProjectOut po{W.rec.as<float4>(), W.meta.as<uint4>(), d_total64, W.gcount.as<uint32_t>(),
                      d_total64 + 1};
        DL_CK(launch_project(S.dtype, attrs, pp, W.cams.as<Cam>(), nv, po, s), "project");
        DL_CK(mark(1), "event");
        // group starts (one extra entry: gstart[ngroups] = number of keys) and
        // the split of the compositing work by list length
        DL_CK(launch_exclusive_scan(W.gcount.as<uint32_t>(), W.gstart.as<uint32_t>(), ngroups + 1,
                                    d_total32, W.gscan_tmp.p, s),
              "group scan");
    }
    const uint32_t* d_nkeys = W.gstart.as<uint32_t>() + ngroups;
    if (direct) {
        // partitioned above
    } else if (warp_path) {
        GroupSlices sl;
        sl.start = W.gstart.as<uint32_t>();
        DL_CK(launch_partition_warp(gwork, n_work, sl, uint32_t(ctx->warp_cap),
                                    ctx->warp_cap < 1024 ? 1024u : 0u, items, block_items, d_meta,
                                    on_device ? d_nkeys : nullptr, key_cap,
                                    on_device ? d_status : nullptr, s),
              "partition");
    } else {
        DL_CK(launch_partition(gwork, n_work, W.gstart.as<uint32_t>(), uint32_t(kSmallCap), small_list,
                               large_list, d_meta, s),
              "partition");
    }
    DL_CK(mark(2), "event");
    int64_t nk = 0, n_visible = 0, n_small = 0, n_large = 0, n_mid = 0, max_len = 0;
    int cap_large = warp_path ? 2048 : 1;
    bool binned = true;
    if (on_device) {
        // upper bounds: the persistent kernels read the item counts on the device
        n_small = n_mid = n_large = n_work;
        cap_large = hint.block_cap;
        nk = int64_t(key_cap);
    } else {
        DL_CK(cudaMemcpyAsync(W.h_total, W.small.p, 256, cudaMemcpyDeviceToHost, s), "copy totals");
        DL_CK(cudaStreamSynchronize(s), "sync");
        const unsigned long long nkeys = W.h_total[0];
        n_visible = int64_t(W.h_total[1]);
        const uint32_t* h_meta =
            reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(W.h_total) + 128);
        n_small = h_meta[0];
        n_large = h_meta[1];
        n_mid = warp_path ? int64_t(h_meta[4]) : 0;  // 1024-key warp class
        max_len = h_meta[2];
        if (nkeys >= (1ull << 31) - 1)
            return fail(ctx, DL_ERR_CAPACITY, "frame needs %llu tile keys (limit 2^31-1)", nkeys);
        nk = int64_t(nkeys);
        while (cap_large < max_len) cap_large <<= 1;
        const int binned_threads = mode == DL_STANDARD ? tw * th : kBinnedThreads;
        const size_t class_smem = warp_path ? block_smem_bytes(cap_large)
                                            : binned_smem_bytes(std::max(cap_large, kSmallCap),
                                                                binned_threads);
        binned = ctx->sort_mode != DL_SORT_RADIX && max_len <= kLargeCap &&
                 class_smem <= max_smem_optin(ctx->device);
        if (ctx->sort_mode == DL_SORT_BINNED && !binned)
            return fail(ctx, DL_ERR_CAPACITY, "a tile list holds %lld keys (binned limit %d)",
                        (long long)max_len, kLargeCap);
        // capacities for the signature's later frames: a quarter more keys
        // (and 65,536) than the slices this frame's counts lay out (its keys,
        // an eighth more and 16 a group), lists up to 1.25 times its longest
        hint.sized = false;
        hint.slices_ready = false;
        if (warp_path && binned) {
            const int64_t laid = nk + nk / 8 + 16 * ngroups;
            const int64_t want = laid + laid / 4 + 65536;
            int bc = 2048;
            while (bc < kLargeCap && bc < max_len + max_len / 4) bc <<= 1;
            if (want < (int64_t(1) << 31) - 2 && block_smem_bytes(bc) <= max_smem_optin(ctx->device)) {
                DL_CK(W.keys[0].reserve(8 * size_t(want)), "alloc keys");
                hint.sized = true;
                hint.key_cap = want;
                hint.block_cap = bc;
            }
        }
    }
    unsigned long long* pairs =
        timing && ctx->count_pairs ? W.pairs.as<unsigned long long>() : nullptr;

    CompositeParams cp{};
    cp.n = S.n;
    cp.width = rw;
    cp.height = rh;
    cp.half_w = pp.half_w;
    cp.half_h = pp.half_h;
    cp.tile_w = tw;
    cp.tile_h = th;
    cp.ntx = pp.ntx;
    cp.ntiles = int32_t(ntiles);
    cp.meta = W.meta.as<uint4>();
    const size_t out_bytes = 12 * size_t(w) * size_t(h);
    float* dst = nullptr;
    st = out_target(ctx, out, kind, out_bytes, s, &dst);
    if (st) return st;
    float* Mm = nullptr;
    float* raycol = nullptr;
    if (mode == DL_STANDARD) {
        DL_CK(W.Mm.reserve(12 * size_t(nv) * size_t(rw) * size_t(rh)), "alloc M_m");
        Mm = W.Mm.as<float>();
    } else {
        DL_CK(W.raycol.reserve(12 * size_t(R->n_rays > 0 ? R->n_rays : 1)), "alloc ray colours");
        raycol = W.raycol.as<float>();
    }
    int sort_bits = 0;
    // cameras, projection, scan, partition (direct emission: and the counts'
    // padding, the cursor reset and the gated re-emission)
    int launches = int32_t((nv + kCamBatch - 1) / kCamBatch) + 1 + 3 + (n_work > 0 ? 1 : 0) +
                   (direct ? 3 : 0);
    DL_CK(W.keys[0].reserve(8 * size_t(nk > 0 ? nk : 1)), "alloc keys");
    if (binned) {
        // ---- binned keys, sorted per tile in shared memory while compositing ----
        DL_CK(mark(3), "event");
        if (!direct) {
            DL_CK(cudaMemcpyAsync(cursor, W.gstart.p, 4 * size_t(ngroups), cudaMemcpyDeviceToDevice,
                                  s),
                  "cursors");
            DL_CK(launch_emit_binned(pp, nv, W.meta.as<uint4>(), cursor,
                                     W.keys[0].as<unsigned long long>(),
                                     on_device ? d_nkeys : nullptr, key_cap,
                                     on_device ? d_status : nullptr, s),
                  "emit binned");
            if (warp_path && hint.sized && in_projection) {
                // the signature's first slices for keys emitted by the
                // projection, from this frame's counts
                for (DevBuf& b : hint.slices)
                    DL_CK(b.reserve(4 * size_t(ngroups + 1)), "alloc slices");
                DL_CK(launch_pad_counts(W.gcount.as<uint32_t>(), nullptr, ngroups,
                                        hint.slices[hint.cur ^ 1].as<uint32_t>(), s),
                      "pad counts");
                DL_CK(launch_exclusive_scan(hint.slices[hint.cur ^ 1].as<uint32_t>(),
                                            hint.slices[hint.cur].as<uint32_t>(), ngroups + 1,
                                            d_total32, W.gscan_tmp.p, s),
                      "slice scan");
                hint.slices_ready = true;
                launches += 4;
            }
        }
        DL_CK(mark(4), "event");
        DL_CK(mark(5), "event");
        DL_CK(mark(6), "event");
        const unsigned long long* keys = W.keys[0].as<unsigned long long>();
        if (mode == DL_STANDARD) {
            DL_CK(launch_composite_full_binned(cp, small_list, n_small, kSmallCap,
                                               W.gstart.as<uint32_t>(), keys, W.rec.as<float4>(), Mm,
                                               pairs, ctx->eval_transposed[mode], s),
                  "composite full (small lists)");
            DL_CK(launch_composite_full_binned(cp, large_list, n_large, cap_large,
                                               W.gstart.as<uint32_t>(), keys, W.rec.as<float4>(), Mm,
                                               pairs, ctx->eval_transposed[mode], s),
                  "composite full (large lists)");
        } else if (warp_path) {
            // one frame through the frame-batched persistent kernels
            FrameDesc fd{};
            fd.cp = cp;
            fd.grouped = G->grouped.as<int2>();
            fd.keys = keys;
            fd.rec = W.rec.as<float4>();
            fd.raycol = raycol;
            fd.items = items;
            fd.gwork = G->gwork.as<int4>();
            fd.block_items = block_items;
            fd.meta = d_meta;
            fd.status = d_meta + 7;
            fd.n_work = n_work;
            DL_CK(W.fdesc.reserve(sizeof(FrameDesc)), "alloc frame table");
            // pageable source: staged by the call, so fd may go out of scope
            DL_CK(cudaMemcpyAsync(W.fdesc.p, &fd, sizeof(FrameDesc), cudaMemcpyHostToDevice, s),
                  "copy frame table");
            const FrameDesc* dF = W.fdesc.as<FrameDesc>();
            int64_t* prefix = reinterpret_cast<int64_t*>(W.small.as<char>() + 192);
            DL_CK(launch_batch_prefix(dF, 1, prefix, s), "prefix");
            DL_CK(launch_composite_rays_warp(ctx->warp_cap, 0, dF, prefix, 1, n_small, d_meta + 3,
                                             pairs, s),
                  "composite rays (warp per group)");
            DL_CK(launch_composite_rays_warp(1024, 1, dF, prefix, 1, n_mid, d_meta + 5, pairs, s),
                  "composite rays (warp per group, 1024 keys)");
            DL_CK(launch_composite_rays_block(cap_large, dF, prefix, 1, n_large, d_meta + 6, pairs, s),
                  "composite rays (block per group)");
            launches += 1;
        } else {
            DL_CK(launch_composite_rays_binned(cp, G->gwork.as<int4>(), small_list, n_small, kSmallCap,
                                               G->grouped.as<int2>(), W.gstart.as<uint32_t>(), keys,
                                               W.rec.as<float4>(), raycol, pairs,
                                               ctx->eval_transposed[mode], s),
                  "composite rays (small lists)");
            DL_CK(launch_composite_rays_binned(cp, G->gwork.as<int4>(), large_list, n_large, cap_large,
                                               G->grouped.as<int2>(), W.gstart.as<uint32_t>(), keys,
                                               W.rec.as<float4>(), raycol, pairs,
                                               ctx->eval_transposed[mode], s),
                  "composite rays (large lists)");
        }
        launches += (direct ? 0 : 1) + (n_small > 0 ? 1 : 0) + (n_mid > 0 ? 1 : 0) +
                    (n_large > 0 ? 1 : 0);
    } else {
        // ---- global tile keys and a stable LSD radix sort ----
        DL_CK(W.count.reserve(4 * size_t(ne)), "alloc counts");
        DL_CK(W.offset.reserve(4 * size_t(ne)), "alloc offsets");
        DL_CK(W.scan_tmp.reserve(scan_tmp_bytes(ne)), "alloc scan");
        DL_CK(W.keys[1].reserve(8 * size_t(nk > 0 ? nk : 1)), "alloc keys");
        for (int i = 0; i < 2; ++i) DL_CK(W.vals[i].reserve(4 * size_t(nk > 0 ? nk : 1)), "alloc vals");
        DL_CK(W.radix_tmp.reserve(radix_tmp_bytes(nk)), "alloc radix");
        DL_CK(W.ranges.reserve(8 * size_t(ngroups)), "alloc ranges");
        DL_CK(mark(3), "event");
        DL_CK(launch_meta_counts(W.meta.as<uint4>(), ne, W.count.as<uint32_t>(), s), "counts");
        DL_CK(launch_exclusive_scan(W.count.as<uint32_t>(), W.offset.as<uint32_t>(), ne, nullptr,
                                    W.scan_tmp.p, s),
              "scan");
        DL_CK(launch_emit_keys(pp, nv, W.meta.as<uint4>(), W.offset.as<uint32_t>(),
                               W.keys[0].as<unsigned long long>(), W.vals[0].as<uint32_t>(), s),
              "emit keys");
        DL_CK(mark(4), "event");
        sort_bits = 28 + bits_for(ngroups);
        int alt = 0;
        DL_CK(radix_sort_pairs(W.keys[0].as<unsigned long long>(), W.vals[0].as<uint32_t>(),
                               W.keys[1].as<unsigned long long>(), W.vals[1].as<uint32_t>(), nk,
                               sort_bits, W.radix_tmp.p, &alt, s),
              "sort");
        unsigned long long* keys = W.keys[alt].as<unsigned long long>();
        uint32_t* vals = W.vals[alt].as<uint32_t>();
        DL_CK(mark(5), "event");
        DL_CK(cudaMemsetAsync(W.ranges.p, 0, 8 * size_t(ngroups), s), "memset");
        DL_CK(launch_key_ranges(keys, nk, 28, W.ranges.as<uint2>(), ngroups, s), "ranges");
        DL_CK(mark(6), "event");
        if (mode == DL_STANDARD) {
            DL_CK(launch_composite_full(cp, nv, W.ranges.as<uint2>(), vals, W.rec.as<float4>(), Mm,
                                        pairs, s),
                  "composite full");
        } else {
            DL_CK(launch_composite_rays(cp, G->work.as<int4>(), G->n_work, G->grouped.as<int2>(),
                                        W.ranges.as<uint2>(), vals, W.rec.as<float4>(), raycol, pairs,
                                        s),
                  "composite rays");
        }
        launches += 3 + 1 + 3 * ((nk > 1) ? (sort_bits + 7) / 8 : 0) + (nk > 0 ? 1 : 0) +
                    (mode == DL_STANDARD ? 1 : (G->n_work > 0 ? 1 : 0));
    }
    DL_CK(mark(7), "event");
    if (lowres) {
        DL_CK(launch_resize_interweave(w, h, rw, rh, D.V.as<uint16_t>(), Mm, dst, s),
              "upsample and interweave");
    } else if (sr) {
        DL_CK(launch_repurposed_interweave(w, h, D.V.as<uint16_t>(), D.rep.src.as<uint32_t>(), Mm, dst, s),
              "repurposed interweave");
    } else if (mode == DL_STANDARD) {
        DL_CK(launch_interweave(w, h, nv, D.V.as<uint16_t>(), Mm, dst, s), "interweave");
    } else {
        // a dropped frame (status set) leaves the output untouched
        DL_CK(launch_reorder(G->slot_of.as<uint32_t>(), raycol, 3 * int64_t(w) * h, dst,
                             on_device ? d_status : nullptr, s),
              "reorder");
    }
    Readback* rbk = nullptr;
    if (on_device) {  // the frame's counter block, read when it has arrived
        rbk = &W.rb[W.rb_next];
        if (rbk->busy) {
            DL_CK(cudaEventSynchronize(rbk->done), "wait for frame counters");
            apply_readback(ctx, *rbk);
        }
        DL_CK(cudaMemcpyAsync(rbk->h, W.small.p, 256, cudaMemcpyDeviceToHost, s), "copy counters");
        DL_CK(cudaEventRecord(rbk->done, s), "event");
        rbk->busy = true;
        rbk->frame = frame;
        rbk->hint = &hint;
        W.rb_next = (W.rb_next + 1) % kReadbacks;
    }
    launches += (mode == DL_STANDARD || lowres || sr)
                    ? 1
                    : reorder_launches(G->slot_of.as<uint32_t>(), 3 * int64_t(w) * h, dst);
    DL_CK(mark(8), "event");
    st = out_finish(ctx, out, kind, dst, out_bytes, s, cs);
    if (st) return st;

    // statistics: the counts of a frame run on device counters arrive with
    // its counter block (apply_readback)
    dl_frame_stats& fs = ctx->stats;
    fs = dl_frame_stats{};
    fs.n_rays = mode == DL_STANDARD ? int64_t(nv) * rw * rh : R->n_rays;
    fs.tile_w = tw;
    fs.tile_h = th;
    fs.sort_bits = sort_bits;
    fs.n_launches = launches;
    if (!on_device) {
        fs.n_keys = nk;
        fs.n_visible = n_visible;
        fs.lists_small = n_small + n_mid;
        fs.lists_large = n_large;
        fs.max_list = max_len;
    }
    W.last_async = on_device ? frame : -1;
    if (timing) {
        PendingFrame& pf = W.pending.back();
        pf.n_keys = fs.n_keys;
        pf.n_visible = fs.n_visible;
        pf.n_rays = fs.n_rays;
        pf.launches = fs.n_launches;
        pf.lists_small = fs.lists_small;
        pf.lists_large = fs.lists_large;
        pf.max_list = fs.max_list;
    }
    W.last_bytes = W.footprint();
    if (kind == kOutHost) {
        DL_CK(cudaStreamSynchronize(s), "sync");
        if (rbk && rbk->busy && rbk->frame == frame) {
            apply_readback(ctx, *rbk);
            // a dropped frame is rendered again, sized (its signature's
            // capacities were reset by apply_readback)
            if (fs.status != 0)
                return render_frame(ctx, scene_id, display_id, L0_c2w, mode, out, kind, s, cs);
        }
    }
    return DL_OK;
}

}  // namespace dl
