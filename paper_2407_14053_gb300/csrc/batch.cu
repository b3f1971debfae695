// Frame batches and the tile-shape autotuner declared in include/directl.h.
// A batch renders the DirectL frames (Sec. 5) of many slots with no host
// synchronisation: per slot the projection, group scan, key emission and
// list partition, then one persistent launch per compositing class over the
// tile lists of every slot, then each slot's reorder.  Capacities are fixed
// when the batch is created, overflows are detected on the device, and the
// whole sequence can be captured into a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "host.h"

namespace dl {
namespace {

// lists of <= 512 and <= 1024 keys: one warp each (two shared-memory sizes);
// longer lists: the four-warp quadrant blocks
constexpr int kWarpCap1 = 512, kWarpCap2 = 1024;
constexpr int kMetaWords = 16;  // per slot: partition counters, key total (u64 at word 8)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Slot {
    // hard limits and key capacity (from the sizing frame)
    int64_t ne_cap = 0, ng_cap = 0, nrays_cap = 0, nwork_cap = 0, key_cap = 0;
    int32_t nv_cap = 0;
    // offsets of the slot's device arrays in the arena
    size_t o_rec = 0, o_meta = 0, o_zero = 0, o_gstart = 0, o_keys = 0, o_lists = 0, o_raycol = 0;
    // keys emitted by the projection: the slices this launch emits into
    // (A) and the ones its counts lay out for the next launch (B, copied to
    // A at the end), ng_cap + 1 words each
    size_t o_slices = 0;
    bool direct = false;
    size_t zero_bytes = 0;  // gcount | gfill | meta, zeroed by every launch
    int64_t cam_first = 0;  // first camera of the slot in the staging cameras
    // assignment
    bool active = false;
    Scene* S = nullptr;
    Display* D = nullptr;
    TileGroups* G = nullptr;
    int32_t tw = 0, th = 0;
    float* out = nullptr;
    ProjectParams pp{};
    int64_t ngroups = 0;
};

bool tile_ok(int32_t v) { return v >= 8 && v <= 256 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace dl

using namespace dl;

struct dl_batch {
    dl_ctx* ctx = nullptr;
    std::vector<Slot> slots;
    DevBuf arena, stage_d, scan_tmp;
    unsigned char* stage_h = nullptr;  // pinned: FrameDesc[n_slots] | Cam[total views]
    uint32_t* status_h = nullptr;      // pinned, n_slots
    size_t stage_bytes = 0, cams_offset = 0;
    int64_t total_views = 0;
    size_t o_prefix = 0, o_globals = 0, globals_bytes = 0;  // arena offsets
    int32_t block_cap = 2048;
    cudaEvent_t done = nullptr;
    bool launched = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_valid = false;

    template <class T>
    T* at(size_t off) const {
        return reinterpret_cast<T*>(static_cast<char*>(arena.p) + off);
    }
    FrameDesc* frames_h() const { return reinterpret_cast<FrameDesc*>(stage_h); }
    Cam* cams_h() const { return reinterpret_cast<Cam*>(stage_h + cams_offset); }
    FrameDesc* frames_d() const { return stage_d.as<FrameDesc>(); }
    Cam* cams_d() const { return reinterpret_cast<Cam*>(stage_d.as<char>() + cams_offset); }
    uint32_t* cursors_d() const { return at<uint32_t>(o_globals); }
    uint32_t* status_d() const { return at<uint32_t>(o_globals) + 8; }

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        graph_valid = false;
    }
    ~dl_batch() {
        drop_graph();
        if (done) cudaEventDestroy(done);
        if (stage_h) cudaFreeHost(stage_h);
        if (status_h) cudaFreeHost(status_h);
    }
};

namespace {

dl_status wait_previous(dl_batch* b) {
    dl_ctx* ctx = b->ctx;
    if (b->launched) DL_CK(cudaEventSynchronize(b->done), "wait for the previous launch");
    return DL_OK;
}

void release_slot(Slot& z) {
    if (z.active) {
        --z.S->in_use;
        --z.D->in_use;
    }
    z.active = false;
    z.S = nullptr;
    z.D = nullptr;
    z.G = nullptr;
    z.out = nullptr;
}

// Everything one launch enqueues (also what a capture records).
dl_status enqueue(dl_batch* b, cudaStream_t s) {
    dl_ctx* ctx = b->ctx;
    const int32_t n_slots = int32_t(b->slots.size());
    // frame table of the assigned slots, in slot order
    int32_t n_act = 0;
    int64_t max_items = 0;
    for (int32_t i = 0; i < n_slots; ++i) {
        Slot& z = b->slots[size_t(i)];
        if (!z.active) continue;
        FrameDesc& fd = b->frames_h()[n_act++];
        fd = FrameDesc{};
        fd.cp.n = z.S->n;
        fd.cp.width = z.D->q.w;
        fd.cp.height = z.D->q.h;
        fd.cp.half_w = z.pp.half_w;
        fd.cp.half_h = z.pp.half_h;
        fd.cp.tile_w = z.tw;
        fd.cp.tile_h = z.th;
        fd.cp.ntx = z.pp.ntx;
        fd.cp.ntiles = z.pp.ntx * z.pp.nty;
        fd.cp.meta = b->at<uint4>(z.o_meta);
        fd.grouped = z.G->grouped.as<int2>();
        fd.keys = b->at<unsigned long long>(z.o_keys);
        fd.rec = b->at<float4>(z.o_rec);
        fd.raycol = b->at<float>(z.o_raycol);
        fd.items = b->at<int4>(z.o_lists);
        fd.block_items = b->at<int4>(z.o_lists + 16 * size_t(z.nwork_cap));
        fd.gwork = z.G->gwork.as<int4>();
        fd.meta = b->at<uint32_t>(z.o_zero + align_up(8 * size_t(z.ng_cap) + 4, 16));
        fd.status = b->status_d() + i;
        fd.n_work = z.G->n_gwork;
        max_items += z.G->n_gwork;
    }
    DL_CK(cudaMemcpyAsync(b->stage_d.p, b->stage_h, b->stage_bytes, cudaMemcpyHostToDevice, s),
          "upload frame table and cameras");
    DL_CK(cudaMemsetAsync(b->at<char>(b->o_globals), 0, b->globals_bytes, s), "memset");
    int32_t f = 0;
    for (int32_t i = 0; i < n_slots; ++i) {
        Slot& z = b->slots[size_t(i)];
        if (!z.active) continue;
        const FrameDesc& fd = b->frames_h()[f++];
        uint32_t* gcount = b->at<uint32_t>(z.o_zero);
        uint32_t* gfill = gcount + (z.ng_cap + 1);
        uint32_t* meta = const_cast<uint32_t*>(fd.meta);
        DL_CK(cudaMemsetAsync(gcount, 0, z.zero_bytes, s), "memset");
        const Scene& S = *z.S;
        const int32_t nv = z.D->q.nv;
        const void* attrs[5] = {S.mean.p, S.log_scale.p, S.rot.p, S.opacity.p, S.sh.p};
        if (z.direct) {
            // the projection emits the keys into slices A (laid out by the
            // slot's previous launch); B from this launch's counts; a slot
            // that outgrew A emits again into B (meta word 12: the flag)
            uint32_t* sa = b->at<uint32_t>(z.o_slices);
            uint32_t* sb = sa + (z.ng_cap + 1);
            uint32_t* redo = meta + 12;
            DL_CK(cudaMemcpyAsync(gfill, sa, 4 * size_t(z.ngroups), cudaMemcpyDeviceToDevice, s),
                  "cursors");
            ProjectOut po{b->at<float4>(z.o_rec), nullptr,
                          reinterpret_cast<unsigned long long*>(meta + 8), nullptr};
            po.keys = b->at<unsigned long long>(z.o_keys);
            po.cursor = gfill;
            po.slice = sa;
            po.key_cap = uint32_t(z.key_cap);
            po.overflow = redo;
            DL_CK(launch_project_direct(S.dtype, attrs, z.pp, b->cams_d() + z.cam_first, nv, po,
                                        false, s),
                  "project");
            DL_CK(launch_pad_counts(gfill, sa, z.ngroups, gcount, s), "pad counts");
            DL_CK(launch_exclusive_scan(gcount, sb, z.ngroups + 1, nullptr, b->scan_tmp.p, s),
                  "slice scan");
            DL_CK(launch_reset_cursor(redo, sb, z.ngroups, gfill, s), "cursors");
            ProjectOut po2 = po;
            po2.slice = sb;
            po2.gate = redo;
            po2.overflow = fd.status;
            DL_CK(launch_project_direct(S.dtype, attrs, z.pp, b->cams_d() + z.cam_first, nv, po2,
                                        true, s),
                  "re-emit keys");
            GroupSlices sl;
            sl.start = sa;
            sl.start_alt = sb;
            sl.use_alt = redo;
            sl.cursor = gfill;
            DL_CK(launch_partition_warp(z.G->gwork.as<int4>(), z.G->n_gwork, sl, kWarpCap1,
                                        kWarpCap2, const_cast<int4*>(fd.items),
                                        const_cast<int4*>(fd.block_items), meta, nullptr,
                                        uint32_t(z.key_cap), fd.status, s),
                  "partition");
            // the next launch's slices (the items hold this launch's offsets)
            DL_CK(cudaMemcpyAsync(sa, sb, 4 * size_t(z.ngroups + 1), cudaMemcpyDeviceToDevice, s),
                  "next slices");
            continue;
        }
        ProjectOut po{b->at<float4>(z.o_rec), b->at<uint4>(z.o_meta),
                      reinterpret_cast<unsigned long long*>(meta + 8), gcount};
        DL_CK(launch_project(S.dtype, attrs, z.pp, b->cams_d() + z.cam_first, nv, po, s), "project");
        uint32_t* gstart = b->at<uint32_t>(z.o_gstart);
        DL_CK(launch_exclusive_scan(gcount, gstart, z.ngroups + 1, nullptr, b->scan_tmp.p, s),
              "group scan");
        DL_CK(cudaMemcpyAsync(gfill, gstart, 4 * size_t(z.ngroups), cudaMemcpyDeviceToDevice, s),
              "cursors");
        DL_CK(launch_emit_binned(z.pp, nv, po.meta, gfill,
                                 b->at<unsigned long long>(z.o_keys), gstart + z.ngroups,
                                 uint32_t(z.key_cap), fd.status, s),
              "emit binned");
        GroupSlices sl;
        sl.start = gstart;
        DL_CK(launch_partition_warp(z.G->gwork.as<int4>(), z.G->n_gwork, sl, kWarpCap1, kWarpCap2,
                                    const_cast<int4*>(fd.items), const_cast<int4*>(fd.block_items),
                                    meta, gstart + z.ngroups, uint32_t(z.key_cap), fd.status, s),
              "partition");
    }
    if (n_act > 0) {
        int64_t* prefix = b->at<int64_t>(b->o_prefix);
        uint32_t* cur = b->cursors_d();
        DL_CK(launch_batch_prefix(b->frames_d(), n_act, prefix, s), "prefix");
        DL_CK(launch_composite_rays_warp(kWarpCap1, 0, b->frames_d(), prefix, n_act, max_items, cur,
                                         nullptr, s),
              "composite rays (warp class 512)");
        if (kWarpCap2 > 0)
            DL_CK(launch_composite_rays_warp(kWarpCap2, 1, b->frames_d(), prefix, n_act, max_items,
                                             cur + 1, nullptr, s),
                  "composite rays (warp class 1024)");
        DL_CK(launch_composite_rays_block(b->block_cap, b->frames_d(), prefix, n_act, max_items,
                                          cur + 2, nullptr, s),
              "composite rays (block class)");
    }
    for (int32_t i = 0; i < n_slots; ++i) {
        Slot& z = b->slots[size_t(i)];
        if (!z.active) continue;
        DL_CK(launch_reorder(z.G->slot_of.as<uint32_t>(), b->at<float>(z.o_raycol),
                             3 * int64_t(z.D->q.w) * z.D->q.h, z.out, b->status_d() + i, s),
              "reorder");
    }
    DL_CK(cudaMemcpyAsync(b->status_h, b->status_d(), 4 * size_t(n_slots), cudaMemcpyDeviceToHost, s),
          "copy status");
    return DL_OK;
}

dl_status resolve_frame(dl_ctx* ctx, int32_t scene_id, int32_t display_id, int32_t tw, int32_t th,
                        Scene** S, Display** D, int32_t* otw, int32_t* oth) {
    auto si = ctx->scenes.find(scene_id);
    if (si == ctx->scenes.end()) return fail(ctx, DL_ERR_NOT_FOUND, "scene %d", scene_id);
    auto di = ctx->displays.find(display_id);
    if (di == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    if (tw == 0 && th == 0) {
        tw = ctx->tile[DL_DIRECTL][0];
        th = ctx->tile[DL_DIRECTL][1];
    }
    if (!tile_ok(tw) || !tile_ok(th)) return fail(ctx, DL_ERR_INVALID_ARG, "tile %dx%d", tw, th);
    *S = si->second.get();
    *D = di->second.get();
    *otw = tw;
    *oth = th;
    return DL_OK;
}

}  // namespace

extern "C" {

dl_status dl_batch_create(dl_ctx* ctx, int32_t n_slots, const dl_slot_plan* plans, double margin,
                          void* stream, dl_batch** out) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!plans || !out || n_slots < 1 || n_slots > 4096 || !(margin >= 1.0) || margin > 64.0)
        return fail(ctx, DL_ERR_INVALID_ARG, "dl_batch_create: n_slots %d, margin %g", n_slots, margin);
    *out = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto b = std::unique_ptr<dl_batch>(new (std::nothrow) dl_batch());
    if (!b) return fail(ctx, DL_ERR_OOM, "batch");
    b->ctx = ctx;
    b->slots.resize(size_t(n_slots));
    // ---- size every slot from its plan frame ----
    const bool timing = ctx->timing;
    ctx->timing = false;
    const int32_t saved_tile[2] = {ctx->tile[DL_DIRECTL][0], ctx->tile[DL_DIRECTL][1]};
    DevBuf tmp_out;
    int64_t longest = 0;
    size_t scan_bytes = 0;
    for (int32_t i = 0; i < n_slots && st == DL_OK; ++i) {
        const dl_slot_plan& pl = plans[i];
        Scene* S = nullptr;
        Display* D = nullptr;
        int32_t tw = 0, th = 0;
        st = resolve_frame(ctx, pl.scene_id, pl.display_id, pl.tile_w, pl.tile_h, &S, &D, &tw, &th);
        if (st) break;
        if (tmp_out.reserve(12 * size_t(D->q.w) * D->q.h) != cudaSuccess) {
            st = fail(ctx, DL_ERR_OOM, "sizing frame output");
            break;
        }
        ctx->tile[DL_DIRECTL][0] = tw;
        ctx->tile[DL_DIRECTL][1] = th;
        st = dl_render_frame(ctx, pl.scene_id, pl.display_id, pl.L0_c2w, DL_DIRECTL,
                             tmp_out.as<float>(), 1, stream);
        if (st) break;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = cuda_fail(ctx, cudaGetLastError(), "sizing frame");
            break;
        }
        st = harvest_readbacks(ctx, true);  // the frame's counts, if read back on the device path
        if (st) break;
        TileGroups* G = nullptr;
        st = get_groups(ctx, *D, D->rep, tw, th, s, &G);
        if (st) break;
        Slot& z = b->slots[size_t(i)];
        z.nv_cap = D->q.nv;
        z.ne_cap = int64_t(D->q.nv) * S->n;
        z.ng_cap = int64_t(D->q.nv) * G->ntiles;
        z.nrays_cap = D->rep.n_rays;
        z.nwork_cap = G->n_gwork;
        // room for the slices the keys are emitted into (count + count/8 +
        // 16 a group) when the projection emits them
        const int64_t nk = ctx->stats.n_keys;
        const int64_t laid = nk + nk / 8 + 16 * z.ng_cap;
        z.key_cap = std::min<int64_t>(int64_t(std::ceil(double(laid) * margin)) + 4096,
                                      (int64_t(1) << 31) - 2);
        longest = std::max<int64_t>(longest, int64_t(std::ceil(double(ctx->stats.max_list) * margin)));
        scan_bytes = std::max(scan_bytes, scan_tmp_bytes(z.ng_cap + 1));
    }
    ctx->tile[DL_DIRECTL][0] = saved_tile[0];
    ctx->tile[DL_DIRECTL][1] = saved_tile[1];
    ctx->timing = timing;
    if (st) return st;
    b->block_cap = 2048;
    while (b->block_cap < longest && b->block_cap < 16384) b->block_cap <<= 1;
    if (block_smem_bytes(b->block_cap) > max_smem_optin(ctx->device))
        return fail(ctx, DL_ERR_CAPACITY, "long-list capacity %d exceeds shared memory", b->block_cap);
    // ---- arena layout ----
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    for (Slot& z : b->slots) {
        z.o_rec = take(16 * kRecordFloat4 * size_t(z.ne_cap));
        z.o_meta = take(16 * size_t(z.ne_cap));
        z.zero_bytes = align_up(8 * size_t(z.ng_cap) + 4, 16) + 4 * kMetaWords;
        z.o_zero = take(z.zero_bytes);
        z.o_gstart = take(4 * size_t(z.ng_cap + 1));
        z.o_keys = take(8 * size_t(z.key_cap));
        z.o_lists = take(32 * size_t(z.nwork_cap) + 16);  // items, then block items
        z.o_slices = take(8 * size_t(z.ng_cap + 1));
        z.o_raycol = take(12 * size_t(std::max<int64_t>(z.nrays_cap, 1)));
        z.cam_first = b->total_views;
        b->total_views += z.nv_cap;
    }
    b->o_prefix = take(8 * 3 * size_t(n_slots + 1));
    b->globals_bytes = 4 * (8 + size_t(n_slots));
    b->o_globals = take(b->globals_bytes);
    DL_CK(b->arena.reserve(off), "alloc batch arena");
    DL_CK(b->scan_tmp.reserve(std::max<size_t>(scan_bytes, 256)), "alloc scan scratch");
    b->cams_offset = align_up(sizeof(FrameDesc) * size_t(n_slots), 256);
    b->stage_bytes = b->cams_offset + sizeof(Cam) * size_t(b->total_views);
    DL_CK(b->stage_d.reserve(b->stage_bytes), "alloc staging");
    void* h = nullptr;
    DL_CK(cudaHostAlloc(&h, b->stage_bytes, cudaHostAllocDefault), "pinned staging");
    b->stage_h = static_cast<unsigned char*>(h);
    std::memset(b->stage_h, 0, b->stage_bytes);
    DL_CK(cudaHostAlloc(&h, 4 * size_t(n_slots), cudaHostAllocDefault), "pinned status");
    b->status_h = static_cast<uint32_t*>(h);
    std::memset(b->status_h, 0, 4 * size_t(n_slots));
    DL_CK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event");
    ++ctx->n_batches;
    *out = b.release();
    return DL_OK;
}

dl_status dl_batch_destroy(dl_batch* b) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (b->launched) cudaEventSynchronize(b->done);
    for (Slot& z : b->slots) release_slot(z);
    --ctx->n_batches;
    delete b;
    return DL_OK;
}

dl_status dl_batch_assign(dl_batch* b, int32_t slot, int32_t scene_id, int32_t display_id,
                          int32_t tile_w, int32_t tile_h, float* out_dev) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (slot < 0 || slot >= int32_t(b->slots.size()) || !out_dev)
        return fail(ctx, DL_ERR_INVALID_ARG, "slot %d / output", slot);
    st = wait_previous(b);
    if (st) return st;
    Scene* S = nullptr;
    Display* D = nullptr;
    int32_t tw = 0, th = 0;
    st = resolve_frame(ctx, scene_id, display_id, tile_w, tile_h, &S, &D, &tw, &th);
    if (st) return st;
    TileGroups* G = nullptr;
    st = get_groups(ctx, *D, D->rep, tw, th, nullptr, &G);
    if (st) return st;
    Slot& z = b->slots[size_t(slot)];
    const int64_t ne = int64_t(D->q.nv) * S->n, ng = int64_t(D->q.nv) * G->ntiles;
    if (D->q.nv > z.nv_cap || ne > z.ne_cap || ng > z.ng_cap || D->rep.n_rays > z.nrays_cap ||
        G->n_gwork > z.nwork_cap)
        return fail(ctx, DL_ERR_CAPACITY,
                    "frame (views %d, views x Gaussians %lld, groups %lld, rays %lld, lists %lld) "
                    "exceeds slot %d (%d, %lld, %lld, %lld, %lld)",
                    D->q.nv, (long long)ne, (long long)ng, (long long)D->rep.n_rays,
                    (long long)G->n_gwork, slot, z.nv_cap, (long long)z.ne_cap,
                    (long long)z.ng_cap, (long long)z.nrays_cap, (long long)z.nwork_cap);
    release_slot(z);
    z.active = true;
    z.S = S;
    z.D = D;
    z.G = G;
    ++S->in_use;
    ++D->in_use;
    z.tw = tw;
    z.th = th;
    z.out = out_dev;
    z.pp = make_project_params(*S, *D, tw, th);
    z.ngroups = ng;
    z.direct = emit_in_projection(ctx->key_emission, S->n);
    if (z.direct) {  // empty slices: the first launch emits into slices of its own counts
        DL_CK(cudaMemsetAsync(b->at<uint32_t>(z.o_slices), 0, 4 * size_t(ng + 1), nullptr),
              "memset");
        DL_CK(cudaStreamSynchronize(nullptr), "sync");
    }
    // identity pose until dl_batch_set_pose
    // a pose on the -z axis at distance 4 until dl_batch_set_pose
    const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, -4, 0, 0, 0, 1};
    std::vector<Cam> cams;
    make_cams(D->prm, I, cams);
    std::memcpy(b->cams_h() + z.cam_first, cams.data(), sizeof(Cam) * cams.size());
    b->drop_graph();
    return DL_OK;
}

dl_status dl_batch_clear(dl_batch* b, int32_t slot) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (slot < 0 || slot >= int32_t(b->slots.size())) return fail(ctx, DL_ERR_INVALID_ARG, "slot %d", slot);
    st = wait_previous(b);
    if (st) return st;
    if (b->slots[size_t(slot)].active) b->drop_graph();
    release_slot(b->slots[size_t(slot)]);
    return DL_OK;
}

dl_status dl_batch_set_pose(dl_batch* b, int32_t slot, const double L0_c2w[16]) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (slot < 0 || slot >= int32_t(b->slots.size()) || !L0_c2w)
        return fail(ctx, DL_ERR_INVALID_ARG, "slot %d / pose", slot);
    Slot& z = b->slots[size_t(slot)];
    if (!z.active) return fail(ctx, DL_ERR_INVALID_ARG, "slot %d is not assigned", slot);
    st = wait_previous(b);
    if (st) return st;
    std::vector<Cam> cams;
    if (!make_cams(z.D->prm, L0_c2w, cams))
        return fail(ctx, DL_ERR_INVALID_ARG, "off-axis rig: the world origin is not in front of L0");
    std::memcpy(b->cams_h() + z.cam_first, cams.data(), sizeof(Cam) * cams.size());
    return DL_OK;
}

dl_status dl_batch_launch(dl_batch* b, void* stream) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->graph_valid) {
        DL_CK(cudaGraphLaunch(b->exec, s), "graph launch");
    } else {
        st = enqueue(b, s);
        if (st) return st;
    }
    DL_CK(cudaEventRecord(b->done, s), "event");
    b->launched = true;
    return DL_OK;
}

dl_status dl_batch_capture(dl_batch* b, void* stream) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) return fail(ctx, DL_ERR_INVALID_ARG, "capture needs a created stream");
    st = wait_previous(b);
    if (st) return st;
    b->drop_graph();
    DL_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "begin capture");
    st = enqueue(b, s);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    b->graph = g;
    DL_CK(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    b->graph_valid = true;
    return DL_OK;
}

dl_status dl_batch_wait(dl_batch* b, uint32_t* status) {
    if (!b) return DL_ERR_INVALID_ARG;
    dl_ctx* ctx = b->ctx;
    dl_status st = check_ctx(ctx);
    if (st) return st;
    st = wait_previous(b);
    if (st) return st;
    int32_t bad = 0;
    for (size_t i = 0; i < b->slots.size(); ++i) {
        const uint32_t v = b->slots[i].active && b->launched ? b->status_h[i] : 0u;
        if (status) status[i] = v;
        if (v) ++bad;
    }
    if (bad) return fail(ctx, DL_ERR_CAPACITY, "%d slot(s) exceeded their capacity", bad);
    return DL_OK;
}

dl_status dl_batch_info(dl_batch* b, size_t* bytes, int32_t* long_list_cap) {
    if (!b) return DL_ERR_INVALID_ARG;
    if (bytes) *bytes = b->arena.bytes + b->stage_d.bytes + b->scan_tmp.bytes;
    if (long_list_cap) *long_list_cap = b->block_cap;
    return DL_OK;
}

dl_status dl_autotune_tile(dl_ctx* ctx, int32_t scene_id, int32_t display_id,
                           const double L0_c2w[16], const int32_t* candidates, int32_t n_candidates,
                           int32_t reps, void* stream, int32_t* best, float* ms) {
    dl_status st = check_ctx(ctx);
    if (st) return st;
    if (!L0_c2w || !candidates || n_candidates < 1 || reps < 1 || reps > 1000 || !best)
        return fail(ctx, DL_ERR_INVALID_ARG, "dl_autotune_tile arguments");
    for (int32_t c = 0; c < n_candidates; ++c)
        if (!tile_ok(candidates[2 * c]) || !tile_ok(candidates[2 * c + 1]))
            return fail(ctx, DL_ERR_INVALID_ARG, "candidate %dx%d", candidates[2 * c],
                        candidates[2 * c + 1]);
    auto di = ctx->displays.find(display_id);
    if (di == ctx->displays.end()) return fail(ctx, DL_ERR_NOT_FOUND, "display %d", display_id);
    const Display& D = *di->second;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf out;
    DL_CK(out.reserve(12 * size_t(D.q.w) * D.q.h), "alloc");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DL_CK(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, cudaGetLastError(), "event");
    }
    const bool timing = ctx->timing;
    ctx->timing = false;
    const int32_t saved[2] = {ctx->tile[DL_DIRECTL][0], ctx->tile[DL_DIRECTL][1]};
    float best_ms = 0.f;
    int32_t best_c = -1;
    std::vector<float> t(static_cast<size_t>(reps));
    for (int32_t c = 0; c < n_candidates && st == DL_OK; ++c) {
        ctx->tile[DL_DIRECTL][0] = candidates[2 * c];
        ctx->tile[DL_DIRECTL][1] = candidates[2 * c + 1];
        st = dl_render_frame(ctx, scene_id, display_id, L0_c2w, DL_DIRECTL, out.as<float>(), 1, stream);
        for (int32_t r = 0; r < reps && st == DL_OK; ++r) {
            cudaEventRecord(e0, s);
            st = dl_render_frame(ctx, scene_id, display_id, L0_c2w, DL_DIRECTL, out.as<float>(), 1,
                                 stream);
            cudaEventRecord(e1, s);
            if (st) break;
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t[size_t(r)], e0, e1) != cudaSuccess) {
                st = cuda_fail(ctx, cudaGetLastError(), "autotune timing");
                break;
            }
        }
        if (st) break;
        std::sort(t.begin(), t.end());
        const float med = t[size_t(reps / 2)];
        if (ms) ms[c] = med;
        if (best_c < 0 || med < best_ms) {
            best_ms = med;
            best_c = c;
        }
    }
    ctx->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) {
        ctx->tile[DL_DIRECTL][0] = saved[0];
        ctx->tile[DL_DIRECTL][1] = saved[1];
        return st;
    }
    ctx->tile[DL_DIRECTL][0] = best[0] = candidates[2 * best_c];
    ctx->tile[DL_DIRECTL][1] = best[1] = candidates[2 * best_c + 1];
    return DL_OK;
}

}  // extern "C"
