// Host-side state of the C ABI (contexts, scenes, displays, workspaces) and
// the helpers that api.cu and batch.cu share.  Host code only.
#pragma once

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/directl.h"
#include "dl_internal.cuh"

namespace dl {

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t n) {
        if (n <= bytes) return cudaSuccess;
        release();
        const size_t want = n + n / 8 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return e;
        }
        bytes = want;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

struct Scene {
    int64_t n = 0;
    int32_t sh_degree = 0, dtype = DL_F32;
    int32_t in_use = 0;  // batch slots holding this scene
    DevBuf mean, log_scale, rot, opacity, sh;
    // ray-order renderer (built on the first DL_RAYCAST frame): per-Gaussian
    // data and boxes, and the 8-wide SAH tree (its nodes and depth)
    bool rc_built = false;
    int32_t rc_depth = 0;
    int64_t rc_n_nodes = 0;
    DevBuf rc_gauss, rc_gbox, rc_nodes;
};

struct TileGroups {
    int32_t tw = 0, th = 0, ntx = 0, nty = 0, ntiles = 0;
    int64_t n_work = 0;   // <= 128-ray chunks (global radix path)
    int64_t n_gwork = 0;  // groups holding rays (binned path)
    // grouped: {pixel, ray id} per position; slot_of: per subpixel, the
    // position of its ray (ray colours are written in grouped order)
    DevBuf grouped, work, gwork, slot_of;
};

struct RaySet {
    bool built = false;
    int64_t n_rays = 0;
    DevBuf src, ray_of, ray_view, ray_pix;
    std::map<int64_t, std::unique_ptr<TileGroups>> groups;
};

struct Display {
    int32_t in_use = 0;  // batch slots holding this display
    dl_display_params prm{};
    DisplayQ q{};
    DevBuf V;
    RaySet rep;    // Alg. 2 assignment (or identity when repurpose == 0)
    RaySet ident;  // identity assignment, built on first DL_REQUIRED_ONLY frame
};

// Events around the stages of one frame (see dl_render_frame).
constexpr int kStageEvents = 9;
struct StageEvents {
    cudaEvent_t e[kStageEvents] = {};
};
struct PendingFrame {
    StageEvents* ev;
    int64_t n_keys, n_rays;
    int32_t launches;
    int64_t lists_small, lists_large, max_list;
    int64_t n_visible;
    int64_t frame = -1;  // frame number; its device counters arrive by a readback
    int32_t status = 0;
    int32_t reemitted = 0;
};

// Capacities a frame signature (scene, display, mode, tile, view size) runs
// with once one of its frames has been sized on the host: the tile-key
// buffer's capacity at that time and the long-list capacity.  Later frames
// of the signature size their launches from device counters and these
// capacities, with no host synchronisation; a frame that exceeds them is
// dropped on the device (its output left untouched, its status word set),
// and the next frame of the signature is sized on the host again, as is one
// after a frame that used more than 85 % of either capacity.
// With the keys emitted by the projection, the signature also keeps the
// slices of the key buffer its next frame emits into: every group gets its
// key count in the last frame plus an eighth and 16 (slices[cur]); a frame
// writes the next layout into slices[cur ^ 1] and flips cur.
// DL_OPT_KEY_EMISSION 2: the projection emits the keys for scenes of at
// least this many Gaussians (with fewer, too few warps are in flight to hide
// its waits on the cursor atomics)
constexpr int64_t kEmitInProjectionMin = 131072;
inline bool emit_in_projection(int32_t option, int64_t n_gaussians) {
    return option == 1 || (option == 2 && n_gaussians >= kEmitInProjectionMin);
}

struct FrameHint {
    bool sized = false;
    int32_t block_cap = 2048;
    int64_t key_cap = 0;
    bool slices_ready = false;
    int cur = 0;
    DevBuf slices[2];  // n_groups + 1 slot offsets each
};
using FrameSig = std::array<int32_t, 7>;

// Pinned copies of the 256-byte counter block of frames rendered without a
// host synchronisation (keys, visible records, list classes, status), in a
// ring; a slot is read ("harvested") once its copy has completed, at the
// latest before the slot is reused.
constexpr int kReadbacks = 8;
struct Readback {
    unsigned long long* h = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    int64_t frame = -1;
    FrameHint* hint = nullptr;
};

struct Workspace {
    DevBuf cams, rec, meta, count, offset, scan_tmp, keys[2], vals[2], ranges, radix_tmp, Mm, out, small,
        pairs, gcount, gstart, gfill, lists, gscan_tmp, raycol, fdesc;
    unsigned long long* h_total = nullptr;  // pinned, 256 bytes (copy of `small`)
    Readback rb[kReadbacks];
    int rb_next = 0;
    int64_t frame_no = 0;      // frames enqueued by render_frame
    int64_t last_async = -1;   // frame number of the last frame read back asynchronously
    int64_t dropped = 0;       // frames dropped on the device (capacity exceeded)
    size_t last_bytes = 0;
    std::vector<StageEvents*> ev_free;
    std::vector<PendingFrame> pending;
    // frames copied to the host on the caller's copy stream
    // (dl_render_frame_async_host): two device frames used in turn, the
    // frame-written and copy-done events of each, and the next one to use
    DevBuf aout[2];
    cudaEvent_t ev_frame[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    bool copy_pending[2] = {false, false};
    int aslot = 0;
    ~Workspace() {
        if (h_total) cudaFreeHost(h_total);
        for (Readback& r : rb) {
            if (r.h) cudaFreeHost(r.h);
            if (r.done) cudaEventDestroy(r.done);
        }
        for (int i = 0; i < 2; ++i) {
            if (ev_frame[i]) cudaEventDestroy(ev_frame[i]);
            if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
        }
        for (auto& f : pending) ev_free.push_back(f.ev);
        for (StageEvents* s : ev_free) {
            for (auto& e : s->e)
                if (e) cudaEventDestroy(e);
            delete s;
        }
    }
    size_t footprint() const {
        size_t b = cams.bytes + rec.bytes + meta.bytes + count.bytes + offset.bytes + scan_tmp.bytes +
                   ranges.bytes +
                   radix_tmp.bytes + Mm.bytes + out.bytes + small.bytes + gcount.bytes + gstart.bytes +
                   gfill.bytes + lists.bytes + gscan_tmp.bytes + raycol.bytes;
        for (int i = 0; i < 2; ++i) b += keys[i].bytes + vals[i].bytes + aout[i].bytes;
        return b;
    }
};

}  // namespace dl

struct dl_ctx {
    int32_t device = 0;
    std::string err;
    int32_t next_id = 1;
    std::map<int32_t, std::unique_ptr<dl::Scene>> scenes;
    std::map<int32_t, std::unique_ptr<dl::Display>> displays;
    dl::Workspace ws;
    int32_t tile[3][2] = {{32, 32}, {16, 16}, {32, 32}};
    int32_t sort_mode = DL_SORT_AUTO;
    int32_t eval_transposed[3] = {1, 0, 1};  // per mode
    int32_t warp_cap = 512;
    int32_t key_emission = 2;  // DL_OPT_KEY_EMISSION (2: by scene size)
    int32_t std_view_w = 0, std_view_h = 0;  // DL_OPT_STANDARD_VIEW_SIZE (0: panel)
    int32_t heap_cap = 128;                  // DL_OPT_HEAP_CAPACITY
    bool timing = false;
    bool count_pairs = false;  // with timing: the compositing pair counters
    dl_frame_stats stats{};
    int32_t n_batches = 0;  // live dl_batch objects on this context
    std::map<dl::FrameSig, dl::FrameHint> hints;
};

namespace dl {

dl_status fail(dl_ctx* c, dl_status s, const char* fmt, ...);
dl_status cuda_fail(dl_ctx* c, cudaError_t e, const char* what);
dl_status check_ctx(dl_ctx* ctx);
int bits_for(int64_t n);
size_t max_smem_optin(int device);
// Reads back every frame counter block whose copy has completed (wait: all
// of them, waiting for the copies), updating the frames' statistics and the
// capacities of their signatures.
dl_status harvest_readbacks(dl_ctx* ctx, bool wait);
// Rays of a ray set grouped by (view, tile) for one tile shape (cached per shape).
dl_status get_groups(dl_ctx* ctx, Display& D, RaySet& R, int32_t tw, int32_t th, cudaStream_t s,
                     TileGroups** out);
// View cameras of Eq. (17) (or of the off-axis rig) for a light-field centre
// pose; false when the off-axis rig's convergence depth is not positive.
bool make_cams(const dl_display_params& p, const double L0[16], std::vector<Cam>& cams);
// Projection parameters of a frame (tile shape tw x th), views rendered at
// rw x rh (0: the panel's resolution).
ProjectParams make_project_params(const Scene& S, const Display& D, int32_t tw, int32_t th,
                                  int32_t rw = 0, int32_t rh = 0);

}  // namespace dl

#define DL_CK(expr, what)                                       \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return dl::cuda_fail(ctx, e_, what); \
    } while (0)
