// Internal declarations shared by the CUDA translation units of libdirectl.
// Nothing here crosses the C ABI (include/directl.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace dl {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// Display constants as the kernels see them.  t3q, lq, kq are the Q32
// fixed-point 3 tan(alpha), L_x and K_offset; win_dx / win_dy the row and
// column extents of the repurposing search range (Sec. 5, Eq. (14)).
struct DisplayQ {
    int32_t w, h, nv, pw;
    int64_t t3q, lq, kq;
    int32_t win_dx, win_dy;
    int32_t slant_neg;
    int32_t n_areas;
    int64_t area_min;
};

// One view's camera: world->camera rotation (row-major), translation, centre.
// 16-byte aligned and padded to five float4, so a kernel reads it with five
// vector loads.
struct alignas(16) Cam {
    float r[9];
    float t[3];
    float c[3];
    float shift;    // principal point (w/2 + shift, h/2): off-axis views
    float shift_f;  // shift / focal
    float pad[3];
};
static_assert(sizeof(Cam) == 80, "five float4");

__device__ __forceinline__ Cam load_cam(const Cam* __restrict__ p) {
    Cam c;
    const float4* s = reinterpret_cast<const float4*>(p);
    float4* d = reinterpret_cast<float4*>(&c);
#pragma unroll
    for (int i = 0; i < 5; ++i) d[i] = __ldg(s + i);
    return c;
}

// Cameras of a frame reach the device as a kernel parameter of a one-block
// copy kernel (stream-ordered, nothing to keep alive on the host).
constexpr int kCamBatch = 128;
struct CamBatch {
    Cam cam[kCamBatch];
};

// Projection constants of a frame.
struct ProjectParams {
    int64_t n;            // Gaussians
    int32_t sh_degree;
    int32_t width, height;
    float focal;
    float half_w, half_h;  // principal point (w/2, h/2)
    float lim_x, lim_y;    // 1.3 tan(fov/2) clamps of the EWA Jacobian
    int32_t tile_w, tile_h, ntx, nty;
    int32_t tile_sx, tile_sy;  // log2 of tile_w, tile_h (powers of two)
};

// Per (view, Gaussian) record written by the projection, 2 x float4 = 32 B
// (one DRAM sector; records start at 32-byte boundaries):
//  q0 = (u - w/2, v - h/2, A, B)
//  q1 = (C, log2(opacity), colour bits lo, colour bits hi)
// with log2 alpha = A dx^2 + B dx dy + C dy^2 + log2(opacity) at pixel offset
// (dx, dy) from the mean (A, B, C are -log2(e)/2 times the conic's xx, 2xy,
// yy).  The colour (r, g, b >= 0) keeps, per channel, the 8 exponent bits and
// the top 13 mantissa bits of its FP32 value, rounded to nearest (relative
// error <= 2^-14): lo = r21 << 11 | b21 >> 10, hi = g21 << 11 | (b21 & 0x3FF),
// x21 being bits 30..10 of the rounded FP32 pattern (the sign bit is 0).
constexpr int kRecordFloat4 = 2;

__device__ __forceinline__ void pack_rgb(float r, float g, float b, float& lo, float& hi) {
    // + 0x200 rounds the dropped 10 bits to nearest; a carry into the
    // exponent is the correct rounding; colours are finite and >= 0
    const uint32_t kr = (__float_as_uint(r) + 0x200u) >> 10;
    const uint32_t kg = (__float_as_uint(g) + 0x200u) >> 10;
    const uint32_t kb = (__float_as_uint(b) + 0x200u) >> 10;
    lo = __uint_as_float((kr << 11) | (kb >> 10));
    hi = __uint_as_float((kg << 11) | (kb & 0x3FFu));
}

__device__ __forceinline__ void unpack_rgb(float lo_f, float hi_f, float& r, float& g, float& b) {
    const uint32_t lo = __float_as_uint(lo_f), hi = __float_as_uint(hi_f);
    r = __uint_as_float((lo & 0xFFFFF800u) >> 1);
    g = __uint_as_float((hi & 0xFFFFF800u) >> 1);
    b = __uint_as_float(((lo & 0x7FFu) << 20) | ((hi & 0x3FFu) << 10));
}
// Per (view, Gaussian) tile metadata written beside the record, all that key
// emission reads (the compositing loaders that test records against pixel
// boxes read the box from here too): {rect_c, rect_r (as in q2), depth key, tiles touched}; the
// depth key is the FP32 bits of z minus those of 0.2 (z > 0.2), clamped to
// 28 bits; tiles touched = 0 marks a culled Gaussian (the rest is then 0).
struct ProjectOut {
    float4* rec;       // nv * n * kRecordFloat4
    uint4* meta;       // nv * n
    unsigned long long* total;  // sum of tiles touched (atomic)
    uint32_t* gcount;  // optional: keys per (view, tile) group (atomic; zeroed by caller)
    unsigned long long* visible = nullptr;  // optional: records written (atomic)
    // launch_project_direct only (meta and gcount unused there)
    unsigned long long* keys = nullptr;  // binned keys, written into their group's slice
    uint32_t* cursor = nullptr;          // per group: next slot (starts at slice[g])
    const uint32_t* slice = nullptr;     // group g's slots: [slice[g], slice[g + 1])
    uint32_t key_cap = 0;                // slots past the key buffer are never written
    uint32_t* overflow = nullptr;        // |= 1 when a key found its slice full
    const uint32_t* gate = nullptr;      // keys-only pass: runs only when *gate != 0
};

template <typename T>
struct GaussiansView {
    const float* mean;
    const T* log_scale;
    const T* rot;
    const T* opacity_logit;
    const T* sh;
};

// ---- scene layout (scene.cu) ----------------------------------------------
// Morton order of the means: *perm (inside tmp) lists the source index of
// each reordered Gaussian.
size_t spatial_order_tmp_bytes(int64_t n);
cudaError_t launch_spatial_order(const float* mean, int64_t n, void* tmp, uint32_t** perm,
                                 cudaStream_t s);
// dst record i = src record perm[i] (record_bytes even).
cudaError_t launch_gather_records(const void* src, void* dst, const uint32_t* perm, int64_t n,
                                  size_t record_bytes, cudaStream_t s);

// ---- a1..a3: display tables (display.cu) --------------------------------
cudaError_t launch_view_map(const DisplayQ& q, uint16_t* V, cudaStream_t s);
cudaError_t launch_repurpose(const DisplayQ& q, const uint16_t* V, uint32_t* src, int identity,
                             cudaStream_t s);
// Ray table: fills ray_of (3wh) and *d_n_rays (device); rays are numbered in
// order of first use by R, then G, then B subpixels.  Scratch comes from
// `tmp` (>= ray_table_tmp_bytes(q)); launch_ray_attributes then reads the
// same scratch to fill ray_view / ray_pix (n_rays each).
size_t ray_table_tmp_bytes(const DisplayQ& q);
cudaError_t launch_ray_table(const DisplayQ& q, const uint16_t* V, const uint32_t* src,
                             uint32_t* ray_of, void* tmp, uint32_t* d_n_rays, cudaStream_t s);
cudaError_t launch_ray_attributes(const DisplayQ& q, const uint16_t* V, const void* tmp,
                                  uint32_t* ray_view, uint32_t* ray_pix, cudaStream_t s);
// Group keys of rays for a compositing tile shape: key = (tile*nv + v) << 16
// | Morton code of the pixel inside the tile; value = ray id.  Sorted, the
// rays are grouped tile-major (every view of a tile, then the next tile), so
// a tile's ray colours are one run and the reorder's gathers for a patch of
// the panel stay in a few kilobytes.
cudaError_t launch_ray_group_keys(const uint32_t* ray_view, const uint32_t* ray_pix, int64_t n_rays,
                                  int32_t tile_w, int32_t tile_h, int32_t ntx, int32_t nv,
                                  unsigned long long* keys, uint32_t* vals, cudaStream_t s);
// (view, row, col) int32 triplets of every ray.
cudaError_t launch_rays_export(const uint32_t* ray_view, const uint32_t* ray_pix, int64_t n_rays,
                               int32_t* out, cudaStream_t s);
// Gathers per grouped ray {pixel, ray id}.
cudaError_t launch_ray_group_gather(const uint32_t* order, const uint32_t* ray_pix, int64_t n_rays,
                                    int2* grouped, cudaStream_t s);
// slot_of[i] = position in `grouped` of subpixel i's ray (ray_of[i]); the
// compositing kernels write a ray's colour at its grouped position, so a
// warp's rays write one contiguous run.  pos_tmp: n_rays words of scratch.
cudaError_t launch_group_slots(const int2* grouped, int64_t n_rays, const uint32_t* ray_of,
                               int64_t n_subpixels, uint32_t* pos_tmp, uint32_t* slot_of,
                               cudaStream_t s);

// ---- a5/a6: projection, key emission (project.cu) ------------------------
// dtype: 0 f32, 1 bf16, 2 f16
// Copies up to kCamBatch cameras from a kernel parameter into device memory.
cudaError_t launch_store_cams(const CamBatch& b, int32_t n, Cam* dst, cudaStream_t s);
cudaError_t launch_project(int dtype, const void* const* attrs, const ProjectParams& p,
                           const Cam* cams, int32_t nv, ProjectOut out, cudaStream_t s);
// Projection that emits the binned keys itself (no tile metadata, no
// emission pass) into slices laid out before the launch (out.slice,
// out.cursor, out.keys, out.key_cap, out.overflow); keys_only: the pass that
// re-emits a frame whose slices overflowed, gated by *out.gate, writing
// neither records nor totals.
cudaError_t launch_project_direct(int dtype, const void* const* attrs, const ProjectParams& p,
                                  const Cam* cams, int32_t nv, ProjectOut out, bool keys_only,
                                  cudaStream_t s);
// padded[g] = count + count / 8 + 16 with count = cursor[g] - slice[g]
// (slice == nullptr: count = cursor[g]); padded[n_groups] = 0.
cudaError_t launch_pad_counts(const uint32_t* cursor, const uint32_t* slice, int64_t n_groups,
                              uint32_t* padded, cudaStream_t s);
// cursor[g] = start[g] for every group when *flag != 0 (else nothing).
cudaError_t launch_reset_cursor(const uint32_t* flag, const uint32_t* start, int64_t n_groups,
                                uint32_t* cursor, cudaStream_t s);
// Keys depth << 32 | Gaussian << 4 | quadrant bits (Gaussians < 2^28; bit q
// of the nibble: the pixel box overlaps quadrant q, x half + 2 * y half, of
// the tile) into their group's slice
// [gstart[g], gstart[g+1]): cursor[g] holds gstart[g] at the launch (a copy
// made by the caller) and is advanced by atomics.
// total_keys (optional) = gstart + n_groups: when it exceeds key_cap no key is
// written and *status |= 1.
cudaError_t launch_emit_binned(const ProjectParams& p, int32_t nv, const uint4* meta,
                               uint32_t* cursor, unsigned long long* keys,
                               const uint32_t* total_keys, uint32_t key_cap, uint32_t* status,
                               cudaStream_t s);
// tiles touched per (view, Gaussian) out of the metadata (for the radix path's scan)
cudaError_t launch_meta_counts(const uint4* meta, int64_t n, uint32_t* count, cudaStream_t s);
cudaError_t launch_emit_keys(const ProjectParams& p, int32_t nv, const uint4* meta,
                             const uint32_t* offset, unsigned long long* keys, uint32_t* vals,
                             cudaStream_t s);

// ---- ray-order 3DGS (raycast.cu) ------------------------------------------
constexpr int kMaxHeap = 256;       // largest heap capacity c_h
constexpr int kRayStack = 256;      // traversal stack entries per ray
constexpr int kMaxWideDepth = (kRayStack - 8) / 7;  // deepest wide level the stack holds
// 8-wide node of the ray-order tree: child boxes (structure of arrays) and
// child references: a wide node index, kRayLeafBit | first << 3 | (count - 1)
// for a leaf of Gaussians [first, first + count), or kRayNoChild.
constexpr uint32_t kRayLeafBit = 0x80000000u;
constexpr uint32_t kRayNoChild = 0x7FFFFFFFu;
struct alignas(16) RayNode {
    float lox[8], loy[8], loz[8], hix[8], hiy[8], hiz[8];
    uint32_t child[8];
    uint32_t pad[8];
};
static_assert(sizeof(RayNode) == 256, "one node, two 128-byte lines");
// Per-Gaussian data of the ray-order renderer: gauss (3 float4: mean and
// opacity, S = Sigma^-1) and gbox (2 float4: the alpha >= 1/255 box).
cudaError_t launch_raycast_prepare(int dtype, const void* const* attrs, int64_t n, float4* gauss,
                                   float4* gbox, cudaStream_t s);
// Scratch of the tree build for n Gaussians.
size_t raycast_build_tmp_bytes(int64_t n);
// Binary SAH tree over gbox (synchronises `s` once per level); *n_bin: its
// internal nodes (the wide tree has at most that many, and at least one).
cudaError_t raycast_build_binary(const float4* gbox, int64_t n, void* tmp, int64_t* n_bin,
                                 cudaStream_t s);
// Collapse into 8-wide nodes (`nodes`: room for max(n_bin, 1)); *n_wide
// nodes, *depth the deepest wide level (0: the root alone).
cudaError_t raycast_collapse(const float4* gbox, int64_t n, void* tmp, int64_t n_bin,
                             RayNode* nodes, int64_t* n_wide, int* depth, cudaStream_t s);
// One thread per ray (view ray_view, pixel ray_pix): ray colours into raycol
// (3 floats per thread, in thread order).  Thread i casts ray order[i].y
// (order: a permutation of the rays as {pixel, ray id}, e.g. a tile
// grouping), or ray i when order is null.  The tree's depth must be at most
// kMaxWideDepth (checked when it is built), which bounds every ray's stack.
cudaError_t launch_raycast(int dtype, int sh_degree, const float4* gauss, const RayNode* nodes,
                           int64_t n, const void* sh, const uint32_t* ray_view,
                           const uint32_t* ray_pix, const int2* order, int64_t n_rays,
                           const Cam* cams, float focal, float half_w, float half_h, int heap_cap,
                           float* raycol, cudaStream_t s);

// ---- scan / radix sort / ranges (sort.cu) ---------------------------------
size_t scan_tmp_bytes(int64_t n);
// out[i] = sum_{j<i} in[j]; *d_total (device) = sum of all.
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                                  void* tmp, cudaStream_t s);
size_t radix_tmp_bytes(int64_t n);
// Sorts (keys, vals) by the low `bits` key bits, stable.  Ping-pongs between
// (keys, vals) and (keys_alt, vals_alt); returns in *result_in_alt whether
// the sorted data ended in the alt buffers.
cudaError_t radix_sort_pairs(unsigned long long* keys, uint32_t* vals, unsigned long long* keys_alt,
                             uint32_t* vals_alt, int64_t n, int bits, void* tmp,
                             int* result_in_alt, cudaStream_t s);
// ranges[g] = [first, last) index of keys whose key >> shift == g < n_groups.
// ranges must be zeroed first.
cudaError_t launch_key_ranges(const unsigned long long* keys, int64_t n, int shift, uint2* ranges,
                              int64_t n_groups, cudaStream_t s);

// ---- a7..a9: compositing (composite.cu) -----------------------------------
struct CompositeParams {
    int64_t n;        // Gaussians per view
    int32_t width, height;
    float half_w, half_h;
    int32_t tile_w, tile_h, ntx, ntiles;
    const uint4* meta;  // per (view, Gaussian) tile metadata of the projection (pixel box)
};
// DirectL: work items {group, begin, end, -} over grouped rays.
// pairs (optional, 2 x u64): evaluated and composited (ray, Gaussian) pairs.
// raycol: 3 floats per ray id.
cudaError_t launch_composite_rays(const CompositeParams& p, const int4* work, int64_t n_work,
                                  const int2* grouped, const uint2* ranges, const uint32_t* vals,
                                  const float4* rec, float* raycol, unsigned long long* pairs,
                                  cudaStream_t s);
// Encoded image from ray colours (Sec. 4 step (3), Sec. 6: the channel
// reorder by precomputed indices): out[i] = raycol[3 ray_of[i] + i mod 3],
// with ray_of either the ray ids (colours in ray-id order) or a tile
// grouping's slot_of (colours in grouped order).
// Nothing is written when skip (optional, device) holds a nonzero word.
cudaError_t launch_reorder(const uint32_t* ray_of, const float* raycol, int64_t n_subpixels,
                           float* out, const uint32_t* skip, cudaStream_t s);
// kernels launch_reorder launches for these arguments (1 or 2)
int reorder_launches(const uint32_t* ray_of, int64_t n_subpixels, const float* out);
// Standard paradigm: every pixel of every view into Mm (nv x h x w x 3).
cudaError_t launch_composite_full(const CompositeParams& p, int32_t nv, const uint2* ranges,
                                  const uint32_t* vals, const float4* rec, float* Mm,
                                  unsigned long long* pairs, cudaStream_t s);
// Binned paths: each block sorts its group's keys in shared memory (bucket
// counting sort, up to `cap` keys, a power of two) and then composites in that
// order; `transposed` selects the evaluation strategy.
// `list` selects the blocks' work entries (size class), gwork holds
// {group, ray begin, ray end, -} per DirectL group with rays.
constexpr int kBinnedThreads = 128;
size_t binned_smem_bytes(int cap_p, int nthr);
// Dynamic shared memory of launch_composite_rays_block for a list capacity.
size_t block_smem_bytes(int cap);
cudaError_t launch_composite_rays_binned(const CompositeParams& p, const int4* gwork,
                                         const int32_t* list, int64_t n_list, int cap_p,
                                         const int2* grouped, const uint32_t* gstart,
                                         const unsigned long long* keys, const float4* rec,
                                         float* raycol, unsigned long long* pairs, int transposed,
                                         cudaStream_t s);
cudaError_t launch_composite_full_binned(const CompositeParams& p, const int32_t* list,
                                         int64_t n_list, int cap_p, const uint32_t* gstart,
                                         const unsigned long long* keys, const float4* rec,
                                         float* Mm, unsigned long long* pairs, int transposed,
                                         cudaStream_t s);
// DirectL groups whose lists hold at most 512 or 1024 keys: one warp per
// group (warp-level sort, cp.async batches of 32, transposed evaluation),
// persistent over self-contained items {group, first key, first ray,
// rays << 16 | keys} made by launch_partition_warp: groups of at most cap1
// keys at the front of `items`, cap1 < keys <= cap2 at the back (from
// items[n_work - 1] down), the other groups as block items {group, first
// key, gwork index, keys}; meta = {n_items1, n_block, max keys, -,
// n_items2}.  When *total_keys (optional: the slices' end) exceeds key_cap
// nothing is written and status |= 1; nothing is written either when status
// bit 0 is already set (keys were dropped).
// Where each group's keys are: [start[g], start[g + 1]) when cursor is
// null; else [s[g], cursor[g]) with s = start_alt when *use_alt != 0, else
// start (the slices of a frame whose keys the projection emitted).
struct GroupSlices {
    const uint32_t* start = nullptr;
    const uint32_t* start_alt = nullptr;
    const uint32_t* use_alt = nullptr;
    const uint32_t* cursor = nullptr;
};
cudaError_t launch_partition_warp(const int4* gwork, int64_t n_work, const GroupSlices& slices,
                                  uint32_t cap1, uint32_t cap2, int4* items, int4* block_items,
                                  uint32_t* meta, const uint32_t* total_keys, uint32_t key_cap,
                                  uint32_t* status, cudaStream_t s);

// One DirectL frame's compositing inputs, as read by the frame-batched
// persistent kernels (device memory, one entry per frame).
struct FrameDesc {
    CompositeParams cp;
    const int2* grouped;              // {pixel, ray id} per grouped ray
    const unsigned long long* keys;   // binned keys (the items give each group's slice)
    const float4* rec;                // records, view-major
    float* raycol;                    // 3 floats per ray id
    const int4* items;                // launch_partition_warp output
    const int4* gwork;                // {group, ray begin, ray end, -}
    const int4* block_items;          // {group, first key, gwork index, keys}
    const uint32_t* meta;             // {n_items1, n_block, max, -, n_items2}
    uint32_t* status;                 // bit 0 keys overflow, bit 1 list longer than the block cap
    int64_t n_work;
};
// prefix[c * (n_frames + 1) + f] = items of class c (0: <= 512 keys,
// 1: <= 1024 keys, 2: block list) in frames before f; one block.
cudaError_t launch_batch_prefix(const FrameDesc* frames, int32_t n_frames, int64_t* prefix,
                                cudaStream_t s);
// Warp class cls (0: items at the front, 1: at the back) over every frame's
// items with a warp sort capacity of cap (512 or 1024) keys; persistent,
// claiming items through *cursor (0 at launch).  Grid: resident warps, at
// most max_items / 4 blocks (max_items: an upper bound on the class's items).
cudaError_t launch_composite_rays_warp(int cap, int cls, const FrameDesc* frames,
                                       const int64_t* prefix, int32_t n_frames, int64_t max_items,
                                       uint32_t* cursor, unsigned long long* pairs, cudaStream_t s);
// Block class (the block lists: lists too long for the warp classes, up to
// block_cap keys, a power of two <= 16384; longer lists set status bit 1 and
// are skipped), persistent: four warps sort a list together, then warp q
// composites the rays in quadrant q of the tile over the records whose key
// marks quadrant q.
cudaError_t launch_composite_rays_block(int block_cap, const FrameDesc* frames,
                                        const int64_t* prefix, int32_t n_frames, int64_t max_items,
                                        uint32_t* cursor, unsigned long long* pairs, cudaStream_t s);
// Splits work entries by their group's key count: <= small_cap -> small
// list, else large list; meta = {n_small, n_large, max count}.  gwork NULL:
// the entries are the groups 0..n_work-1 themselves.
cudaError_t launch_partition(const int4* gwork, int64_t n_work, const uint32_t* gstart,
                             uint32_t small_cap, int32_t* small_list, int32_t* large_list,
                             uint32_t* meta, cudaStream_t s);

// Alg. 1 sampling step at native resolution.
// Alg. 1 with upsampling: views rendered at rw x rh (Mm: nv x rh x rw x 3),
// each subpixel sampling its view bilinearly (see resize_interweave_kernel).
cudaError_t launch_resize_interweave(int32_t w, int32_t h, int32_t rw, int32_t rh,
                                     const uint16_t* V, const float* Mm, float* out,
                                     cudaStream_t s);
// "HR w SR": out[i] = channel k of view V[i] at the repurposed source pixel src[i].
cudaError_t launch_repurposed_interweave(int32_t w, int32_t h, const uint16_t* V, const uint32_t* src,
                                        const float* Mm, float* out, cudaStream_t s);
cudaError_t launch_interweave(int32_t w, int32_t h, int32_t nv, const uint16_t* V, const float* Mm,
                              float* out, cudaStream_t s);

int num_sms();

}  // namespace dl
