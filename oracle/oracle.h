/*
 * DirectL FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised restatement of what the DirectL
 * light-field renderer computes (arXiv 2407.14053).  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * renderer itself never does.  It shares no code with the CUDA library.
 *
 * Parity status per function (see the pins in tests/test_oracle_*.py):
 *   or_view_map            pinned (periodicity, row-shift identity, offset
 *                          shift, hand-worked values, per-lens balance).
 *   or_repurpose           pinned by invariants and by two small panels
 *                          worked through Alg. 2 by hand under the readings
 *                          of the choices the paper leaves open (iteration
 *                          order, search order, buffer capacity); those
 *                          readings themselves are not fixed by the paper.
 *   or_ray_table           pinned by invariants (R-first order, uniqueness)
 *                          and by the two hand-worked panels' ray tables.
 *   or_raycast_rays        pinned (closed-form t and alpha of isotropic
 *                          Gaussians, t maximises the density along the ray,
 *                          heap capacity, SH at the ray direction).
 *   or_cameras             pinned (arc radius, angles, look-at, leftmost v=0;
 *                          off-axis rig: parallel axes, straight baseline,
 *                          no parallax on the convergence plane).
 *   or_project_splat /     pinned (isotropic closed form, finite-difference
 *   or_render_rays         Jacobian, 1-3 Gaussian brute force, back-to-front
 *                          identity, SH addition theorem and orthonormality).
 *   or_render_rays lo/hi/  pinned (hand-built on-axis stacks: alpha inside and
 *   flags (the envelope)   outside its 1e-6 window, depth near-ties and a
 *                          chain of them, T inside and outside its 1e-8
 *                          window, the stop as the end of the examined
 *                          contributors; flags == 0 gives lo == hi == value).
 */
#ifndef DIRECTL_ORACLE_H
#define DIRECTL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Display description (same meaning as the library's dl_display_params). */
typedef struct {
    int32_t width, height;   /* panel pixels: w columns, h rows            */
    int32_t num_views;       /* N_v                                        */
    int32_t p_w;             /* grating units per repurposing area         */
    double pitch_lx;         /* line count L_x, in subpixel widths         */
    double tan_slant;        /* tan(alpha)                                 */
    double offset_k;         /* K_offset, in subpixel widths               */
    double view_span_deg;    /* theta_d, angle between outermost cameras   */
    double fov_x_deg;        /* horizontal field of view of each camera    */
    int32_t repurpose;       /* 0 = identity assignment, 1 = Alg. 2        */
    int32_t reverse_views;   /* 1 = view 0 is the rightmost camera         */
    int32_t rig;             /* 0 = arc (Sec. 3.2), 1 = off-axis straight line */
} or_display;

/* Gaussian scene, FP64 structure of arrays. */
typedef struct {
    int64_t n;
    int32_t sh_degree;          /* 0..3 */
    const double* mean;         /* n*3 */
    const double* log_scale;    /* n*3 */
    const double* rot_wxyz;     /* n*4, need not be normalised */
    const double* opacity_logit;/* n   */
    const double* sh;           /* n*(d+1)^2*3, coefficient-major, RGB inner */
} or_scene;

/* One projected Gaussian in one view. */
typedef struct {
    double u, v;          /* image-plane mean (u = column, v = row)       */
    double conic[3];      /* inverse 2D covariance: xx, xy, yy            */
    double cov2d[3];      /* 2D covariance incl. the 0.3 low-pass         */
    double opacity;
    double rgb[3];
    double depth;         /* camera-space z                               */
    int32_t valid;        /* 0 when culled by the near plane              */
} or_splat;

/* Q32 fixed-point display constants (the display's exact definition). */
int or_quantise(const or_display* p, int64_t* t3q, int64_t* lq, int64_t* kq);

/* View-index map V (h x 3w, row-major), Eqs. (1)-(3). */
int or_view_map(const or_display* p, uint16_t* V);

/* Area id of every subpixel (h x 3w), grouping P_w lens units. */
int or_area_map(const or_display* p, int64_t* area);

/* Encoded-image index matrix M_i as packed source pixels: src[(x*w+y)*3+k]
 * = (x' << 16) | y'.  Alg. 2 (or the identity when repurpose == 0). */
int or_repurpose(const or_display* p, const uint16_t* V, uint32_t* src);

/* Unique rays in R-first order.  ray_of[(x*w+y)*3+k] = ray id; rays get
 * (view, row, col).  ray_* arrays need room for 3*w*h entries.  Returns the
 * number of rays through *n_rays. */
int or_ray_table(const or_display* p, const uint16_t* V, const uint32_t* src,
                 uint32_t* ray_of, int32_t* ray_v, int32_t* ray_r, int32_t* ray_c,
                 int64_t* n_rays);

/* Camera-to-world poses of every view (N_v x 16, row-major) and the shift of
 * each view's principal point along the image columns (N_v pixels; may be
 * NULL).  rig 0: T_v = R_v L_0 on an arc (Sec. 3.2), no shift.  rig 1: the
 * "off-axis perspective with straight lines" of Sec. 3.2: L_0 translated by
 * D tan(theta_v) along its x axis, D the depth of the world origin in L_0's
 * camera, and the principal point shifted by f x_v / D so that the plane at
 * depth D has no parallax.  Returns -1 when D <= 0 for rig 1. */
int or_cameras(const or_display* p, const double L0[16], double* c2w, double* shift);

/* Real spherical-harmonic basis up to degree 3 at a unit direction. */
void or_sh_basis(const double dir[3], double out[16]);

/* Project Gaussian g of the scene into a camera (c2w, 4x4 row-major). */
void or_project_splat(const or_scene* sc, int64_t g, const double c2w[16],
                      double focal, int32_t width, int32_t height, or_splat* out);
/* The same with the principal point at (w/2 + shift, h/2). */
void or_project_splat_shift(const or_scene* sc, int64_t g, const double c2w[16], double focal,
                            double shift, int32_t width, int32_t height, or_splat* out);

/* Ray-order 3DGS (Sec. 7, Alg. 3) colour of rays (view, row, col): per ray
 * (origin at the view's camera, unit direction through the pixel), every
 * Gaussian with alpha_j = o_j G(o + t_j d) >= 1/255 at its highest-density
 * point t_j = (mu - o)^T S^-1 d / (d^T S^-1 d) > 0.2 enters a heap keeping
 * the heap_cap nearest (t, index); those are blended in t order with the
 * SH colour at d.  rgb/lo/hi as or_render_rays. */
int or_raycast_rays(const or_scene* sc, const or_display* p, const double L0[16], int64_t n_rays,
                    const int32_t* ray_v, const int32_t* ray_r, const int32_t* ray_c,
                    int32_t heap_cap, double* rgb, double* lo, double* hi, int32_t* flags,
                    int n_threads);

/* Colour of rays (view, row, col) by front-to-back compositing over every
 * Gaussian.  rgb/lo/hi are n_rays*3; lo/hi bound the results of the
 * alternative decisions at FP32-resolution ties and thresholds (flags bit 0:
 * depth near-tie between consecutive included contributors, bit 1: alpha
 * within 1e-6 of 1/255, bit 2: T within 1e-8 of 1e-4).  Only contributors up
 * to the one that stops compositing are examined for the alpha and T
 * windows; the depth check also reaches the first included contributor
 * after it, which a swap can bring in front of it.  n_contrib
 * (optional) receives the number of composited Gaussians per ray.
 * n_threads <= 0 uses every core. */
int or_render_rays(const or_scene* sc, const or_display* p, const double L0[16],
                   int64_t n_rays, const int32_t* ray_v, const int32_t* ray_r,
                   const int32_t* ray_c, double* rgb, double* lo, double* hi,
                   int32_t* flags, int64_t* n_contrib, int n_threads);

/* Alg. 1 sampling step: M_e[x,y,k] = M_m[V(x,3y+k), x, y, k]. */
int or_interweave(const or_display* p, const uint16_t* V, const double* Mm, double* Me);

/* Number of threads the render call would use. */
int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
