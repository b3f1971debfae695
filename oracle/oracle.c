/*
 * DirectL FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain restatement, in double precision, of what the DirectL light-field
 * renderer computes (arXiv 2407.14053).  Only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the renderer never does, and the
 * two share no code.  Every function cites the passage of the paper it
 * follows.  Where the paper is silent or ambiguous the reading taken is
 * stated next to the code (and listed in the repository's design notes).
 *
 * Parity status: see oracle.h (every function is pinned by tests; the
 * repurposing assignment is pinned under stated readings of the choices
 * Alg. 2 leaves open).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_Q32 4294967296.0
#define OR_EMPTY 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Display constants.                                                        */
/* ------------------------------------------------------------------------ */

/* Reading (Q32 display definition): tan(alpha), L_x and K_offset enter the
 * map as Q32 fixed-point numbers, each rounded to nearest-even once, in FP64:
 * T3 = round(3 tan(alpha) 2^32), Lq = round(L_x 2^32), Kq = round(K 2^32).
 * The map is then exact integer arithmetic. */
int or_quantise(const or_display* p, int64_t* t3q, int64_t* lq, int64_t* kq) {
    if (p->pitch_lx <= 0.0 || p->pitch_lx > 1024.0) return -1;
    if (fabs(p->tan_slant) > 8.0 || fabs(p->offset_k) > 1048576.0) return -1;
    *t3q = (int64_t)nearbyint(3.0 * p->tan_slant * OR_Q32);
    *lq = (int64_t)nearbyint(p->pitch_lx * OR_Q32);
    *kq = (int64_t)nearbyint(p->offset_k * OR_Q32);
    return *lq > 0 ? 0 : -1;
}

static int or_check_display(const or_display* p) {
    if (p->width <= 0 || p->height <= 0 || p->width > 16384 || p->height > 16384) return -1;
    if (p->num_views <= 0 || p->num_views > 65535) return -1;
    if (p->p_w <= 0) return -1;
    return 0;
}

/* d_offset of subpixel column s = 3y + k in row x, Eq. (1), as a Q32 integer:
 * d = 3y + 3x tan(alpha) + k - K_offset. */
static int64_t or_d_offset(int64_t x, int64_t s, int64_t t3q, int64_t kq) {
    return s * (int64_t)4294967296LL + x * t3q - kq;
}

static int64_t or_floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* ------------------------------------------------------------------------ */
/* a1: view-index map, Eqs. (1)-(3) and Alg. 1 (CalculateView).              */
/* ------------------------------------------------------------------------ */

/* x_offset = d_offset mod L_x, taken into [0, L_x) (Eq. 2 says x_offset lies
 * in that interval, so a negative d_offset wraps by floor-mod);
 * v = floor(N_v x_offset / L_x) (Eq. 3), counted from 0. */
int or_view_map(const or_display* p, uint16_t* V) {
    int64_t t3q, lq, kq;
    if (or_check_display(p) || or_quantise(p, &t3q, &lq, &kq)) return -1;
    const int64_t S = 3 * (int64_t)p->width;
    for (int64_t x = 0; x < p->height; ++x) {
        for (int64_t s = 0; s < S; ++s) {
            int64_t d = or_d_offset(x, s, t3q, kq);
            int64_t xo = d % lq;
            if (xo < 0) xo += lq;
            int64_t v = ((int64_t)p->num_views * xo) / lq;
            V[x * S + s] = (uint16_t)v;
        }
    }
    return 0;
}

/* Reading (areas): a subpixel's grating unit is floor(d_offset / L_x), the
 * slanted lens stripe it sits under; an area groups P_w consecutive units
 * (Sec. 5, "non-intersecting areas, each comprising P_w grating units"). */
int or_area_map(const or_display* p, int64_t* area) {
    int64_t t3q, lq, kq;
    if (or_check_display(p) || or_quantise(p, &t3q, &lq, &kq)) return -1;
    const int64_t S = 3 * (int64_t)p->width;
    for (int64_t x = 0; x < p->height; ++x)
        for (int64_t s = 0; s < S; ++s) {
            int64_t unit = or_floor_div(or_d_offset(x, s, t3q, kq), lq);
            area[x * S + s] = or_floor_div(unit, p->p_w);
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a2: subpixel repurposing, Sec. 5, Alg. 2 with Eqs. (11)-(14).             */
/* ------------------------------------------------------------------------ */

static uint32_t or_pack(int64_t x, int64_t y) { return ((uint32_t)x << 16) | (uint32_t)y; }

typedef struct {
    int64_t x_low, x_high, y_first, y_last; /* columns scanned y_first -> y_last */
    int step;                               /* -1 (tan >= 0) or +1 (tan < 0)   */
} or_window;

/* Search range, Eq. (14).  Reading: the bounds are taken with the Q32 line
 * count L = Lq / 2^32, x_high = min(x + floor(2 N_v/L + N_v/(2L)), h-1),
 * y_low = max(floor(y - N_v/(3L)), 0), y_high = y.  The printed range only
 * fits a clockwise tilt; for tan(alpha) < 0 the column range is mirrored to
 * [y, min(ceil(y + N_v/(3L)), w-1)]. */
static or_window or_search_range(const or_display* p, int64_t lq, int64_t t3q, int64_t x,
                                 int64_t y) {
    or_window win;
    const int64_t nv = p->num_views;
    const int64_t dx = (5 * nv * (int64_t)2147483648LL) / lq;              /* floor(5 N_v / (2L)) */
    const int64_t dy = (nv * (int64_t)4294967296LL + 3 * lq - 1) / (3 * lq); /* ceil(N_v / (3L))  */
    win.x_low = x + 2 < p->height - 1 ? x + 2 : p->height - 1;
    win.x_high = x + dx < p->height - 1 ? x + dx : p->height - 1;
    if (t3q >= 0) {
        win.y_first = y;
        win.y_last = y - dy > 0 ? y - dy : 0;
        win.step = -1;
    } else {
        win.y_first = y;
        win.y_last = y + dy < p->width - 1 ? y + dy : p->width - 1;
        win.step = +1;
    }
    return win;
}

int or_repurpose(const or_display* p, const uint16_t* V, uint32_t* src) {
    int64_t t3q, lq, kq;
    if (or_check_display(p) || or_quantise(p, &t3q, &lq, &kq)) return -1;
    const int64_t w = p->width, h = p->height, S = 3 * w, n = S * h;

    if (!p->repurpose) { /* identity: every subpixel samples its own pixel */
        for (int64_t x = 0; x < h; ++x)
            for (int64_t s = 0; s < S; ++s) src[x * S + s] = or_pack(x, s / 3);
        return 0;
    }

    int64_t* area = (int64_t*)malloc(sizeof(int64_t) * n);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * n);
    uint32_t* buf = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)p->num_views);
    if (!area || !order || !buf) { free(area); free(order); free(buf); return -2; }
    or_area_map(p, area);

    /* SplitArea: visit areas by increasing id and, inside an area, subpixels
     * in row-major (x, y, k) order (reading: the paper gives no order). */
    int64_t amin = area[0], amax = area[0];
    for (int64_t i = 1; i < n; ++i) {
        if (area[i] < amin) amin = area[i];
        if (area[i] > amax) amax = area[i];
    }
    int64_t nb = amax - amin + 1;
    int64_t* start = (int64_t*)calloc((size_t)nb + 1, sizeof(int64_t));
    if (!start) { free(area); free(order); free(buf); return -2; }
    for (int64_t i = 0; i < n; ++i) start[area[i] - amin + 1]++;
    for (int64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
    for (int64_t i = 0; i < n; ++i) order[start[area[i] - amin]++] = i;
    free(start);

    /* CreateSubpixelBuffer: B_rgb holds one idle (x, y) per (view, channel). */
    for (int64_t i = 0; i < 3 * (int64_t)p->num_views; ++i) buf[i] = OR_EMPTY;
    for (int64_t i = 0; i < n; ++i) src[i] = OR_EMPTY;

    for (int64_t oi = 0; oi < n; ++oi) {
        int64_t cur = order[oi];
        const int64_t a = area[cur];
        const int64_t vi = V[cur]; /* GetViewpoint */
        uint32_t* B = buf + 3 * vi;
        while (src[cur] == OR_EMPTY && area[cur] == a) {
            int64_t cx = cur / S, cs = cur % S, cy = cs / 3, ck = cs % 3;
            if (B[ck] != OR_EMPTY) {
                /* RepurposeSubpixel, Eq. (13); ClearUsedSubpixel. */
                src[cur] = B[ck];
                B[ck] = OR_EMPTY;
            } else {
                /* SampleNewSubpixel, Eq. (11); AddUnusedSubpixel, Eq. (12):
                 * B(v, (k-1) mod 3) = B(v, (k-2) mod 3) = (x, y). */
                src[cur] = or_pack(cx, cy);
                B[(ck + 2) % 3] = or_pack(cx, cy);
                B[(ck + 1) % 3] = or_pack(cx, cy);
            }
            /* CalculateSearchRange, Eq. (14), then SearchTheSameViewpoint.
             * Reading: the search returns the first subpixel in scan order
             * (rows ascending, columns from y outward, channels 0,1,2) that
             * shows view v_i and whose channel has an idle subpixel waiting
             * in B_rgb(v_i, .).  It does not look at M_i or at the area: the
             * while condition above ends the chain when that subpixel is
             * already filled or lies outside the current area. */
            or_window win = or_search_range(p, lq, t3q, cx, cy);
            int64_t found = -1;
            for (int64_t r = win.x_low; r <= win.x_high && found < 0; ++r) {
                for (int64_t c = win.y_first;; c += win.step) {
                    for (int64_t ch = 0; ch < 3; ++ch) {
                        int64_t j = r * S + 3 * c + ch;
                        if (V[j] == vi && B[ch] != OR_EMPTY) {
                            found = j;
                            break;
                        }
                    }
                    if (found >= 0 || c == win.y_last) break;
                }
            }
            if (found < 0) break; /* no position left for view v_i */
            cur = found;
        }
        /* ClearSubpixelBuffer(B_rgb, v_i). */
        B[0] = B[1] = B[2] = OR_EMPTY;
    }
    free(area);
    free(order);
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a3: ray set U_rays and its R-first order, Sec. 5 (end).                   */
/* ------------------------------------------------------------------------ */

/* The rows of R~_rays follow the R subpixels in row-major order, so the first
 * rays are the rays of the R subpixels (wh of them whenever the three
 * channels of every pixel show different views).  Reading: every ray is
 * numbered in order of first use, scanning the R subpixels (row-major), then
 * the G subpixels, then the B subpixels.  (When N_v < L_x two channels of a
 * pixel can show one view; Alg. 2 can then give one ray's channel to two
 * subpixels, and two R subpixels may share a ray.) */
int or_ray_table(const or_display* p, const uint16_t* V, const uint32_t* src,
                 uint32_t* ray_of, int32_t* ray_v, int32_t* ray_r, int32_t* ray_c,
                 int64_t* n_rays) {
    if (or_check_display(p)) return -1;
    const int64_t w = p->width, h = p->height, n = 3 * w * h;
    /* open-addressing hash set of (v, x', y') -> ray id */
    uint64_t cap = 1;
    while (cap < (uint64_t)(2 * n)) cap <<= 1;
    int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * cap);
    uint32_t* vals = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    if (!keys || !vals) { free(keys); free(vals); return -2; }
    for (uint64_t i = 0; i < cap; ++i) keys[i] = -1;
    int64_t count = 0;
    int rc = 0;
    for (int k = 0; k < 3 && rc == 0; ++k) {
        for (int64_t x = 0; x < h && rc == 0; ++x) {
            for (int64_t y = 0; y < w; ++y) {
                int64_t i = (x * w + y) * 3 + k;
                uint32_t s = src[i];
                if (s == OR_EMPTY) { rc = -3; break; }
                int64_t xs = s >> 16, ys = s & 0xFFFF;
                int64_t v = V[x * 3 * w + 3 * y + k];
                int64_t key = (v * h + xs) * w + ys;
                uint64_t hsh = ((uint64_t)key * 0x9E3779B97F4A7C15ull) & (cap - 1);
                while (keys[hsh] != -1 && keys[hsh] != key) hsh = (hsh + 1) & (cap - 1);
                if (keys[hsh] == -1) {
                    keys[hsh] = key;
                    vals[hsh] = (uint32_t)count;
                    ray_v[count] = (int32_t)v;
                    ray_r[count] = (int32_t)xs;
                    ray_c[count] = (int32_t)ys;
                    count++;
                }
                ray_of[i] = vals[hsh];
            }
        }
    }
    free(keys);
    free(vals);
    *n_rays = count;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* a4: per-view cameras, Sec. 3.1 (multiview rendering) and Eq. (17).        */
/* ------------------------------------------------------------------------ */

/* N_v cameras evenly spaced on an arc, converging on the centre.  Reading:
 * theta_v = -theta_d/2 + v theta_d/(N_v - 1), v = 0 the leftmost camera;
 * R_v turns the light-field centre about the world y axis through the origin
 * so that a positive theta moves the camera towards its own +x (right):
 * T_v = R_y(-theta_v) L_0. */
int or_cameras(const or_display* p, const double L0[16], double* c2w, double* shift) {
    const double pi = 3.14159265358979323846;
    /* off-axis rig: depth of the world origin in L0's camera (camera z axis
     * = third column of the rotation) */
    const double D = -(L0[2] * L0[3] + L0[6] * L0[7] + L0[10] * L0[11]);
    const double focal = 0.5 * p->width / tan(0.5 * p->fov_x_deg * pi / 180.0);
    if (p->rig == 1 && !(D > 0.0)) return -1;
    for (int32_t v = 0; v < p->num_views; ++v) {
        int32_t vv = p->reverse_views ? p->num_views - 1 - v : v;
        double th = 0.0;
        if (p->num_views > 1)
            th = (-0.5 * p->view_span_deg + vv * p->view_span_deg / (p->num_views - 1)) * pi / 180.0;
        if (p->rig == 1) {
            const double xv = D * tan(th);
            double* T = c2w + 16 * (int64_t)v;
            for (int i = 0; i < 16; ++i) T[i] = L0[i];
            for (int i = 0; i < 3; ++i) T[4 * i + 3] = L0[4 * i + 3] + xv * L0[4 * i + 0];
            if (shift) shift[v] = focal * xv / D;
            continue;
        }
        if (shift) shift[v] = 0.0;
        double phi = -th;
        double R[16] = {cos(phi), 0, sin(phi), 0, 0, 1, 0, 0, -sin(phi), 0, cos(phi), 0, 0, 0, 0, 1};
        double* T = c2w + 16 * (int64_t)v;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) acc += R[4 * i + k] * L0[4 * k + j];
                T[4 * i + j] = acc;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a5: 3DGS projection, Sec. 3.3, Eqs. (7)-(10).                             */
/* ------------------------------------------------------------------------ */

/* Real spherical harmonics up to degree 3 (the basis 3DGS colours use; the
 * paper only says "spherical harmonics").  Normalisation constants from their
 * closed forms. */
void or_sh_basis(const double d[3], double o[16]) {
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    const double c0 = 0.5 / sqrt(pi);
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi);
    const double c3e = 0.25 * sqrt(105.0 / pi);
    o[0] = c0;
    o[1] = -c1 * y;
    o[2] = c1 * z;
    o[3] = -c1 * x;
    o[4] = c2a * x * y;
    o[5] = -c2a * y * z;
    o[6] = c2b * (2.0 * z * z - x * x - y * y);
    o[7] = -c2a * x * z;
    o[8] = c2c * (x * x - y * y);
    o[9] = -c3a * y * (3.0 * x * x - y * y);
    o[10] = c3b * x * y * z;
    o[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    o[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    o[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    o[14] = c3e * z * (x * x - y * y);
    o[15] = -c3a * x * (x * x - 3.0 * y * y);
}

/* Reading (camera model): camera axes x right, y down, z forward; pixel
 * (row r, col c) samples image point (u, v) = (c, r); principal point
 * (w/2, h/2); focal f = (w/2) / tan(fov_x/2), square pixels.
 * Reading (3DGS practice the paper leaves implicit): Gaussians with camera
 * z <= 0.2 are culled; J uses x/z and y/z clamped to 1.3 tan(fov/2); the 2D
 * covariance gets +0.3 on its diagonal (low-pass); opacity = sigmoid(logit);
 * colour = max(0, SH(dir) + 0.5) with dir = normalise(mu - camera centre). */
void or_project_splat(const or_scene* sc, int64_t g, const double c2w[16], double focal,
                      int32_t width, int32_t height, or_splat* out) {
    or_project_splat_shift(sc, g, c2w, focal, 0.0, width, height, out);
}

void or_project_splat_shift(const or_scene* sc, int64_t g, const double c2w[16], double focal,
                            double shift, int32_t width, int32_t height, or_splat* out) {
    memset(out, 0, sizeof(*out));
    const double* mu = sc->mean + 3 * g;
    double Rc[3][3], cen[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Rc[i][j] = c2w[4 * i + j];
        cen[i] = c2w[4 * i + 3];
    }
    /* viewing transform W = Rc^T (world -> camera) */
    double t[3];
    for (int i = 0; i < 3; ++i) {
        t[i] = 0.0;
        for (int j = 0; j < 3; ++j) t[i] += Rc[j][i] * (mu[j] - cen[j]);
    }
    out->depth = t[2];
    if (!(t[2] > 0.2)) return;

    /* Sigma = R S S^T R^T, Eq. (8) */
    const double* q = sc->rot_wxyz + 4 * g;
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
    double R[3][3] = {
        {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
        {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
        {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    double s2[3];
    for (int i = 0; i < 3; ++i) s2[i] = exp(2.0 * sc->log_scale[3 * g + i]);
    double Sig[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Sig[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) Sig[i][j] += R[i][k] * s2[k] * R[j][k];
        }
    /* Sigma_cam = W Sigma W^T */
    double Sc[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += Rc[a][i] * Sig[a][b] * Rc[b][j];
            Sc[i][j] = acc;
        }
    /* Sigma' = J W Sigma W^T J^T, Eq. (9), J the Jacobian of the perspective map */
    double thx = 0.5 * width / focal, thy = 0.5 * height / focal;
    double limx = 1.3 * thx, limy = 1.3 * thy;
    /* the clamp window follows a shifted principal point: x/z + shift/f in
     * [-limx, limx] */
    const double sz = shift / focal;
    double xz = t[0] / t[2], yz = t[1] / t[2];
    if (xz < -limx - sz) xz = -limx - sz;
    if (xz > limx - sz) xz = limx - sz;
    if (yz < -limy) yz = -limy;
    if (yz > limy) yz = limy;
    double J[2][3] = {{focal / t[2], 0.0, -focal * xz / t[2]}, {0.0, focal / t[2], -focal * yz / t[2]}};
    double C2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += J[i][a] * Sc[a][b] * J[j][b];
            C2[i][j] = acc;
        }
    C2[0][0] += 0.3;
    C2[1][1] += 0.3;
    double det = C2[0][0] * C2[1][1] - C2[0][1] * C2[1][0];
    if (!(det > 0.0)) return;
    out->cov2d[0] = C2[0][0];
    out->cov2d[1] = C2[0][1];
    out->cov2d[2] = C2[1][1];
    out->conic[0] = C2[1][1] / det;
    out->conic[1] = -C2[0][1] / det;
    out->conic[2] = C2[0][0] / det;
    out->u = focal * t[0] / t[2] + 0.5 * width + shift;
    out->v = focal * t[1] / t[2] + 0.5 * height;
    out->opacity = 1.0 / (1.0 + exp(-sc->opacity_logit[g]));

    double dir[3], dn = 0.0;
    for (int i = 0; i < 3; ++i) {
        dir[i] = mu[i] - cen[i];
        dn += dir[i] * dir[i];
    }
    dn = sqrt(dn);
    for (int i = 0; i < 3; ++i) dir[i] /= dn;
    double Y[16];
    or_sh_basis(dir, Y);
    int nc = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    const double* sh = sc->sh + (int64_t)nc * 3 * g;
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int i = 0; i < nc; ++i) acc += Y[i] * sh[3 * i + c];
        acc += 0.5;
        out->rgb[c] = acc > 0.0 ? acc : 0.0;
    }
    out->valid = 1;
}

/* ------------------------------------------------------------------------ */
/* a7/a8: per-pixel front-to-back compositing, Eqs. (5), (10).               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double depth;
    int64_t idx;
    double alpha;
    const double* rgb;
    int include;
} or_contrib;

static int or_cmp_contrib(const void* a, const void* b) {
    const or_contrib* x = (const or_contrib*)a;
    const or_contrib* y = (const or_contrib*)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_T_STOP 1e-4

/* C = sum_i alpha_i T_i c_i, T_i = prod_{j<i} (1 - alpha_j), Eq. (5), over
 * the Gaussians in depth order.  Reading (3DGS conventions): alpha is clamped
 * to 0.99, Gaussians with alpha < 1/255 are skipped, and compositing stops
 * before the Gaussian that would take T below 1e-4.  Returns the index one
 * past the last Gaussian looked at. */
static int64_t or_composite(const or_contrib* c, int64_t n, double t_stop, double out[3],
                            int64_t* used) {
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int64_t i = 0, u = 0;
    for (; i < n; ++i) {
        if (!c[i].include) continue;
        double a = c[i].alpha;
        double Tn = T * (1.0 - a);
        if (Tn < t_stop) { ++i; break; }
        for (int k = 0; k < 3; ++k) C[k] += a * T * c[i].rgb[k];
        T = Tn;
        ++u;
    }
    for (int k = 0; k < 3; ++k) out[k] = C[k];
    if (used) *used = u;
    return i;
}

static void or_envelope(const double v[3], double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) {
        if (v[k] < lo[k]) lo[k] = v[k];
        if (v[k] > hi[k]) hi[k] = v[k];
    }
}

static void or_render_one(const or_splat* sp, int64_t n, int32_t r, int32_t c, double* rgb,
                          double* lo, double* hi, int32_t* flag, int64_t* n_used) {
    /* candidates: alpha >= 1/255 - 1e-6 (the band keeps near-threshold ones) */
    int64_t cap = 64, m = 0;
    or_contrib* L = (or_contrib*)malloc(sizeof(or_contrib) * cap);
    for (int64_t g = 0; g < n; ++g) {
        const or_splat* s = sp + g;
        if (!s->valid) continue;
        double dx = (double)c - s->u, dy = (double)r - s->v;
        double power = -0.5 * (s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy +
                               s->conic[2] * dy * dy);
        if (power < -60.0) continue; /* alpha < 1e-26: far below 1/255 */
        double a = s->opacity * exp(power); /* Eq. (10) */
        if (a > 0.99) a = 0.99;
        if (a < OR_ALPHA_MIN - 1e-6) continue;
        if (m == cap) {
            cap *= 2;
            L = (or_contrib*)realloc(L, sizeof(or_contrib) * cap);
        }
        L[m].depth = s->depth;
        L[m].idx = g;
        L[m].alpha = a;
        L[m].rgb = s->rgb;
        L[m].include = a >= OR_ALPHA_MIN;
        ++m;
    }
    qsort(L, (size_t)m, sizeof(or_contrib), or_cmp_contrib);

    double base[3];
    int64_t used = 0;
    int64_t stop = or_composite(L, m, OR_T_STOP, base, &used);
    for (int k = 0; k < 3; ++k) rgb[k] = lo[k] = hi[k] = base[k];
    int32_t f = 0;
    double alt[3];
    /* A contributor's own alpha decision can change the result only up to
     * the Gaussian that stops compositing (index stop - 1).  A depth swap can
     * also bring the first included contributor after that one in front of
     * it, so the tie check reaches one past that contributor. */
    int64_t lim = stop;
    while (lim < m && !L[lim].include) ++lim;
    lim = lim < m ? lim + 1 : m;
    /* alpha within 1e-6 of 1/255: either decision is an acceptable result */
    for (int64_t i = 0; i < stop; ++i) {
        if (fabs(L[i].alpha - OR_ALPHA_MIN) < 1e-6) {
            f |= 2;
            L[i].include = !L[i].include;
            or_composite(L, m, OR_T_STOP, alt, NULL);
            or_envelope(alt, lo, hi);
            L[i].include = !L[i].include;
        }
    }
    /* depth near-ties (|dz| <= 2^-20 z) between consecutive contributors */
    {
        int64_t prev = -1;
        for (int64_t i = 0; i < lim; ++i) {
            if (!L[i].include) continue;
            if (prev >= 0 && fabs(L[i].depth - L[prev].depth) <= ldexp(fabs(L[prev].depth), -20)) {
                f |= 1;
                or_contrib t = L[i];
                L[i] = L[prev];
                L[prev] = t;
                or_composite(L, m, OR_T_STOP, alt, NULL);
                or_envelope(alt, lo, hi);
                t = L[i];
                L[i] = L[prev];
                L[prev] = t;
            }
            prev = i;
        }
    }
    /* transmittance within 1e-8 of the 1e-4 stop */
    {
        double T = 1.0;
        for (int64_t i = 0; i < stop; ++i) {
            if (!L[i].include) continue;
            double Tn = T * (1.0 - L[i].alpha);
            if (fabs(Tn - OR_T_STOP) < 1e-8) {
                f |= 4;
                or_composite(L, m, OR_T_STOP + 2e-8, alt, NULL);
                or_envelope(alt, lo, hi);
                or_composite(L, m, OR_T_STOP - 2e-8, alt, NULL);
                or_envelope(alt, lo, hi);
                break;
            }
            if (Tn < OR_T_STOP) break;
            T = Tn;
        }
    }
    *flag = f;
    if (n_used) *n_used = used;
    free(L);
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_render_rays(const or_scene* sc, const or_display* p, const double L0[16], int64_t n_rays,
                   const int32_t* ray_v, const int32_t* ray_r, const int32_t* ray_c, double* rgb,
                   double* lo, double* hi, int32_t* flags, int64_t* n_contrib, int n_threads) {
    if (or_check_display(p)) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const int32_t nv = p->num_views;
    for (int64_t i = 0; i < n_rays; ++i)
        if (ray_v[i] < 0 || ray_v[i] >= nv) return -1;
    double* cams = (double*)malloc(sizeof(double) * 17 * (size_t)nv);
    or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)(sc->n > 0 ? sc->n : 1));
    int64_t* cnt = (int64_t*)calloc((size_t)nv + 1, sizeof(int64_t));
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_rays > 0 ? n_rays : 1));
    if (!cams || !sp || !cnt || !idx) { free(cams); free(sp); free(cnt); free(idx); return -2; }
    double* shift = cams + 16 * (size_t)nv;
    if (or_cameras(p, L0, cams, shift)) { free(cams); free(sp); free(cnt); free(idx); return -1; }
    const double pi = 3.14159265358979323846;
    const double focal = 0.5 * p->width / tan(0.5 * p->fov_x_deg * pi / 180.0);
    /* group the rays by view */
    for (int64_t i = 0; i < n_rays; ++i) cnt[ray_v[i] + 1]++;
    for (int32_t v = 0; v < nv; ++v) cnt[v + 1] += cnt[v];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nv);
        for (int32_t v = 0; v < nv; ++v) fill[v] = cnt[v];
        for (int64_t i = 0; i < n_rays; ++i) idx[fill[ray_v[i]]++] = i;
        free(fill);
    }
    for (int32_t v = 0; v < nv; ++v) {
        if (cnt[v + 1] == cnt[v]) continue;
        const double* T = cams + 16 * (int64_t)v;
#pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < sc->n; ++g)
            or_project_splat_shift(sc, g, T, focal, shift[v], p->width, p->height, sp + g);
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t j = cnt[v]; j < cnt[v + 1]; ++j) {
            int64_t i = idx[j];
            int64_t used = 0;
            int32_t f = 0;
            or_render_one(sp, sc->n, ray_r[i], ray_c[i], rgb + 3 * i, lo + 3 * i, hi + 3 * i, &f,
                          &used);
            if (flags) flags[i] = f;
            if (n_contrib) n_contrib[i] = used;
        }
    }
    free(cams);
    free(sp);
    free(cnt);
    free(idx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a9: interlacing, Alg. 1 (the sampling step, at native resolution).        */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* Ray-order 3DGS (Sec. 7, Alg. 3): per ray, every Gaussian it meets gives the */
/* point of highest density along the ray, t_j = (mu - o)^T S^-1 d /        */
/* (d^T S^-1 d) (Eq. (16)), and alpha_j = o_j G(o + t_j d) (Eq. (17)); a     */
/* max-heap of capacity c_h keeps the c_h nearest; they are sorted by t and */
/* alpha-blended, colour from the SH at the ray direction d.                */
/* Readings: the ray meets a Gaussian when alpha_j >= 1/255 at t_j and t_j  */
/* exceeds the 0.2 near plane; the heap keeps the c_h smallest (t, index);  */
/* alpha is clamped to 0.99 and blending follows or_composite.              */
/* ------------------------------------------------------------------------ */

/* or_composite over the first `cap` included contributors. */
static int64_t or_composite_cap(or_contrib* c, int64_t n, double t_stop, int64_t cap,
                                double out[3]) {
    int64_t kept = 0, cut = n;
    for (int64_t i = 0; i < n; ++i)
        if (c[i].include && ++kept == cap) { cut = i + 1; break; }
    return or_composite(c, cut, t_stop, out, NULL);
}

int or_raycast_rays(const or_scene* sc, const or_display* p, const double L0[16], int64_t n_rays,
                    const int32_t* ray_v, const int32_t* ray_r, const int32_t* ray_c,
                    int32_t heap_cap, double* rgb, double* lo, double* hi, int32_t* flags,
                    int n_threads) {
    if (or_check_display(p) || heap_cap < 1) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const int32_t nv = p->num_views;
    for (int64_t i = 0; i < n_rays; ++i)
        if (ray_v[i] < 0 || ray_v[i] >= nv) return -1;
    const int64_t n = sc->n;
    const int nc = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    double* cams = (double*)malloc(sizeof(double) * 17 * (size_t)nv);
    double* sinv = (double*)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
    if (!cams || !sinv) { free(cams); free(sinv); return -2; }
    double* shift = cams + 16 * (size_t)nv;
    if (or_cameras(p, L0, cams, shift)) { free(cams); free(sinv); return -1; }
    const double pi = 3.14159265358979323846;
    const double focal = 0.5 * p->width / tan(0.5 * p->fov_x_deg * pi / 180.0);
    /* Sigma^-1 = R diag(s^-2) R^T (Eq. (8) inverted), upper triangle */
    for (int64_t g = 0; g < n; ++g) {
        const double* q = sc->rot_wxyz + 4 * g;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
        double R[3][3] = {
            {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
            {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
            {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        double is2[3];
        for (int i = 0; i < 3; ++i) is2[i] = exp(-2.0 * sc->log_scale[3 * g + i]);
        double* o = sinv + 6 * g;
        const int ij[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        for (int e = 0; e < 6; ++e) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[ij[e][0]][k] * is2[k] * R[ij[e][1]][k];
            o[e] = acc;
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_rays; ++i) {
        const double* T = cams + 16 * (int64_t)ray_v[i];
        const double dc[3] = {((double)ray_c[i] - 0.5 * p->width - shift[ray_v[i]]) / focal,
                              ((double)ray_r[i] - 0.5 * p->height) / focal, 1.0};
        double d[3], o[3], dn = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = T[4 * a] * dc[0] + T[4 * a + 1] * dc[1] + T[4 * a + 2] * dc[2];
            o[a] = T[4 * a + 3];
            dn += d[a] * d[a];
        }
        dn = sqrt(dn);
        for (int a = 0; a < 3; ++a) d[a] /= dn;
        double Y[16];
        or_sh_basis(d, Y);
        int64_t cap = 64, m = 0;
        or_contrib* L = (or_contrib*)malloc(sizeof(or_contrib) * (size_t)cap);
        double* col = (double*)malloc(sizeof(double) * 3 * (size_t)cap);
        for (int64_t g = 0; g < n; ++g) {
            const double* S = sinv + 6 * g;
            const double* mu = sc->mean + 3 * g;
            const double Sd[3] = {S[0] * d[0] + S[1] * d[1] + S[2] * d[2],
                                  S[1] * d[0] + S[3] * d[1] + S[4] * d[2],
                                  S[2] * d[0] + S[4] * d[1] + S[5] * d[2]};
            const double den = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
            const double t = ((mu[0] - o[0]) * Sd[0] + (mu[1] - o[1]) * Sd[1] +
                              (mu[2] - o[2]) * Sd[2]) / den;
            if (!(t > 0.2)) continue;
            const double x[3] = {o[0] + t * d[0] - mu[0], o[1] + t * d[1] - mu[1],
                                 o[2] + t * d[2] - mu[2]};
            const double qf = S[0] * x[0] * x[0] + S[3] * x[1] * x[1] + S[5] * x[2] * x[2] +
                              2.0 * (S[1] * x[0] * x[1] + S[2] * x[0] * x[2] + S[4] * x[1] * x[2]);
            if (qf > 120.0) continue; /* alpha < 1e-26 */
            double a = 1.0 / (1.0 + exp(-sc->opacity_logit[g])) * exp(-0.5 * qf);
            if (a > 0.99) a = 0.99;
            if (a < OR_ALPHA_MIN - 1e-6) continue;
            if (m == cap) {
                cap *= 2;
                L = (or_contrib*)realloc(L, sizeof(or_contrib) * (size_t)cap);
                col = (double*)realloc(col, sizeof(double) * 3 * (size_t)cap);
            }
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int j = 0; j < nc; ++j) acc += Y[j] * sc->sh[(g * nc + j) * 3 + k];
                acc += 0.5;
                col[3 * m + k] = acc > 0.0 ? acc : 0.0;
            }
            L[m].depth = t;
            L[m].idx = g;
            L[m].alpha = a;
            L[m].include = a >= OR_ALPHA_MIN;
            ++m;
        }
        for (int64_t j = 0; j < m; ++j) L[j].rgb = col + 3 * j;  /* arrays no longer move */
        qsort(L, (size_t)m, sizeof(or_contrib), or_cmp_contrib);
        double base[3], alt[3];
        or_composite_cap(L, m, OR_T_STOP, heap_cap, base);
        double* R3 = rgb + 3 * i;
        double* lo3 = lo + 3 * i;
        double* hi3 = hi + 3 * i;
        for (int k = 0; k < 3; ++k) R3[k] = lo3[k] = hi3[k] = base[k];
        int32_t f = 0;
        /* alternatives: alpha within 1e-6 of 1/255, t near-ties (|dt| <=
         * 2^-20 t, incl. the heap's last slot), T within 1e-8 of 1e-4 */
        for (int64_t j = 0; j < m; ++j)
            if (fabs(L[j].alpha - OR_ALPHA_MIN) < 1e-6) {
                f |= 2;
                L[j].include = !L[j].include;
                or_composite_cap(L, m, OR_T_STOP, heap_cap, alt);
                or_envelope(alt, lo3, hi3);
                L[j].include = !L[j].include;
            }
        {
            int64_t prev = -1;
            for (int64_t j = 0; j < m; ++j) {
                if (!L[j].include) continue;
                if (prev >= 0 && fabs(L[j].depth - L[prev].depth) <= ldexp(fabs(L[prev].depth), -20)) {
                    f |= 1;
                    or_contrib tmp = L[j];
                    L[j] = L[prev];
                    L[prev] = tmp;
                    or_composite_cap(L, m, OR_T_STOP, heap_cap, alt);
                    or_envelope(alt, lo3, hi3);
                    tmp = L[j];
                    L[j] = L[prev];
                    L[prev] = tmp;
                }
                prev = j;
            }
        }
        {
            double Tt = 1.0;
            int64_t kept = 0;
            for (int64_t j = 0; j < m && kept < heap_cap; ++j) {
                if (!L[j].include) continue;
                ++kept;
                double Tn = Tt * (1.0 - L[j].alpha);
                if (fabs(Tn - OR_T_STOP) < 1e-8) {
                    f |= 4;
                    or_composite_cap(L, m, OR_T_STOP + 2e-8, heap_cap, alt);
                    or_envelope(alt, lo3, hi3);
                    or_composite_cap(L, m, OR_T_STOP - 2e-8, heap_cap, alt);
                    or_envelope(alt, lo3, hi3);
                    break;
                }
                if (Tn < OR_T_STOP) break;
                Tt = Tn;
            }
        }
        if (flags) flags[i] = f;
        free(L);
        free(col);
    }
    free(cams);
    free(sinv);
    return 0;
}

int or_interweave(const or_display* p, const uint16_t* V, const double* Mm, double* Me) {
    if (or_check_display(p)) return -1;
    const int64_t w = p->width, h = p->height;
    for (int64_t x = 0; x < h; ++x)
        for (int64_t y = 0; y < w; ++y)
            for (int64_t k = 0; k < 3; ++k) {
                int64_t v = V[x * 3 * w + 3 * y + k];
                if (v >= p->num_views) return -1;
                Me[(x * w + y) * 3 + k] = Mm[((v * h + x) * w + y) * 3 + k];
            }
    return 0;
}
