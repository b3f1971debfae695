"""Pins of the oracle's cameras, 3DGS projection and compositing.

Cameras (Sec. 3.1, multiview rendering; Eq. (17)): on an arc of the given
radius and angular span, evenly spaced, every one looking at the centre.
Projection (Sec. 3.3, Eqs. (8)-(9)): the 2D covariance equals J Sigma_cam J^T
+ 0.3 I with J taken by finite differences of the pinhole map and Sigma from
scipy's own quaternion rotation; the on-axis isotropic closed form.
SH colour: the real basis satisfies the addition theorem and is orthonormal.
Compositing (Eqs. (5), (10)): 1-3 Gaussians against the back-to-front
"over" recursion written out by hand; the early stop; independence of the
input order; the near plane; Alg. 1 (render every view, then interweave)
against the per-subpixel definition."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

Y00 = 0.5 / math.sqrt(math.pi)


def _scene(means, log_scales, opacities, rgbs, quats=None, sh=None, deg=0):
    n = len(means)
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    logits = [math.log(o / (1.0 - o)) for o in opacities]
    if sh is None:
        sh = ((np.asarray(rgbs, dtype=np.float64) - 0.5) / Y00).reshape(n, 1, 3)
    return oracle.Scene({"mean": np.asarray(means, float), "log_scale": np.asarray(log_scales, float),
                         "rot_wxyz": np.asarray(quats, float), "opacity_logit": np.asarray(logits, float),
                         "sh": np.asarray(sh, float), "sh_degree": deg})


# ----------------------------------------------------------------- cameras --
def test_camera_arc():
    d = W.WORKLOADS["tiny"].display
    L0 = W.light_field_centre(4.0, yaw_deg=7.0)
    C = oracle.cameras(d, L0)
    centres = C[:, :3, 3]
    assert np.allclose(np.linalg.norm(centres, axis=1), 4.0, atol=1e-12)
    # even spacing over the span
    u = centres / 4.0
    ang = np.degrees(np.arccos(np.clip(np.sum(u[1:] * u[:-1], axis=1), -1, 1)))
    assert np.allclose(ang, d.view_span_deg / (d.num_views - 1), atol=1e-9)
    first_last = np.degrees(np.arccos(np.dot(u[0], u[-1])))
    assert abs(first_last - d.view_span_deg) < 1e-9
    # every camera looks at the origin: the origin maps to camera (0, 0, 4)
    for T in C:
        Rc, c = T[:3, :3], T[:3, 3]
        assert np.allclose(Rc.T @ Rc, np.eye(3), atol=1e-12)
        assert np.allclose(Rc.T @ (np.zeros(3) - c), [0, 0, 4.0], atol=1e-12)
    # view 0 is the leftmost along the centre camera's x axis
    xs = centres @ L0[:3, 0]
    assert np.all(np.diff(xs) > 0)
    Cr = oracle.cameras(d.replace(reverse_views=1), L0)
    assert np.allclose(Cr, C[::-1])
    assert np.allclose(oracle.cameras(d.replace(num_views=1), L0)[0], L0)


# ----------------------------------------------------------------- SH basis --
def test_sh_addition_theorem():
    rng = np.random.default_rng(3)
    for _ in range(20):
        dvec = rng.normal(size=3)
        dvec /= np.linalg.norm(dvec)
        Y = oracle.sh_basis(dvec)
        for l, (a, b) in enumerate([(0, 1), (1, 4), (4, 9), (9, 16)]):
            assert abs(np.sum(Y[a:b] ** 2) - (2 * l + 1) / (4 * math.pi)) < 1e-12


def test_sh_orthonormal():
    mu, wmu = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * 2 * math.pi / 32
    G = np.zeros((16, 16))
    for m, wm in zip(mu, wmu):
        s = math.sqrt(1 - m * m)
        for ph in phis:
            Y = oracle.sh_basis([s * math.cos(ph), s * math.sin(ph), m])
            G += wm * (2 * math.pi / 32) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_colour_reproduces_degree_two_function():
    # coefficients of f(d) = d_x d_y + 0.3 d_z - 0.1 by quadrature projection
    f = lambda d: d[0] * d[1] + 0.3 * d[2] - 0.1
    mu, wmu = np.polynomial.legendre.leggauss(16)
    coef = np.zeros(16)
    for m, wm in zip(mu, wmu):
        s = math.sqrt(1 - m * m)
        for j in range(32):
            ph = j * 2 * math.pi / 32
            dv = [s * math.cos(ph), s * math.sin(ph), m]
            coef += wm * (2 * math.pi / 32) * f(dv) * oracle.sh_basis(dv)
    sh = np.zeros((1, 16, 3))
    sh[0, :, 0] = coef
    sh[0, :, 1] = 0.5 * coef
    mean = np.array([[0.4, -0.3, 0.2]])
    sc = _scene(mean, [[-3, -3, -3]], [0.5], None, sh=sh, deg=3)
    L0 = W.light_field_centre(4.0)
    d = W.WORKLOADS["tiny"].display
    p = oracle.project(sc, 0, L0, d)
    dvec = mean[0] - L0[:3, 3]
    dvec /= np.linalg.norm(dvec)
    assert abs(p["rgb"][0] - (f(dvec) + 0.5)) < 1e-10
    assert abs(p["rgb"][1] - (0.5 * f(dvec) + 0.5)) < 1e-10
    assert abs(p["rgb"][2] - 0.5) < 1e-12


# --------------------------------------------------------------- projection --
def test_isotropic_on_axis_closed_form():
    d = W.WORKLOADS["tiny"].display
    L0 = W.light_field_centre(4.0)
    f = oracle.focal(d)
    for z, ls in [(4.0, -3.0), (2.5, -2.0), (7.0, -4.0)]:
        sc = _scene([[0.0, 0.0, z - 4.0]], [[ls] * 3], [0.7], [[0.2, 0.4, 0.6]])
        p = oracle.project(sc, 0, L0, d)
        var = (f * math.exp(ls) / z) ** 2 + 0.3
        assert p["valid"] and abs(p["depth"] - z) < 1e-12
        assert abs(p["u"] - d.width / 2) < 1e-9 and abs(p["v"] - d.height / 2) < 1e-9
        assert np.allclose(p["cov2d"], [var, 0.0, var], rtol=1e-12, atol=1e-12)
        assert np.allclose(p["conic"], [1 / var, 0.0, 1 / var], rtol=1e-12)
        assert abs(p["opacity"] - 0.7) < 1e-12
        assert np.allclose(p["rgb"], [0.2, 0.4, 0.6], atol=1e-12)


def test_anisotropic_matches_finite_difference_jacobian():
    from scipy.spatial.transform import Rotation
    d = W.WORKLOADS["tiny"].display
    f = oracle.focal(d)
    rng = np.random.default_rng(5)
    C = oracle.cameras(d, W.light_field_centre(4.0, 3.0))
    for _ in range(10):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        mean = rng.uniform(-0.6, 0.6, size=3)
        ls = rng.normal(-2.5, 0.5, size=3)
        sc = _scene([mean], [ls], [0.5], [[0.5, 0.5, 0.5]], quats=[q * 1.7])
        T = C[rng.integers(0, d.num_views)]
        p = oracle.project(sc, 0, T, d)
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar last
        Sig = Rm @ np.diag(np.exp(2 * ls)) @ Rm.T
        Rw = T[:3, :3].T
        t = Rw @ (mean - T[:3, 3])
        Sc = Rw @ Sig @ Rw.T

        def proj(tt):
            return np.array([f * tt[0] / tt[2] + d.width / 2, f * tt[1] / tt[2] + d.height / 2])

        h = 1e-6
        J = np.stack([(proj(t + h * e) - proj(t - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        cov = J @ Sc @ J.T + 0.3 * np.eye(2)
        assert np.allclose(p["cov2d"], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6)
        assert np.allclose(p["depth"], t[2], rtol=1e-12)
        assert np.allclose([p["u"], p["v"]], proj(t), rtol=1e-12)


def test_near_plane_culls():
    d = W.WORKLOADS["tiny"].display
    L0 = W.light_field_centre(4.0)
    sc = _scene([[0, 0, -3.85], [0, 0, 0.0]], [[-3] * 3] * 2, [0.9, 0.5], [[1, 0, 0], [0, 1, 0]])
    assert not oracle.project(sc, 0, L0, d)["valid"]       # depth 0.15 <= 0.2
    r = oracle.render_rays(sc, d, L0, [[22, 67, 120]])
    # centre view (22 of 45) sees only the second Gaussian at the image centre
    C = oracle.cameras(d, L0)[22]
    p = oracle.project(sc, 1, C, d)
    a = 0.5 * math.exp(-0.5 * (p["conic"][0] * (120 - p["u"]) ** 2 + 2 * p["conic"][1] * (120 - p["u"]) * (67 - p["v"])
                               + p["conic"][2] * (67 - p["v"]) ** 2))
    assert np.allclose(r["rgb"][0], [0, a, 0], atol=1e-12)


# -------------------------------------------------------------- compositing --
def _axis_scene(depths, log_scales, opacities, rgbs):
    return _scene([[0.0, 0.0, z - 4.0] for z in depths], [[s] * 3 for s in log_scales], opacities, rgbs)


def _over(alphas, colours):
    """Back-to-front 'over' recursion: C = a_i c_i + (1 - a_i) C_behind."""
    C = np.zeros(3)
    for a, c in reversed(list(zip(alphas, colours))):
        C = a * np.asarray(c) + (1.0 - a) * C
    return C


@pytest.mark.parametrize("n", [1, 2, 3])
def test_brute_force_small_stacks(n):
    d = W.Display(64, 48, 1, 5.3, 1 / 6, view_span_deg=0.0)
    L0 = W.light_field_centre(4.0)
    f = oracle.focal(d)
    depths = [3.0, 4.0, 5.5][:n]
    scales = [-3.2, -2.9, -2.6][:n]
    ops = [0.6, 0.8, 0.9][:n]
    cols = [[0.9, 0.1, 0.2], [0.2, 0.7, 0.3], [0.1, 0.3, 0.95]][:n]
    perm = np.random.default_rng(n).permutation(n)            # input order must not matter
    sc = _axis_scene([depths[i] for i in perm], [scales[i] for i in perm], [ops[i] for i in perm],
                     [cols[i] for i in perm])
    rays = [[0, 24 + dr, 32 + dc] for dr, dc in [(0, 0), (1, 2), (-3, 4), (6, -5), (12, 9)]]
    got = oracle.render_rays(sc, d, L0, rays)
    for (v, r, c), rgb in zip(rays, got["rgb"]):
        rr = (r - 24) ** 2 + (c - 32) ** 2
        alphas, colours = [], []
        for z, s, o, col in zip(depths, scales, ops, cols):       # nearest first
            var = (f * math.exp(s) / z) ** 2 + 0.3
            a = min(0.99, o * math.exp(-0.5 * rr / var))
            if a >= 1 / 255:
                alphas.append(a)
                colours.append(col)
        assert np.allclose(rgb, _over(alphas, colours), atol=1e-12)


def test_early_stop_before_transmittance_drops_below_threshold():
    d = W.Display(32, 32, 1, 5.3, 1 / 6, view_span_deg=0.0)
    L0 = W.light_field_centre(4.0)
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]]
    sc = _axis_scene([2.0, 2.5, 3.0, 3.5, 4.0], [-1.0] * 5, [0.95] * 5, cols)
    got = oracle.render_rays(sc, d, L0, [[0, 16, 16]])
    # T after k layers is 0.05^k: 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4,
    # so the fourth and fifth Gaussians are never composited.
    expect = 0.95 * (np.array(cols[0]) + 0.05 * np.array(cols[1]) + 0.0025 * np.array(cols[2]))
    assert np.allclose(got["rgb"][0], expect, atol=1e-12)
    assert got["n_contrib"][0] == 3


def test_alpha_clamp_and_threshold():
    d = W.Display(32, 32, 1, 5.3, 1 / 6, view_span_deg=0.0)
    L0 = W.light_field_centre(4.0)
    f = oracle.focal(d)
    sc = _axis_scene([3.0], [-3.0], [0.999], [[0.3, 0.6, 0.9]])
    var = (f * math.exp(-3.0) / 3.0) ** 2 + 0.3
    # the radius where alpha crosses 1/255
    r_cut = math.sqrt(2 * var * math.log(255 * 0.999))
    rays = [[0, 16, 16], [0, 16, 16 + int(math.floor(r_cut))], [0, 16, 16 + int(math.ceil(r_cut))]]
    got = oracle.render_rays(sc, d, L0, rays)
    assert np.allclose(got["rgb"][0], 0.99 * np.array([0.3, 0.6, 0.9]), atol=1e-12)
    a_in = 0.999 * math.exp(-0.5 * math.floor(r_cut) ** 2 / var)
    assert a_in >= 1 / 255
    assert np.allclose(got["rgb"][1], a_in * np.array([0.3, 0.6, 0.9]), atol=1e-12)
    assert np.allclose(got["rgb"][2], 0.0)


def test_alg1_interweave_equals_per_subpixel_standard():
    d = W.Display(24, 16, 5, 5.3, 1 / 6, view_span_deg=20.0)
    L0 = W.light_field_centre(4.0)
    scd = W.make_scene(W.SceneSpec(300, 1, "uniform", "f32", seed=4))
    sc = oracle.Scene(scd)
    # Alg. 1: render every view at native resolution, then interweave
    vv, rr, cc = np.meshgrid(np.arange(d.num_views), np.arange(d.height), np.arange(d.width), indexing="ij")
    rays = np.stack([vv.ravel(), rr.ravel(), cc.ravel()], axis=1)
    Mm = oracle.render_rays(sc, d, L0, rays)["rgb"].reshape(d.num_views, d.height, d.width, 3)
    V = oracle.view_map(d)
    Me = oracle.interweave(d, V, Mm)
    E = oracle.render_frame(sc, d, L0, mode="standard")["value"]
    assert np.array_equal(Me, E)
    # identity repurposing: DirectL gives the standard paradigm's image
    Ed = oracle.render_frame(sc, d.replace(repurpose=0), L0, mode="directl")["value"]
    assert np.array_equal(Ed, E)
    assert np.abs(E).max() > 0.05


# ---- the off-axis (straight-line) rig of Sec. 3.2 -------------------------
def _theta(d, v):
    return math.radians(-0.5 * d.view_span_deg + v * d.view_span_deg / (d.num_views - 1))


def test_off_axis_rig_cameras():
    d = W.Display(240, 135, 9, 5.3, 1 / 6, view_span_deg=24.0, rig=1)
    L0 = W.light_field_centre(4.0, 7.0)
    c2w, shift = oracle.cameras(d, L0, with_shift=True)
    f = oracle.focal(d)
    for v in range(d.num_views):
        xv = 4.0 * math.tan(_theta(d, v))
        assert np.array_equal(c2w[v, :3, :3], L0[:3, :3])            # parallel axes
        assert np.allclose(c2w[v, :3, 3], L0[:3, 3] + xv * L0[:3, 0], atol=1e-12)
        assert shift[v] == pytest.approx(f * xv / 4.0, rel=1e-12)
    assert c2w[0, :3, 3] @ L0[:3, 0] < c2w[-1, :3, 3] @ L0[:3, 0]     # view 0 leftmost
    arc = oracle.cameras(d.replace(rig=0), L0)
    assert np.allclose(arc[4], c2w[4], atol=1e-12)                     # same centre view
    with pytest.raises(RuntimeError):                                  # origin behind L0
        flipped = L0.copy()
        flipped[:3, 2] *= -1.0
        flipped[:3, 0] *= -1.0
        oracle.cameras(d, flipped)


def test_off_axis_rig_has_no_parallax_on_the_convergence_plane():
    d = W.Display(240, 135, 7, 5.3, 1 / 6, view_span_deg=30.0, rig=1)
    L0 = W.light_field_centre(4.0, 0.0)            # optical axis = world +z, origin at depth 4
    c2w, shift = oracle.cameras(d, L0, with_shift=True)
    sc = W.make_scene(W.SceneSpec(3, 0, "uniform", "f32", seed=1))
    sc["mean"][:] = np.array([[0.3, -0.2, 0.0], [0.1, 0.15, -1.0], [-0.2, 0.1, 1.5]], np.float32)
    scene = oracle.Scene(sc)
    us = np.array([[oracle.project(scene, g, c2w[v], d, shift[v])["u"] for v in range(7)]
                   for g in range(3)])
    vs = np.array([[oracle.project(scene, g, c2w[v], d, shift[v])["v"] for v in range(7)]
                   for g in range(3)])
    assert np.ptp(us[0]) < 1e-9 and np.ptp(vs[0]) < 1e-9   # on the plane: one pixel in all views
    assert np.all(np.diff(us[1]) < 0)                        # nearer: moves left as x_v grows
    assert np.all(np.diff(us[2]) > 0)                        # farther: moves right
    assert np.ptp(vs[1]) < 1e-9                              # a horizontal rig: rows do not move


# ---- the standard paradigm below panel resolution (Alg. 1, Resize) --------
def test_bilinear_taps_match_scipy_order_one_sampling():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    img = rng.normal(size=(9, 16))
    w, h = 48, 27  # panel; the view is 16 x 9 (the 4K panel's LR aspect)
    r, c = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    x0, x1, fx = oracle.bilinear_taps(w, 16, c.ravel())
    y0, y1, fy = oracle.bilinear_taps(h, 9, r.ravel())
    ours = ((1 - fy) * ((1 - fx) * img[y0, x0] + fx * img[y0, x1]) +
            fy * ((1 - fx) * img[y1, x0] + fx * img[y1, x1]))
    ref = ndimage.map_coordinates(img, [r.ravel() * 9 / h, c.ravel() * 16 / w], order=1,
                                  mode="nearest")
    assert np.allclose(ours, ref, atol=1e-12)
    # the last columns and rows clamp at the border
    assert x0.max() == 15 and x1.max() == 15 and y1.max() == 8


def test_lowres_standard_at_panel_resolution_is_the_standard_frame():
    d = W.Display(48, 27, 5, 5.3, 1 / 6, view_span_deg=10.0)
    sc = oracle.Scene(W.make_scene(W.SceneSpec(150, 1, "uniform", "f32", seed=2)))
    L0 = W.light_field_centre(4.0, 1.0)
    V = oracle.view_map(d)
    sub = np.arange(3 * d.width * d.height)
    hr = oracle.render_subpixels(sc, d, L0, sub, V, None)
    same = oracle.render_subpixels_lowres(sc, d, L0, sub, V, d.width, d.height)
    assert np.array_equal(same["value"], hr["value"])
    # views of a third of the panel: every subpixel is a convex mix of the
    # four view pixels around its position, so it lies within their range
    low = oracle.render_subpixels_lowres(sc, d, L0, sub, V, 16, 9)
    small = d.replace(width=16, height=9)
    vv, rr, cc = np.meshgrid(np.arange(5), np.arange(9), np.arange(16), indexing="ij")
    views = oracle.render_rays(sc, small, L0, np.stack([vv.ravel(), rr.ravel(), cc.ravel()], 1))
    img = views["rgb"].reshape(5, 9, 16, 3)
    row, col, k = sub // (3 * d.width), (sub % (3 * d.width)) // 3, sub % 3
    v = V.reshape(-1)[sub]
    x0, x1, _ = oracle.bilinear_taps(d.width, 16, col)
    y0, y1, _ = oracle.bilinear_taps(d.height, 9, row)
    taps = np.stack([img[v, y0, x0, k], img[v, y0, x1, k], img[v, y1, x0, k], img[v, y1, x1, k]])
    assert np.all(low["value"] >= taps.min(0) - 1e-12) and np.all(low["value"] <= taps.max(0) + 1e-12)
