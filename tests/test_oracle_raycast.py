"""Pins of the oracle's ray-order 3DGS (Sec. 7, Alg. 3): the highest-density
point t_j and alpha_j of Eqs. (16)-(17) against closed forms and the
maximisation they define, the heap capacity, and the SH colour taken at the
ray direction."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

Y00 = 0.5 / math.sqrt(math.pi)


def _scene(means, log_scales, rots, opac_logit, rgb, sh_deg=0, sh_hi=None):
    n = len(means)
    nc = (sh_deg + 1) ** 2
    sh = np.zeros((n, nc, 3), np.float64)
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    if sh_hi is not None:
        sh[:, 1:, :] = sh_hi
    return oracle.Scene({"mean": np.asarray(means, np.float64), "log_scale": np.asarray(log_scales, np.float64),
                         "rot_wxyz": np.asarray(rots, np.float64),
                         "opacity_logit": np.asarray(opac_logit, np.float64), "sh": sh,
                         "sh_degree": sh_deg})


D = W.Display(64, 48, 1, 5.3, 1 / 6, view_span_deg=0.0)
L0 = W.light_field_centre(4.0, 0.0)  # camera at (0, 0, -4) looking along +z


def _ray_to(point):
    """(view 0, row, col) of the pixel whose ray passes closest to `point`."""
    f = oracle.focal(D)
    x, y, z = point[0], point[1], point[2] + 4.0
    return [0, int(round(y / z * f + D.height / 2)), int(round(x / z * f + D.width / 2))]


def _dir(ray):
    f = oracle.focal(D)
    d = np.array([(ray[2] - D.width / 2) / f, (ray[1] - D.height / 2) / f, 1.0])
    return d / np.linalg.norm(d)


def _logit(p):
    return math.log(p / (1 - p))


def test_isotropic_gaussian_closed_form():
    # ray with unit direction d from o=(0,0,-4); an isotropic Gaussian of
    # sigma s at mu: t = (mu - o).d and alpha = opacity * exp(-rho^2 / (2 s^2)),
    # rho the distance from mu to the ray
    s, op = 0.3, 0.8
    ray = [0, 20, 40]
    d = _dir(ray)
    o = np.array([0.0, 0.0, -4.0])
    mu = o + 3.1 * d + np.array([0.05, -0.02, 0.0])
    sc = _scene([mu], [[math.log(s)] * 3], [[1, 0, 0, 0]], [_logit(op)], [[0.2, 0.5, 0.9]])
    res = oracle.raycast_rays(sc, D, L0, np.array([ray]))
    t = (mu - o) @ d
    rho2 = np.sum((o + t * d - mu) ** 2)
    alpha = op * math.exp(-rho2 / (2 * s * s))
    assert np.allclose(res["rgb"][0], alpha * np.array([0.2, 0.5, 0.9]), atol=1e-12)


def test_t_maximises_the_density_along_the_ray():
    rng = np.random.default_rng(3)
    ray = [0, 30, 17]
    d = _dir(ray)
    o = np.array([0.0, 0.0, -4.0])
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    ls = np.log([0.5, 0.12, 0.3])
    mu = o + 4.0 * d + np.array([0.1, 0.05, -0.2])
    sc = _scene([mu], [ls], [q], [_logit(0.9)], [[1.0, 1.0, 1.0]])
    got = oracle.raycast_rays(sc, D, L0, np.array([ray]))["rgb"][0, 0]
    # Sigma from the same parametrisation, alpha along the ray by brute force
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    Si = R @ np.diag(np.exp(-2 * ls)) @ R.T
    ts = np.linspace(0.5, 8.0, 200001)
    pts = o + ts[:, None] * d - mu
    dens = np.exp(-0.5 * np.einsum("ni,ij,nj->n", pts, Si, pts))
    assert got == pytest.approx(0.9 * dens.max(), rel=1e-8)


def test_heap_keeps_the_nearest_and_sh_uses_the_ray_direction():
    # three opaque-ish Gaussians stacked along one ray: capacity 1 keeps the
    # nearest only, capacity 3 composites all three front to back
    ray = [0, 24, 32]
    d = _dir(ray)
    o = np.array([0.0, 0.0, -4.0])
    mus = [o + t * d for t in (5.0, 3.0, 4.0)]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    sc = _scene(mus, [[math.log(0.2)] * 3] * 3, [[1, 0, 0, 0]] * 3, [_logit(0.6)] * 3, cols)
    one = oracle.raycast_rays(sc, D, L0, np.array([ray]), heap_cap=1)["rgb"][0]
    assert np.allclose(one, [0.0, 0.6, 0.0])  # t = 3 is the nearest
    three = oracle.raycast_rays(sc, D, L0, np.array([ray]), heap_cap=3)["rgb"][0]
    assert np.allclose(three, [0.6 * 0.16, 0.6, 0.6 * 0.4])  # t order 3, 4, 5
    # degree-1 SH: colour = SH + 0.5 at the ray's own direction d, not at
    # the direction to the Gaussian's centre (the centre sits off the ray)
    ray2 = [0, 10, 50]
    d2 = _dir(ray2)
    mu = o + 3.0 * d2 + np.array([0.0, 0.04, 0.0])
    hi = np.zeros((1, 3, 3))
    hi[0, 1, 0] = 0.4  # degree-1 coefficient of z on the red channel (basis term 2)
    hi[0, 2, 0] = 0.3  # degree-1 coefficient of x on the red channel (basis term 3)
    sc1 = _scene([mu], [[math.log(0.2)] * 3], [[1, 0, 0, 0]], [_logit(0.5)],
                 [[0.5, 0.5, 0.5]], sh_deg=1, sh_hi=hi)
    got = oracle.raycast_rays(sc1, D, L0, np.array([ray2]))["rgb"][0]
    t = (mu - o) @ d2
    alpha = 0.5 * math.exp(-np.sum((o + t * d2 - mu) ** 2) / (2 * 0.2 * 0.2))
    b = oracle.sh_basis(d2)
    assert got[0] == pytest.approx(alpha * (0.5 + 0.4 * b[2] + 0.3 * b[3]), rel=1e-10)
    b_centre = oracle.sh_basis((mu - o) / np.linalg.norm(mu - o))
    assert abs(alpha * (0.5 + 0.4 * b_centre[2] + 0.3 * b_centre[3]) - got[0]) > 1e-6


def test_near_plane_and_misses():
    ray = [0, 24, 32]
    d = _dir(ray)
    o = np.array([0.0, 0.0, -4.0])
    sc = _scene([o + 0.1 * d, o + 2.0 * d + np.array([5.0, 0, 0])], [[math.log(0.05)] * 3] * 2,
                [[1, 0, 0, 0]] * 2, [_logit(0.9)] * 2, [[1, 1, 1]] * 2)
    assert np.allclose(oracle.raycast_rays(sc, D, L0, np.array([ray]))["rgb"], 0.0)
