"""Pins of the oracle's envelope of alternative results (readings c16-c17).

Several results are correct where FP32 cannot decide: two contributors'
depths within 2^-20 z of each other (either order), an alpha within 1e-6 of
the 1/255 cut of Eq. (10)'s alpha rules (either decision), a transmittance
within 1e-8 of the 1e-4 stop (either decision).  The oracle returns the
value and [lo, hi] over those alternatives.  Each case here is built from
two to six Gaussians on the optical axis of a one-view panel, seen at the
centre pixel, where alpha equals the opacity exactly, so every alternative
is written out by hand with the compositing sum of Eq. (5).  The envelope
must equal the hand-computed alternatives and be no wider."""
import itertools
import math

import numpy as np
import pytest

import envelope
import oracle
import workloads as W

Y00 = 0.5 / math.sqrt(math.pi)
DISPLAY = W.Display(32, 32, 1, 5.3, 1 / 6, view_span_deg=0.0)
CENTRE = [[0, 16, 16]]   # (view, row, col): the principal point, on the optical axis
L0 = W.light_field_centre(4.0)


def _render(depths, alphas, colours):
    n = len(depths)
    sc = oracle.Scene({
        "mean": np.array([[0.0, 0.0, z - 4.0] for z in depths]),
        "log_scale": np.full((n, 3), -3.0),
        "rot_wxyz": np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)),
        "opacity_logit": np.array([math.log(a / (1.0 - a)) for a in alphas]),
        "sh": ((np.asarray(colours, float) - 0.5) / Y00).reshape(n, 1, 3),
        "sh_degree": 0})
    r = oracle.render_rays(sc, DISPLAY, L0, CENTRE)
    return r["rgb"][0], r["lo"][0], r["hi"][0], int(r["flags"][0])


def _sum(layers, t_stop=1e-4):
    """Eq. (5) front to back over (alpha, colour) in the given order, with the
    early stop before the layer that would take T below t_stop."""
    T, C = 1.0, np.zeros(3)
    for a, c in layers:
        if T * (1.0 - a) < t_stop:
            break
        C = C + a * T * np.asarray(c, float)
        T *= 1.0 - a
    return C


def _env(*values):
    v = np.array(values)
    return v.min(0), v.max(0)


C1, C2, C3 = [0.9, 0.2, 0.1], [0.1, 0.5, 0.8], [0.3, 0.9, 0.4]


@pytest.mark.parametrize("delta", [5e-7, -5e-7])
def test_alpha_inside_the_window_gives_both_decisions(delta):
    a1 = 1 / 255 + delta
    rgb, lo, hi, f = _render([3.0, 5.0], [a1, 0.6], [C1, C2])
    with_front = _sum([(a1, C1), (0.6, C2)])
    without = _sum([(0.6, C2)])
    assert f == 2
    assert np.allclose(rgb, with_front if delta > 0 else without, rtol=0, atol=1e-15)
    elo, ehi = _env(with_front, without)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)


@pytest.mark.parametrize("delta", [3e-6, -3e-6])
def test_alpha_outside_the_window_is_exact(delta):
    a1 = 1 / 255 + delta
    rgb, lo, hi, f = _render([3.0, 5.0], [a1, 0.6], [C1, C2])
    expect = _sum([(a1, C1), (0.6, C2)] if delta > 0 else [(0.6, C2)])
    assert f == 0
    assert np.allclose(rgb, expect, rtol=0, atol=1e-15)
    assert np.array_equal(lo, rgb) and np.array_equal(hi, rgb)


def test_depth_near_tie_gives_both_orders():
    z2 = 4.0 + 2.0 ** -19           # |dz| = 2^-21 z
    rgb, lo, hi, f = _render([4.0, z2], [0.5, 0.7], [C1, C2])
    first = _sum([(0.5, C1), (0.7, C2)])
    swapped = _sum([(0.7, C2), (0.5, C1)])
    assert f == 1
    assert np.allclose(rgb, first, rtol=0, atol=1e-15)
    elo, ehi = _env(first, swapped)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)


def test_depth_beyond_the_tie_resolution_is_exact():
    z2 = 4.0 + 2.0 ** -17           # |dz| = 2^-19 z
    rgb, lo, hi, f = _render([z2, 4.0], [0.5, 0.7], [C1, C2])
    assert f == 0
    assert np.allclose(rgb, _sum([(0.7, C2), (0.5, C1)]), rtol=0, atol=1e-15)
    assert np.array_equal(lo, rgb) and np.array_equal(hi, rgb)


def test_tie_chain_swaps_only_consecutive_pairs():
    # z0 ~ z1 and z1 ~ z2 within 2^-20 z, but z0 and z2 are not: the
    # alternatives are the two adjacent swaps, not every permutation
    z = [4.0, 4.0 + 3 * 2.0 ** -20, 4.0 + 6 * 2.0 ** -20]
    a = [0.8, 0.5, 0.9]
    cols = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]
    rgb, lo, hi, f = _render(z, a, cols)
    layer = list(zip(a, cols))
    allowed = [_sum([layer[i] for i in p]) for p in ((0, 1, 2), (1, 0, 2), (0, 2, 1))]
    assert f == 1
    assert np.allclose(rgb, allowed[0], rtol=0, atol=1e-15)
    elo, ehi = _env(*allowed)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)
    # every permutation would be wider: (2, 1, 0) puts blue at 0.9
    plo, phi = _env(*[_sum([layer[i] for i in p]) for p in itertools.permutations(range(3))])
    assert phi[2] > hi[2] + 0.5


def _three_layers_then(alpha3_gap):
    """Layers of alpha 0.9, 0.9, a3, 0.5 where a3 leaves T = 1e-4 + gap."""
    T2 = (1.0 - 0.9) * (1.0 - 0.9)
    a3 = 1.0 - (1e-4 + alpha3_gap) / T2
    return [2.0, 3.0, 4.0, 5.0], [0.9, 0.9, a3, 0.5], [C1, C2, C3, [0.5, 0.5, 0.5]]


def test_transmittance_inside_the_window_gives_both_decisions():
    z, a, cols = _three_layers_then(5e-9)
    rgb, lo, hi, f = _render(z, a, cols)
    layers = list(zip(a, cols))
    with3 = _sum(layers[:3])            # the fourth would take T to 5e-5: never composited
    without3 = _sum(layers[:2])
    assert f == 4
    assert np.allclose(rgb, with3, rtol=0, atol=1e-15)
    elo, ehi = _env(with3, without3)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)


def test_transmittance_outside_the_window_is_exact():
    z, a, cols = _three_layers_then(5e-8)
    rgb, lo, hi, f = _render(z, a, cols)
    assert f == 0
    assert np.allclose(rgb, _sum(list(zip(a, cols))[:3]), rtol=0, atol=1e-15)
    assert np.array_equal(lo, rgb) and np.array_equal(hi, rgb)


def test_alpha_window_ends_at_the_stopping_contributor():
    # T = 0.05^3 = 1.25e-4 after three layers; the 0.5 layer would take it
    # below 1e-4 and stops compositing.  A near-1/255 layer behind it cannot
    # change the result and is not flagged; in front of it, it is.
    a_near = 1 / 255 + 5e-7
    base = [1.0, 1.5, 2.0, 4.0]
    alphas = [0.95, 0.95, 0.95, 0.5]
    cols = [C1, C2, C3, [0.2, 0.2, 0.2]]
    rgb, lo, hi, f = _render(base + [4.5], alphas + [a_near], cols + [[1.0, 1.0, 1.0]])
    assert f == 0 and np.array_equal(lo, rgb) and np.array_equal(hi, rgb)
    assert np.allclose(rgb, _sum(list(zip(alphas, cols))), rtol=0, atol=1e-15)
    rgb, lo, hi, f = _render(base[:3] + [3.0, 4.0], alphas[:3] + [a_near, 0.5],
                             cols[:3] + [[1.0, 1.0, 1.0], [0.2, 0.2, 0.2]])
    assert f == 2
    layers = list(zip(alphas[:3], cols[:3]))
    with_near = _sum(layers + [(a_near, [1.0, 1.0, 1.0]), (0.5, [0.2, 0.2, 0.2])])
    without = _sum(layers + [(0.5, [0.2, 0.2, 0.2])])
    elo, ehi = _env(with_near, without)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)


def test_tie_with_the_stopper_reaches_past_an_excluded_candidate():
    # the stopper S (alpha 0.5 at depth 4) ties with Y (alpha 0.1) although a
    # candidate X just below 1/255 lies between them.  Swapped, Y composites
    # before S stops: T = 1.25e-4 * 0.9 >= 1e-4.
    cY = [50.0, 0.0, 0.0]
    z = [1.0, 1.5, 2.0, 4.0, 4.0 + 2.0 ** -20, 4.0 + 2.0 ** -19]
    a = [0.95, 0.95, 0.95, 0.5, 1 / 255 - 5e-7, 0.1]
    cols = [C1, C2, C3, [0.2, 0.2, 0.2], [1.0, 1.0, 1.0], cY]
    rgb, lo, hi, f = _render(z, a, cols)
    layers = list(zip(a, cols))
    base = _sum(layers[:3])
    swapped = _sum(layers[:3] + [layers[5], layers[3]])
    assert f == 1
    assert np.allclose(rgb, base, rtol=0, atol=1e-15)
    assert swapped[0] - base[0] == pytest.approx(1.25e-4 * 0.1 * 50.0, rel=1e-9)
    elo, ehi = _env(base, swapped)
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)


def test_unflagged_subpixels_have_no_envelope_and_wide_ones_are_rare():
    wl = W.WORKLOADS["tiny"]
    r = oracle.render_frame(oracle.Scene(W.make_scene(wl.scene)), wl.display,
                            W.light_field_centre(wl.camera_distance, 3.0), mode="directl")
    val, lo, hi = r["value"], r["lo"], r["hi"]
    flags = np.repeat(r["flags"].reshape(-1, 1), 1, axis=1).reshape(val.shape)
    plain = flags == 0
    assert np.array_equal(lo[plain], val[plain]) and np.array_equal(hi[plain], val[plain])
    assert np.all(lo <= val) and np.all(val <= hi)
    # an alternative decision can move a value by more than the 2e-3
    # tolerance only where the envelope is that wide: 1.3e-4 of this frame
    wide = float((hi - lo > 2e-3).mean())
    assert wide < envelope.RELIED_MAX_FRACTION
    n = val.size
    print(f"tiny DirectL frame: {n} subpixels, flagged {int((~plain).sum())}, "
          f"envelope wider than 2e-3 at {wide:.2e}")


def test_accept_counts():
    ref = {"value": np.array([0.5, 0.5, 0.5, 0.5]), "lo": np.array([0.5, 0.49, 0.5, 0.5]),
           "hi": np.array([0.5, 0.51, 0.5, 0.5]), "flags": np.array([0, 2, 0, 1])}
    got = np.array([0.5005, 0.507, 0.6, 0.5])
    ok, maxerr, nbad, st = envelope.accept(got, ref, 2e-3, "unit")
    envelope.RECORDS.remove(st)
    assert list(ok) == [True, True, False, True]
    assert nbad == 1 and st["relied"] == 1 and st["wide"] == 1
    assert st["flagged"] == 2 and st["alpha"] == 1 and st["depth"] == 1 and st["T"] == 0
    assert maxerr == pytest.approx(0.1)


def test_transmittance_alternatives_move_the_stop_by_2e_8_only():
    # T lands 1e-6 above the stop after the third layer (not flagged) and
    # 5e-9 above it after the fourth (flagged): the alternatives keep the
    # third layer and take or drop the fourth, nothing more
    T2 = (1.0 - 0.9) * (1.0 - 0.9)
    a3 = 1.0 - (1e-4 + 1e-6) / T2
    T3 = T2 * (1.0 - a3)
    a4 = 1.0 - (1e-4 + 5e-9) / T3
    a = [0.9, 0.9, a3, a4, 0.5]
    cols = [C1, C2, C3, [0.7, 0.1, 0.6], [0.5, 0.5, 0.5]]
    rgb, lo, hi, f = _render([2.0, 3.0, 4.0, 5.0, 6.0], a, cols)
    layers = list(zip(a, cols))
    assert f == 4
    assert np.allclose(rgb, _sum(layers[:4]), rtol=0, atol=1e-15)
    elo, ehi = _env(_sum(layers[:4]), _sum(layers[:3]))
    assert np.allclose(lo, elo, rtol=0, atol=1e-15) and np.allclose(hi, ehi, rtol=0, atol=1e-15)
