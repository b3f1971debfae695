"""Pins of the oracle's view-index map (Sec. 3.1, Eqs. (1)-(3); Alg. 1).

Each check is fixed by the equations themselves, not by re-typing them:
hand-worked values, exact periodicity over the lens pitch, the row-shift
identity of a slant with 3 tan(alpha) = 1/2, the shift produced by K_offset,
and the balance of views within a lens period."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "viewmap_hand.txt")


def _golden_panels():
    panels, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("panel"):
            w, h, nv, lx, tan, k = line.split()[1:]
            cur = {"display": W.Display(int(w), int(h), int(nv), float(lx), float(tan), float(k)),
                   "rows": {}}
            panels.append(cur)
        else:
            head, vals = line.split(":")
            cur["rows"][int(head.split()[1])] = [int(v) for v in vals.split()]
    return panels


@pytest.mark.parametrize("panel", _golden_panels(), ids=["A", "B"])
def test_hand_worked_values(panel):
    V = oracle.view_map(panel["display"])
    for x, vals in panel["rows"].items():
        assert V[x].tolist() == vals


def test_q32_constants_exact_for_dyadic_params():
    t3, lq, kq = oracle.quantise(W.Display(4, 4, 7, 21 / 4, 1 / 6, 1.25))
    assert t3 == 2 ** 31          # 3 tan = 1/2 exactly
    assert lq == 21 * 2 ** 30     # 5.25 * 2^32
    assert kq == 5 * 2 ** 30      # 1.25 * 2^32


@pytest.mark.parametrize("tan,k", [(1 / 6, 0.0), (0.18, 0.0), (-0.13, 2.5), (0.2, 23.6677)])
def test_periodic_over_lens_pitch(tan, k):
    # L_x = 21/4: 21 subpixel columns span exactly 4 lens units, so
    # d_offset(s + 21) = d_offset(s) + 4 L_x and the view repeats.
    d = W.Display(60, 17, 45, 21 / 4, tan, k)
    V = oracle.view_map(d)
    assert np.array_equal(V[:, 21:], V[:, :-21])


def test_row_shift_identity_half_slant():
    # 3 tan(alpha) = 1/2: two rows down add exactly one subpixel width.
    for d in (W.WORKLOADS["tiny"].display, W.Display(50, 31, 48, 6.2221, 1 / 6, 4.2077)):
        V = oracle.view_map(d)
        assert np.array_equal(V[2:, :-1], V[:-2, 1:])


def test_offset_shifts_map_by_one_subpixel():
    base = W.Display(40, 9, 45, 5.3, 0.18, 0.0)
    V0 = oracle.view_map(base)
    V1 = oracle.view_map(base.replace(offset_k=1.0))
    assert np.array_equal(V1[:, 1:], V0[:, :-1])


def test_zero_slant_rows_identical():
    V = oracle.view_map(W.Display(30, 8, 45, 5.3, 0.0, 0.7))
    assert (V == V[0]).all()


def test_views_balanced_over_a_period():
    # L_x = 21/4, N_v = 7: the 21 x_offsets of one period are the multiples of
    # 1/4 in [0, 5.25), each view bin (width 3/4) holds exactly three of them.
    V = oracle.view_map(W.Display(70, 5, 7, 21 / 4, 0.1, 0.3))
    for x in range(5):
        for s0 in range(0, 210 - 21, 21):
            counts = np.bincount(V[x, s0:s0 + 21], minlength=7)
            assert (counts == 3).all()


@pytest.mark.parametrize("name", list(W.PAPER_PANELS))
def test_views_balanced_over_a_real_panel(name):
    # With an irrational-looking pitch and slant the x_offsets of a whole
    # panel spread evenly over [0, L_x), so each view covers 1/N_v of it.
    d = W.PAPER_PANELS[name]
    V = oracle.view_map(d)
    counts = np.bincount(V.ravel(), minlength=d.num_views)
    mean = V.size / d.num_views
    assert np.abs(counts / mean - 1.0).max() < 1e-3


@pytest.mark.parametrize("name", list(W.PAPER_PANELS) + list(W.WORKLOADS))
def test_view_range(name):
    d = W.PAPER_PANELS.get(name) or W.WORKLOADS[name].display
    V = oracle.view_map(d)
    assert V.shape == (d.height, 3 * d.width)
    assert int(V.max()) < d.num_views
    # every view index is used somewhere on a full panel
    assert len(np.unique(V)) == d.num_views or name == "8k"
