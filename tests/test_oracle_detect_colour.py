"""Pins of the oracle's contact detection (Sec. 3.2) and colouring.

Detection: a hand-derived golden set, and the cell method equal to brute
force over all pairs on seeded random inputs.  Colouring: validity (no two
contacts of one colour share a particle), the greedy bound K <= Delta + 1 of
the contact graph, and a star whose contacts all need distinct colours.
"""

import numpy as np
import pytest

import oracle as O
from oracle_adapter import params
from golden_cases import hand_geometry, load_hand_case
from paper_1104_3516_gb300 import workloads as W


def hand_params(name="detect_hand_2d.txt"):
    disc, expect, prm = load_hand_case(name)
    dim, lo, hi, per3, mask, wp = hand_geometry(prm)
    p = O.make_params(dim=dim, delta=prm["delta"][0], box_lo=lo, box_hi=hi, periodic=per3, wall_mask=mask)
    return p, disc, expect, dim, wp


@pytest.mark.parametrize("name", ["detect_hand_2d.txt", "detect_hand_3d.txt"])
@pytest.mark.parametrize("method", ["brute", "cells"])
def test_hand_derived_contact_set(method, name):
    p, disc, expect, dim, wp = hand_params(name)
    f = O.detect_brute if method == "brute" else O.detect_cells
    pairs = f(p, disc[:, :dim], disc[:, dim], wp)
    assert [tuple(map(int, q)) for q in pairs] == expect


def random_case(dim, n, periodic, walls, seed, phi=None):
    phi = phi if phi is not None else (0.4 if dim == 2 else 0.2)
    r = W.uniform(seed, n, 0.8, 1.2)
    vol = float(np.sum(np.pi * r ** 2)) if dim == 2 else float(np.sum(4.0 / 3.0 * np.pi * r ** 3))
    L = (vol / phi) ** (1.0 / dim)
    lo = (0.0,) * dim
    hi = (L,) * dim
    x = W.rsa(dim, n, r, lo, hi, periodic, seed, min_gap=0.0)
    p = O.make_params(dim=dim, delta=0.24, box_lo=lo + (0.0,) * (3 - dim), box_hi=hi + (1.0,) * (3 - dim),
                      periodic=tuple(periodic) + (0,) * (3 - dim), wall_mask=walls)
    wp = np.zeros(6)
    for k in range(2 * dim):
        wp[k] = 0.0 if k % 2 == 0 else L
    return p, x, r, wp


@pytest.mark.parametrize("dim,periodic,walls", [
    (2, (0, 0), 0b1111), (2, (1, 0), 0b1100), (2, (1, 1), 0), (3, (0, 0, 0), 0b111111), (3, (1, 1, 0), 0b110000),
])
def test_cell_method_equals_brute_force(dim, periodic, walls):
    for seed in (1, 2):
        n = 250 if dim == 2 else 500
        p, x, r, wp = random_case(dim, n, periodic, walls, seed)
        a = O.detect_brute(p, x, r, wp)
        b = O.detect_cells(p, x, r, wp)
        assert len(a) > n // 4
        assert np.array_equal(a, b)
        # sorted by key, each pair a < b
        keys = a[:, 0].astype(np.int64) * (1 << 32) + a[:, 1]
        assert np.all(np.diff(keys) > 0) and np.all(a[:, 0] < a[:, 1])


def test_geometry_normal_gap_and_mass_matrix():
    """n is the unit vector from a to b, g the surface gap; the mass matrix of
    Eq. 5 for two discs is diag(1/(1/m_a+1/m_b), 1/(1/m_a+1/m_b+r_a^2/I_a+r_b^2/I_b))."""
    p = O.make_params(dim=2, delta=0.5, box_lo=(0, 0, 0), box_hi=(10, 10, 1), wall_mask=0b0100)
    x = np.array([[2.0, 3.0], [4.4, 3.0 + 0.7]])
    r = np.array([1.0, 1.5])
    inv_m, inv_I = W.masses(2, r)
    pairs = np.array([[0, 1]], dtype=np.int32)
    normal, gap, mn, mt = O.contact_geometry(p, x, r, inv_m, inv_I, np.zeros(6), pairs)
    d = np.hypot(2.4, 0.7)
    assert np.allclose(normal[0], [2.4 / d, 0.7 / d, 0.0], rtol=0, atol=1e-16)
    assert gap[0] == pytest.approx(d - 2.5, rel=1e-15)
    ma, mb = 1 / inv_m[0], 1 / inv_m[1]
    Ia, Ib = 1 / inv_I[0], 1 / inv_I[1]
    assert mn[0] == pytest.approx(ma * mb / (ma + mb), rel=1e-14)
    # discs: r^2 / I = 2 / m, so w_t = 3 (1/m_a + 1/m_b)
    assert mt[0] == pytest.approx(1.0 / (1 / ma + 1 / mb + 1.0 * 1.0 / Ia + 1.5 * 1.5 / Ib), rel=1e-14)
    assert mt[0] == pytest.approx(mn[0] / 3.0, rel=1e-14)
    # floor contact: normal from the particle into the wall, gap above the floor
    pairs = np.array([[0, 2 + 2]], dtype=np.int32)
    x2 = np.array([[2.0, 1.1], [9.0, 9.0]])
    normal, gap, mn, mt = O.contact_geometry(p, x2, r, inv_m, inv_I, np.zeros(6), pairs)
    assert np.array_equal(normal[0], [0.0, -1.0, 0.0])
    assert gap[0] == pytest.approx(0.1, rel=1e-14)
    assert mn[0] == pytest.approx(ma, rel=1e-14)


def test_geometry_3d_spheres_periodic_image_and_ceiling():
    """3D: the normal follows the periodic minimum image (offset (2, 2, 1),
    length 3, exact), the gap is |d| - r_a - r_b; for spheres r^2 / I =
    5 / (2 m), so the tangential mass of Eq. 5 is m_t = 2 m_n / 7, for a pair
    and against a wall (infinite mass); the ceiling's normal points from the
    particle into the wall (+z) and its gap is z_wall - z - r."""
    p = O.make_params(dim=3, delta=0.5, box_lo=(0, 0, 0), box_hi=(10, 10, 20), periodic=(1, 0, 0),
                      wall_mask=0b110000)
    r = np.array([1.25, 1.0])
    inv_m, inv_I = W.masses(3, r)
    wp = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 20.0])
    x = np.array([[9.5, 3.0, 5.0], [1.5, 5.0, 6.0]])          # min image dx = 1.5 - 9.5 + 10 = 2
    normal, gap, mn, mt = O.contact_geometry(p, x, r, inv_m, inv_I, wp, np.array([[0, 1]], dtype=np.int32))
    assert np.allclose(normal[0], [2.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0], rtol=0, atol=1e-16)
    assert gap[0] == 3.0 - 2.25
    ma, mb = 1 / inv_m[0], 1 / inv_m[1]
    assert mn[0] == pytest.approx(ma * mb / (ma + mb), rel=1e-14)
    assert mt[0] == pytest.approx(2.0 * mn[0] / 7.0, rel=1e-14)
    x2 = np.array([[5.0, 5.0, 18.5], [2.0, 2.0, 5.0]])
    normal, gap, mn, mt = O.contact_geometry(p, x2, r, inv_m, inv_I, wp, np.array([[0, 2 + 5]], dtype=np.int32))
    assert np.array_equal(normal[0], [0.0, 0.0, 1.0])
    assert gap[0] == 20.0 - 18.5 - 1.25
    assert mn[0] == pytest.approx(ma, rel=1e-14)
    assert mt[0] == pytest.approx(2.0 * ma / 7.0, rel=1e-14)


def _conflicts(n, pairs, colour):
    bad = 0
    for k in np.unique(colour):
        sel = pairs[colour == k]
        parts = sel.ravel()
        parts = parts[parts < n]
        bad += len(parts) - len(np.unique(parts))
    return bad


@pytest.mark.parametrize("dim", [2, 3])
def test_greedy_colouring_is_valid_and_bounded(dim):
    p, x, r, wp = random_case(dim, 400, (0,) * dim, (1 << (2 * dim)) - 1, 5, phi=0.45 if dim == 2 else 0.25)
    pairs = O.detect_cells(p, x, r, wp)
    n = r.shape[0]
    colour, K = O.colour_greedy(n, pairs, seed=99)
    assert _conflicts(n, pairs, colour) == 0
    assert K == colour.max() + 1 and colour.min() >= 0
    # line-graph degree bound: a contact meets at most deg(a)-1 + deg(b)-1 others
    deg = np.bincount(pairs.ravel(), minlength=n + 6)[:n]
    dyn = lambda q: deg[q] - 1 if q < n else 0
    delta = max(dyn(a) + dyn(b) for a, b in pairs)
    assert K <= delta + 1
    # different seeds give different (still valid) colourings
    colour2, _ = O.colour_greedy(n, pairs, seed=100)
    assert _conflicts(n, pairs, colour2) == 0 and not np.array_equal(colour, colour2)


def test_star_needs_all_colours_and_walls_do_not_conflict():
    # particle 0 touches particles 1..5: five contacts sharing particle 0
    n = 6
    pairs = np.array([[0, k] for k in range(1, 6)], dtype=np.int32)
    colour, K = O.colour_greedy(n, pairs, seed=3)
    assert K == 5 and sorted(colour.tolist()) == [0, 1, 2, 3, 4]
    # five particles each touching the same wall: no conflict through the wall
    pairs = np.array([[k, n + 2] for k in range(5)], dtype=np.int32)
    colour, K = O.colour_greedy(n, pairs, seed=3)
    assert K == 1


def test_repair_moves_the_top_colour_along_a_kempe_chain():
    """A path of four contacts p0-p1-p2-p3-p4 coloured 0, 1, 2, 0 (greedy in
    the order e1, e4, e2, e3).  Contact e3 = (p2, p3) has colour 2 while no
    particle has more than two contacts.  Colour 0 is free at p2, colour 1 at
    p3; the (0, 1) path from p3 is e4 alone, swapping it gives e4 colour 1
    and frees 0 at p3, so e3 takes 0: colours 0, 1, 0, 1."""
    n = 5
    pairs = np.array([[0, 1], [1, 2], [2, 3], [3, 4]], dtype=np.int32)
    col, K = O.colour_repair(n, pairs, np.array([0, 1, 2, 0]))
    assert K == 2 and col.tolist() == [0, 1, 0, 1]


def test_repair_keeps_an_odd_cycle_at_three_colours():
    """A triangle of particles needs three colours although each has two
    contacts: the (1, 0) path from the third particle returns to the first,
    so the repair fails and leaves the colouring alone."""
    n = 3
    pairs = np.array([[0, 1], [0, 2], [1, 2]], dtype=np.int32)
    col, K = O.colour_repair(n, pairs, np.array([0, 2, 1]))
    assert K == 3 and col.tolist() == [0, 2, 1]


def test_repair_takes_a_colour_free_at_both_ends_and_skips_large_classes():
    """A contact whose ends both lack a lower colour takes the smallest one
    directly; a top class larger than max(1, min(1024, nc / 256)) is left as
    it is; a three-contact path coloured 0, 2, 1 is repaired through the
    (1, 0) chain of its third contact."""
    n = 4
    pairs = np.array([[0, 1], [2, 3]], dtype=np.int32)
    col, K = O.colour_repair(n, pairs, np.array([0, 1]))
    assert K == 1 and col.tolist() == [0, 0]
    m = 300
    pairs = np.array([[2 * i, 2 * i + 1] for i in range(m)], dtype=np.int32)
    start = np.array([i % 2 for i in range(m)])
    col, K = O.colour_repair(2 * m, pairs, start)
    assert K == 2 and np.array_equal(col, start)  # 150 contacts of colour 1 > max(1, 300 // 256)
    pairs = np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32)
    col, K = O.colour_repair(n, pairs, np.array([0, 2, 1]))
    # (1, 2) has colour 2; colour 0 is taken at p1, free at p2; colour 1 is free at p1, taken at p2
    # -> path from p2 with colour 1: (2, 3); swap -> (2, 3) gets 0; (1, 2) gets 1
    assert K == 2 and col.tolist() == [0, 1, 0]


def test_repaired_pile_uses_as_many_colours_as_the_busiest_particle():
    """On the dense deposit the greedy colouring needs one colour more than
    the largest particle degree; the repair removes it and stays proper."""
    wl = W.dense_biaxial_discs(n=5000)
    p = params(wl)
    pairs = O.detect_cells(p, wl.x, wl.r, np.asarray(wl.wall_pos, dtype=np.float64))
    colour, K = O.colour_greedy(wl.n, pairs, wl.seed)
    deg = np.bincount(pairs[:, 0], minlength=wl.n) + np.bincount(pairs[:, 1][pairs[:, 1] < wl.n], minlength=wl.n)
    assert _conflicts(wl.n, pairs, colour) == 0
    assert K == int(deg.max())
