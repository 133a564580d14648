"""Pins of the oracle's convergence tests (Sec. 2.1, tests (I) and (II)).

R_avg is the mean over the contacts of the impulse magnitude |P|; R^0 is that
mean over the starting impulses (zero, or the warm start).  Test (II)
compares the relative change of R_avg between iteration steps,
|R^j - R^(j-1)| / (R^j + R^(j-1)), with alpha (the paper squares the ratio;
the plain ratio is the default reading).  Test (I) passes when at least 90%
of the contacts change by a squared relative amount below alpha and every
other contact by a squared amount of at most alpha (R^(j-1))^2.

Every number below is derived by hand from these definitions on systems
whose impulses have closed forms, so that a plausible slip in the residual
changes a pinned value: the mean of P_n (or of P_n + |P_t|) in place of |P|,
a sum in place of the mean, R^j alone as the denominator, R^0 taken after
the first sweep or ignoring the warm start, a dropped square, the 90% rule
read as a strict inequality, or the absolute branch of test (I) skipped.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle_cases as cases
from oracle_adapter import params, system

G, DT = cases.G, cases.DT


def _step(wl, **over):
    s = system(wl, **over)
    return s, s.step()


# --- test (II) ---------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_resting_particle_residual_is_one_then_zero(dim):
    """One particle resting on the floor, forces from zero.  Sweep 1 takes P
    from 0 to m g dt: R^0 = 0, R^1 = m g dt, so the ratio is exactly 1.
    Sweep 2 leaves P where it is: the ratio is 0 (to rounding) and test (II)
    stops there."""
    wl = cases.resting_disc(dim=dim)
    mgdt = G * DT / wl.inv_m[0]
    _, st1 = _step(wl, criterion=O.CRIT_NONE, max_sweeps=1)
    assert st1["r_avg_prev"] == 0.0
    assert st1["r_avg"] == pytest.approx(mgdt, rel=1e-15)
    assert st1["residual"] == 1.0
    _, st2 = _step(wl, criterion=O.CRIT_NONE, max_sweeps=2)
    assert st2["r_avg_prev"] == st1["r_avg"]
    assert st2["residual"] <= 1e-15
    for crit in (O.CRIT_GLOBAL_REL, O.CRIT_GLOBAL_SQ):
        _, st = _step(wl, criterion=crit, alpha=1e-6, max_sweeps=100)
        assert st["sweeps"] == 2 and st["converged"]


@pytest.mark.parametrize("dim,azimuth", [(2, 0.0), (3, 0.7)])
def test_residual_averages_the_impulse_magnitude(dim, azimuth):
    """A particle sticking on an incline with rotation frozen: P_n = m g
    cos(theta) dt and |P_t| = m g sin(theta) dt (3D: along a downhill
    direction off both floor axes), so |P| = m g dt.  R_avg is that
    magnitude: the mean of P_n would be 2% lower, P_n + |P_t| 18% higher."""
    theta = math.atan(0.2)
    wl = cases.incline(theta, mu=0.4, dim=dim, azimuth=azimuth)
    mgdt = G * DT / wl.inv_m[0]
    s, st = _step(wl, criterion=O.CRIT_NONE, max_sweeps=1)
    P = s.impulses[0]
    assert P[0] == pytest.approx(mgdt * math.cos(theta), rel=1e-14)
    assert np.linalg.norm(P[1:]) == pytest.approx(mgdt * math.sin(theta), rel=1e-13)
    assert st["r_avg"] == pytest.approx(mgdt, rel=1e-14)
    assert st["residual"] == 1.0


def _stack_ravg(k):
    """Two discs stacked on the floor, forces from zero, the disc-disc
    contact B updated before the floor contact A: B_k = A_(k-1) / 2 and
    A_k = 1 + B_k in units of m g dt, so A_k = 2 - 2^(1-k), B_k = 1 - 2^(1-k)
    and R^k = (A_k + B_k) / 2 = (3 - 2^(2-k)) / 2 for k >= 1, R^0 = 0."""
    return 0.0 if k == 0 else (3.0 - 2.0 ** (2 - k)) / 2.0


def _stack_ratio(k):
    """|R^k - R^(k-1)| / (R^k + R^(k-1)): 1 at k = 1, then
    2^(1-k) / (3 (1 - 2^(1-k))) = 1 / (3 (2^(k-1) - 1))."""
    return 1.0 if k == 1 else 1.0 / (3.0 * (2.0 ** (k - 1) - 1.0))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8])
def test_stack_residual_sequence_closed_form(k):
    wl = cases.stack2()
    unit = G * DT / wl.inv_m[0]
    s, st = _step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=k, warm_start=0)
    assert s.contacts.tolist() == [[0, 1], [0, 4]]
    assert st["sweeps"] == k
    assert st["r_avg"] == pytest.approx(_stack_ravg(k) * unit, rel=1e-13)
    assert st["r_avg_prev"] == pytest.approx(_stack_ravg(k - 1) * unit, rel=1e-13, abs=0)
    assert st["residual"] == pytest.approx(_stack_ratio(k), rel=1e-10)


@pytest.mark.parametrize("crit,alpha", [(O.CRIT_GLOBAL_REL, 1e-6), (O.CRIT_GLOBAL_REL, 1e-3),
                                        (O.CRIT_GLOBAL_SQ, 1e-6), (O.CRIT_GLOBAL_SQ, 1e-10)])
def test_stack_stops_where_the_closed_form_ratio_falls_below_alpha(crit, alpha):
    """The first sweep whose ratio (squared for the paper's form) is below
    alpha: 20 for the plain ratio at 1e-6, 10 at 1e-3 and for the squared
    ratio at 1e-6, 17 for the squared ratio at 1e-10."""
    expect = {(O.CRIT_GLOBAL_REL, 1e-6): 20, (O.CRIT_GLOBAL_REL, 1e-3): 10,
              (O.CRIT_GLOBAL_SQ, 1e-6): 10, (O.CRIT_GLOBAL_SQ, 1e-10): 17}[(crit, alpha)]
    power = 2 if crit == O.CRIT_GLOBAL_SQ else 1
    k = 1
    while not _stack_ratio(k) ** power < alpha:
        k += 1
    assert k == expect
    wl = cases.stack2()
    _, st = _step(wl, order=O.ORDER_COLOUR, criterion=crit, alpha=alpha, max_sweeps=1000, warm_start=0)
    assert st["converged"] and st["sweeps"] == expect
    assert st["residual"] == pytest.approx(_stack_ratio(expect) ** power, rel=1e-8)


def test_warm_started_residual_starts_from_the_carried_forces():
    """Stepped twice, the resting particle's second solve starts from the
    carried impulse m g dt: R^0 = m g dt, the first sweep keeps it, the ratio
    is 0 and test (II) stops after one sweep (R^0 = 0 would give 1 and a
    second sweep)."""
    wl = cases.resting_disc()
    mgdt = G * DT / wl.inv_m[0]
    s = system(wl, criterion=O.CRIT_GLOBAL_REL, alpha=1e-6, max_sweeps=100)
    st1 = s.step()
    st2 = s.step()
    assert st1["sweeps"] == 2
    assert st2["sweeps"] == 1 and st2["converged"]
    assert st2["r_avg_prev"] == pytest.approx(mgdt, rel=1e-15)
    assert st2["residual"] <= 1e-15


# --- test (I) ------------------------------------------------------------------

def _row_solve(radii, warm, alpha=1e-6, max_sweeps=1):
    """A row of discs resting on the floor, each with its floor contact only;
    `warm[i]` gives disc i its exact weight impulse m g dt to start from,
    else it starts from zero.  One local-test solve from there."""
    wl = cases.floor_row(radii)
    p = params(wl, criterion=O.CRIT_LOCAL, alpha=alpha, max_sweeps=max_sweeps, order=O.ORDER_RANDOM)
    wp = np.asarray(wl.wall_pos, dtype=np.float64)
    pairs = O.detect_brute(p, wl.x, wl.r, wp)
    assert pairs.tolist() == [[i, wl.n + 2] for i in range(wl.n)]
    normal, gap, mn, mt = O.contact_geometry(p, wl.x, wl.r, wl.inv_m, wl.inv_I, wp, pairs)
    P0 = np.zeros((wl.n, 2))
    P0[:, 0] = np.where(warm, G * DT / wl.inv_m, 0.0)
    vfree = wl.v.copy()
    vfree[:, 1] -= G * DT
    return O.solve(p, vfree, wl.w, wl.r, wl.inv_m, wl.inv_I, pairs, normal, gap, mn, mt, P0=P0)


def test_local_test_passes_at_exactly_ninety_percent():
    """Nine discs start from their weight (no change: relative test passed);
    a tenth, 2500 times lighter (r = 0.02), starts from zero and changes by
    its whole weight: relative test failed, but its squared change, (m g
    dt)^2, is below alpha (R^0)^2 with R^0 = 0.9 M g dt.  9 of 10 is 90%:
    converged after one sweep, with 1/10 of the contacts outside the
    relative test."""
    P, v, w, st = _row_solve([1.0] * 9 + [0.02], [True] * 9 + [False])
    assert st["converged"] and st["sweeps"] == 1
    assert st["residual"] == 0.1


def test_local_test_fails_below_ninety_percent():
    """Eight of ten discs unchanged (80%): not converged after one sweep
    (residual 0.2); the second sweep changes nothing and passes."""
    radii, warm = [1.0] * 8 + [0.02] * 2, [True] * 8 + [False] * 2
    P, v, w, st = _row_solve(radii, warm)
    assert not st["converged"] and st["sweeps"] == 1
    assert st["residual"] == 0.2
    P, v, w, st = _row_solve(radii, warm, max_sweeps=10)
    assert st["converged"] and st["sweeps"] == 2


@pytest.mark.parametrize("radius", [1.0, 0.1])
def test_local_test_needs_the_rest_below_the_absolute_bound(radius):
    """19 of 20 contacts unchanged (95%), but the twentieth changes by (m g
    dt)^2 above alpha (R^0)^2 (a disc of radius 1 or 0.1, mass ratio 1 or
    1/100 against sqrt(alpha) = 1/1000): not converged after one sweep."""
    P, v, w, st = _row_solve([1.0] * 19 + [radius], [True] * 19 + [False])
    assert not st["converged"] and st["sweeps"] == 1
    assert st["residual"] == pytest.approx(0.05, rel=1e-15)


def test_nan_impulses_never_pass_the_global_tests():
    """A NaN starting impulse spreads through the velocities: every R_avg is
    NaN and must not pass tests (II), which count only 0/0 (both averages
    zero) as converged; the solve runs to the cap with a NaN residual."""
    for crit in (O.CRIT_GLOBAL_REL, O.CRIT_GLOBAL_SQ):
        wl = cases.floor_row([1.0] * 4)
        p = params(wl, criterion=crit, alpha=1e-6, max_sweeps=50, order=O.ORDER_RANDOM)
        wp = np.asarray(wl.wall_pos, dtype=np.float64)
        pairs = O.detect_brute(p, wl.x, wl.r, wp)
        normal, gap, mn, mt = O.contact_geometry(p, wl.x, wl.r, wl.inv_m, wl.inv_I, wp, pairs)
        P0 = np.zeros((wl.n, 2))
        P0[1, 0] = np.nan
        vfree = wl.v.copy()
        vfree[:, 1] -= G * DT
        P, v, w, st = O.solve(p, vfree, wl.w, wl.r, wl.inv_m, wl.inv_I, pairs, normal, gap, mn, mt, P0=P0)
        assert not st["converged"] and st["sweeps"] == 50
        assert math.isnan(st["residual"])
