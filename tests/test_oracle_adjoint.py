"""Pins of the oracle's frozen-state step map and its complex-step
derivatives (oracle/adjoint.py): it must reproduce the oracle's own
iteration, agree with central finite differences of that iteration, and hit
the closed forms of single contacts (rolling, sliding, inelastic collision)
and the conservation of momentum."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from oracle_adapter import system
from oracle_cases import DT, G, colliding_gas, head_on, leaning_column, periodic_gas, resting_disc

TIGHT = dict(criterion=O.CRIT_GLOBAL_REL, alpha=1e-15, max_sweeps=100000, order=O.ORDER_COLOUR)


def rollout(wl, steps, x=None, v=None, w=None, mu=None):
    """Real oracle rollout from a (possibly perturbed) start; returns the
    final system and the per-step frozen decisions."""
    import copy
    wl2 = copy.copy(wl)
    if x is not None:
        wl2.x = x
    if v is not None:
        wl2.v = v
    if w is not None:
        wl2.w = w
    if mu is not None:
        wl2.mu = mu
    s = system(wl2, **TIGHT)
    recs = A.record_rollout(s, steps)
    return s, recs


def directions(wl, k, seed, with_mu=True):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        out.append((rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape),
                    rng.standard_normal(wl.w.shape), float(rng.standard_normal()) if with_mu else 0.0))
    return out


def same_states(ra, rb):
    return len(ra) == len(rb) and all(
        a.pairs.shape == b.pairs.shape and np.array_equal(a.pairs, b.pairs) and np.array_equal(a.state, b.state)
        and np.array_equal(a.sign[a.state == A.SLIDE], b.sign[b.state == A.SLIDE]) for a, b in zip(ra, rb))


@pytest.mark.parametrize("mk", [colliding_gas, periodic_gas])
def test_frozen_map_reproduces_the_iteration(mk):
    wl = mk(n=100, phi=0.62, vsig=3.0, dt=0.02)
    s, recs = rollout(wl, 6)
    counts = np.sum([np.bincount(r.state, minlength=3) for r in recs], axis=0)
    assert counts[A.STICK] > 10 and counts[A.SLIDE] > 10     # all three states occur
    cs = A.consts_of(s)
    x, v, w = A.rollout_map(cs, recs, wl.x, wl.v, wl.w, wl.mu)
    assert np.abs(x - s.x.reshape(-1, 2)).max() < 1e-11
    vs = max(np.abs(s.v).max(), 1.0)
    assert np.abs(v - s.v.reshape(-1, 2)).max() < 1e-11 * vs
    assert np.abs(w - s.w).max() < 1e-11 * vs


def check_fd(wl, steps, dirs, h=1e-6, tol=1e-5, need=6):
    """Central differences of the oracle's Gauss-Seidel rollout against the
    complex step of the frozen-state map along `dirs`, skipping directions
    whose +-h runs change a contact state (a kink of the map)."""
    s, recs = rollout(wl, steps)
    cs = A.consts_of(s)
    rng = np.random.default_rng(5)
    weights = (rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape), rng.standard_normal(wl.w.shape))

    def loss(sy):
        return (np.sum(weights[0] * sy.x.reshape(-1, 2)) + np.sum(weights[1] * sy.v.reshape(-1, 2))
                + np.sum(weights[2] * sy.w))

    cstep = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, weights, dirs)
    clean = 0
    for (ex, ev, ew, em), d in zip(dirs, cstep):
        sp, rp = rollout(wl, steps, wl.x + h * ex, wl.v + h * ev, wl.w + h * ew, wl.mu + h * em)
        sm, rm = rollout(wl, steps, wl.x - h * ex, wl.v - h * ev, wl.w - h * ew, wl.mu - h * em)
        if not (same_states(recs, rp) and same_states(recs, rm)):
            continue
        clean += 1
        fd = (loss(sp) - loss(sm)) / (2 * h)
        assert abs(fd - d) <= tol * max(abs(d), 1.0), (fd, d)
    assert clean >= need
    return recs


def test_complex_step_matches_finite_differences_one_step_of_collisions():
    """One step of a fast gas: fresh collisions, sticking and sliding."""
    wl = colliding_gas(n=300, phi=0.62, vsig=3.0, dt=0.05)
    recs = check_fd(wl, 1, directions(wl, 8, seed=6))
    counts = np.bincount(recs[0].state, minlength=3)
    assert counts[A.STICK] >= 5 and counts[A.SLIDE] >= 5


def test_complex_step_matches_finite_differences_over_steps():
    """Four steps of a leaning column: every contact carries weight in every
    step, some stick and some slide; the position part of each direction is
    scaled by dt so that it moves the gaps by less than the step moves them."""
    wl = leaning_column(mu=0.18)
    dirs = [(1e-3 * ex, ev, ew, em) for (ex, ev, ew, em) in directions(wl, 8, seed=6)]
    recs = check_fd(wl, 4, dirs, need=8)
    counts = np.sum([np.bincount(r.state, minlength=3) for r in recs], axis=0)
    assert counts[A.STICK] >= 8 and counts[A.SLIDE] >= 8


def test_rolling_disc_closed_form():
    """A disc (I = m r^2 / 2) on the floor with v_x and omega that sticks:
    v_x' + r omega' = 0 with P_t = m (v_x + r omega) / 3, so
    dv_x'/dv_x = 2/3, dv_x'/domega = -r/3, domega'/dv_x = -2/(3 r),
    domega'/domega = 1/3; the normal row closes the gap: dv_y'/dy = -1/dt."""
    r = 0.9
    wl = resting_disc(radius=r, mu=1.0)
    wl.v = np.array([[1e-3, 0.0]])
    wl.w = np.array([2e-4])
    s, recs = rollout(wl, 1)
    assert recs[0].state.tolist() == [A.STICK]
    cs = A.consts_of(s)
    z2, z1 = np.zeros((1, 2)), np.zeros(1)

    def e(a, i):
        m = np.zeros_like(a, dtype=np.float64)
        m[i] = 1.0
        return m

    # derivatives of v_x'
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, e(z2, (0, 0)), z1),
                                  [(z2, e(z2, (0, 0)), z1, 0.0), (z2, z2, e(z1, 0), 0.0)])
    assert d == pytest.approx([2.0 / 3.0, -r / 3.0], rel=1e-12)
    # derivatives of omega'
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, z2, e(z1, 0)),
                                  [(z2, e(z2, (0, 0)), z1, 0.0), (z2, z2, e(z1, 0), 0.0)])
    assert d == pytest.approx([-2.0 / (3.0 * r), 1.0 / 3.0], rel=1e-12)
    # v_y' = -gap / dt
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, e(z2, (0, 1)), z1),
                                  [(e(z2, (0, 1)), z2, z1, 0.0)])
    assert d[0] == pytest.approx(-1.0 / DT, rel=1e-12)


@pytest.mark.parametrize("rotations", [0, 1])
def test_sliding_disc_friction_derivative(rotations):
    """A fast disc sliding on the floor: P_t = mu m g dt against the motion,
    so dv_x'/dmu = -g dt, dv_x'/dv_x = 1 and (rolling allowed)
    domega'/dmu = -2 g dt / r; nothing depends on mu when rotations are
    frozen except v_x'."""
    r = 1.1
    wl = resting_disc(radius=r, mu=0.3)
    wl.v = np.array([[1.0, 0.0]])
    if not rotations:
        wl.inv_I = np.zeros(1)
    s, recs = rollout(wl, 1)
    assert recs[0].state.tolist() == [A.SLIDE]
    cs = A.consts_of(s)
    z2, z1 = np.zeros((1, 2)), np.zeros(1)
    ex = np.array([[1.0, 0.0]])
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, ex, z1),
                                  [(z2, z2, z1, 1.0), (z2, ex, z1, 0.0)])
    assert d == pytest.approx([-G * DT, 1.0], rel=1e-12)
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, z2, np.ones(1)), [(z2, z2, z1, 1.0)])
    expect = -2.0 * G * DT / r if rotations else 0.0
    assert d[0] == pytest.approx(expect, rel=1e-12, abs=1e-300)


def test_inelastic_collision_closed_form():
    """Head-on discs of unequal mass: v1' = (m1 v1 + m2 v2 + m2 g / dt) / M
    (momentum, and the gap closes), so dv1'/dv1 = m1/M, dv1'/dv2 = m2/M,
    dv1'/dx2 = -dv1'/dx1 = m2 / (M dt), and dx1'/dv1 = dt m1 / M."""
    r1, r2 = 1.0, 1.3
    wl = head_on(1.0, -1.0, r1=r1, r2=r2)
    s, recs = rollout(wl, 1)
    assert recs[0].state.tolist() == [A.STICK]
    m1, m2 = 1.0 / wl.inv_m[0], 1.0 / wl.inv_m[1]
    M = m1 + m2
    cs = A.consts_of(s)
    z2, z1 = np.zeros((2, 2)), np.zeros(2)

    def unit(i, k):
        e = np.zeros((2, 2))
        e[i, k] = 1.0
        return e

    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, unit(0, 0), z1),
                                  [(z2, unit(0, 0), z1, 0.0), (z2, unit(1, 0), z1, 0.0), (unit(1, 0), z2, z1, 0.0),
                                   (unit(0, 0), z2, z1, 0.0), (z2, z2, z1, 1.0)])
    assert d == pytest.approx([m1 / M, m2 / M, m2 / (M * DT), -m2 / (M * DT), 0.0], rel=1e-12, abs=1e-12)
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (unit(0, 0), z2, z1), [(z2, unit(0, 0), z1, 0.0)])
    assert d[0] == pytest.approx(DT * m1 / M, rel=1e-12)


def test_momentum_is_conserved_to_first_order():
    """No walls, no gravity: sum m v_x after any number of steps has gradient
    m_j with respect to v0_j,x and zero with respect to everything else."""
    wl = periodic_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    s, recs = rollout(wl, 6)
    cs = A.consts_of(s)
    m = 1.0 / wl.inv_m
    cv = np.stack([m, np.zeros_like(m)], axis=1)
    dirs = directions(wl, 6, seed=9)
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (np.zeros_like(wl.x), cv, np.zeros_like(wl.w)),
                                  dirs)
    expect = [float(np.sum(m * ev[:, 0])) for (_, ev, _, _) in dirs]
    assert d == pytest.approx(expect, rel=1e-11)


def test_classify_reads_the_branches():
    P = np.array([[0.0, 0.0], [2.0, 0.3 * 2.0], [2.0, -(0.3 * 2.0)], [2.0, 0.1], [3.0, 0.0]])
    st, sg = A.classify(P, 0.3)
    assert st.tolist() == [A.OPEN, A.SLIDE, A.SLIDE, A.STICK, A.STICK]
    assert sg[1] == 1.0 and sg[2] == -1.0
    assert math.isfinite(A.jacobian_condition(A.Consts(
        n=1, r=np.ones(1), inv_m=np.ones(1), inv_I=np.ones(1), dt=DT, gravity=np.zeros(2), f_ext=None,
        lo=np.zeros(2), hi=np.ones(2), periodic=np.zeros(2, dtype=int), wall_vel=np.zeros((6, 3))),
        A.StepRecord(pairs=np.array([[0, 3]]), state=np.array([A.STICK]), sign=np.ones(1), shift=np.zeros((1, 2)),
                     wall_pos=np.zeros(6), P=np.zeros((1, 2))), np.array([[0.5, 1.0]]), 0.3))


def test_floor_force_closed_form():
    """A disc pressed on the floor (gap 0, moving down at v_y): it sticks,
    v_y' = -gap/dt, so the floor force F = P_n / dt = m (g - v_y / dt - gap /
    dt^2) and dF/dv_y = -m/dt, dF/dy = -m/dt^2, dF/dmu = 0."""
    wl = resting_disc(radius=1.0, mu=0.3)
    wl.v = np.array([[0.0, -0.01]])
    s, recs = rollout(wl, 1)
    assert recs[0].state.tolist() == [A.STICK]
    m = 1.0 / wl.inv_m[0]
    cs = A.consts_of(s)
    z2, z1 = np.zeros((1, 2)), np.zeros(1)
    cF = np.zeros(6)
    cF[2] = 1.0
    ey = np.array([[0.0, 1.0]])
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, (z2, z2, z1),
                                  [(z2, ey, z1, 0.0), (ey, z2, z1, 0.0), (z2, z2, z1, 1.0)], wall_weights=cF)
    assert d == pytest.approx([-m / DT, -m / DT ** 2, 0.0], rel=1e-12, abs=1e-9)
    x, v, w, F = A.rollout_map(cs, recs, wl.x, wl.v, wl.w, wl.mu, with_forces=True)
    assert F[2] == pytest.approx(wall_force(s, 2), rel=1e-12)


def test_wall_force_derivatives_match_finite_differences():
    """The complex step of a loss on the last step's wall forces against
    central differences of the oracle's iteration (one step of the gas)."""
    wl = colliding_gas(n=300, phi=0.62, vsig=3.0, dt=0.05)
    s, recs = rollout(wl, 1)
    cs = A.consts_of(s)
    cF = np.array([0.3, -0.7, 1.0, 0.0, 0.0, 0.0])
    zero = (np.zeros_like(wl.x), np.zeros_like(wl.v), np.zeros_like(wl.w))
    dirs = directions(wl, 6, seed=21)
    d = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, zero, dirs, wall_weights=cF)
    h, clean = 1e-6, 0
    for (ex, ev, ew, em), dd in zip(dirs, d):
        sp, rp = rollout(wl, 1, wl.x + h * ex, wl.v + h * ev, wl.w + h * ew, wl.mu + h * em)
        sm, rm = rollout(wl, 1, wl.x - h * ex, wl.v - h * ev, wl.w - h * ew, wl.mu - h * em)
        if not (same_states(recs, rp) and same_states(recs, rm)):
            continue
        clean += 1
        Fp = np.array([wall_force(sp, k) for k in range(6)])
        Fm = np.array([wall_force(sm, k) for k in range(6)])
        fd = float(np.sum(cF * (Fp - Fm)) / (2 * h))
        assert abs(fd - dd) <= 1e-5 * max(abs(dd), 1.0), (fd, dd)
    assert clean >= 4


def wall_force(sys, k):
    """Force on wall k in the oracle's last step, from its own impulses."""
    pairs, P = sys.contacts, sys.impulses
    return float(sum(P[c, 0] for c in range(len(pairs)) if pairs[c, 1] == sys.n + k) / sys.p.dt)


def test_sliding_pyramids_mu_derivative_matches_finite_differences():
    """Pyramids of three discs on a floor sliding sideways under them, 200
    steps: the complex-step derivative of the last step's floor force with
    respect to mu against central differences of the oracle's iteration.  The
    floor impulses carry rounding noise of ~1e-10 (gap / dt terms), so the
    step is 1e-4 (noise / h and truncation both near 1e-6 relative); the
    derivative is far from zero (friction drives the pyramids)."""
    from paper_1104_3516_gb300 import workloads as W
    wl = W.sliding_pyramids(n_pyramids=3)
    s, recs = rollout(wl, 200)
    cs = A.consts_of(s)
    zero = (np.zeros_like(wl.x), np.zeros_like(wl.v), np.zeros_like(wl.w))
    cF = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 0.0])
    e_mu = (np.zeros_like(wl.x), np.zeros_like(wl.v), np.zeros_like(wl.w), 1.0)
    d = float(A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, zero, [e_mu], wall_weights=cF)[0])
    h = 1e-4
    sp, rp = rollout(wl, 200, mu=wl.mu + h)
    sm, rm = rollout(wl, 200, mu=wl.mu - h)
    assert same_states(recs, rp) and same_states(recs, rm)
    fd = (wall_force(sp, 2) - wall_force(sm, 2)) / (2 * h)
    assert abs(d) > 1.0
    assert abs(fd - d) <= 1e-5 * abs(d), (fd, d)
