"""Pins of the FP64 oracle against what the paper and mechanics fix.

Each test checks a closed form, a threshold, an invariant or a special case
that a plausible slip in the oracle (dropped term, wrong sign, transposed
operand, wrong update order) would break.  No GPU needed.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle_adapter import params, system
import oracle_cases as cases

G, DT = cases.G, cases.DT


def _one_step(wl, **over):
    s = system(wl, **over)
    st = s.step()
    return s, st


# --- single contact (Fig. 2, Eqs. 3-5) -------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_resting_particle_normal_impulse_is_weight(dim):
    """A particle at rest on the floor: P_n = m g dt after the solve, P_t = 0,
    and the new velocity is zero (Sec. 2.1, Eqs. 1, 3, 5)."""
    wl = cases.resting_disc(dim=dim)
    s, st = _one_step(wl, criterion=O.CRIT_GLOBAL_REL, alpha=1e-14)
    m = 1.0 / wl.inv_m[0]
    P = s.impulses
    assert s.nc == 1 and st["converged"]
    assert P[0, 0] == pytest.approx(m * G * DT, rel=1e-15, abs=0)
    assert np.all(np.abs(P[0, 1:]) < 1e-18)
    assert np.all(np.abs(s.v) < 1e-18)
    # wall force reported by the solve: the weight m g
    assert st["wall_force"][2 if dim == 2 else 4] == pytest.approx(m * G, rel=1e-14)


def _moving_floor(dim, u):
    """A particle resting on a kinematic floor that moves along its normal
    (up, +y in 2D and +z in 3D) at speed u."""
    wl = cases.resting_disc(dim=dim)
    k = 2 if dim == 2 else 4
    wv = np.zeros((6, 3))
    wv[k, dim - 1] = u
    wl.wall_vel = wv
    return wl, k


@pytest.mark.parametrize("dim", [2, 3])
def test_rising_floor_carries_the_particle(dim):
    """A kinematic wall (infinite mass, prescribed velocity) moving up at u
    under a touching particle: the contact closes perfectly inelastically, so
    the particle leaves with the wall's velocity, P_n = m (u + g dt), and
    both advance by u dt (Eqs. 1-5, the walls moving kinematically)."""
    u = 0.5
    wl, k = _moving_floor(dim, u)
    y0 = float(wl.x[0, dim - 1])
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    m = 1.0 / wl.inv_m[0]
    P = s.impulses
    assert s.nc == 1
    assert P[0, 0] == pytest.approx(m * (u + G * DT), rel=1e-14)
    v = np.asarray(s.v).reshape(-1)
    assert v[dim - 1] == pytest.approx(u, rel=1e-14)
    assert np.all(np.abs(np.delete(v, dim - 1)) < 1e-18)
    assert s.wall_pos[k] == pytest.approx(u * DT, rel=1e-14)
    assert float(np.asarray(s.x).reshape(-1)[dim - 1]) == pytest.approx(y0 + u * DT, rel=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_receding_floor_opens_the_contact(dim):
    """The floor moving down faster than the particle falls in one step
    (u > g dt): the contact opens (P = 0, Eq. 3) and the particle falls
    freely, v = -g dt."""
    wl, k = _moving_floor(dim, -10.0 * G * DT)
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    assert s.nc == 1
    assert np.all(s.impulses == 0.0)
    v = np.asarray(s.v).reshape(-1)
    assert v[dim - 1] == pytest.approx(-G * DT, rel=1e-15)


def test_open_contact_keeps_zero_force():
    """Eq. 3: a contact whose gap stays positive with R = 0 gets no force."""
    wl = cases.resting_disc()
    wl.x[0, 1] = 1.1          # gap 0.1 < delta: detected, but stays open
    s, st = _one_step(wl)
    assert s.nc == 1
    assert np.all(s.impulses == 0.0)
    assert s.v[1] == pytest.approx(-G * DT, rel=1e-15)
    assert st["sweeps"] == 1 and st["converged"]


# --- the iterated network (Sec. 2.1) -----------------------------------------

@pytest.mark.parametrize("order", [O.ORDER_RANDOM, O.ORDER_COLOUR])
def test_vertical_column_static_force_chain(order):
    """Column of n equal discs on the floor: contact k from the top carries
    k m g dt, no tangential force; same in random sequential and colour order."""
    n = 6
    wl = cases.column(n=n)
    s, st = _one_step(wl, order=order, criterion=O.CRIT_GLOBAL_REL, alpha=1e-15, max_sweeps=20000)
    m = 1.0 / wl.inv_m[0]
    pairs, P = s.contacts, s.impulses
    assert st["converged"]
    assert len(pairs) == n     # n-1 disc pairs + floor
    for (a, b), (pn, pt) in zip(pairs, P):
        k = n - a if b == n + 2 else n - 1 - a   # discs above this contact
        assert pn == pytest.approx(k * m * G * DT, rel=1e-9)
        assert abs(pt) < 1e-15
    assert np.max(np.abs(s.v)) < 1e-9


def test_column_local_criterion_reaches_the_chain():
    """Convergence test (I) stops with every contact close to k m g dt."""
    n = 6
    wl = cases.column(n=n)
    s, st = _one_step(wl, order=O.ORDER_RANDOM, criterion=O.CRIT_LOCAL, alpha=1e-12, max_sweeps=20000)
    assert st["converged"]
    m = 1.0 / wl.inv_m[0]
    for (a, b), (pn, _) in zip(s.contacts, s.impulses):
        k = n - a if b == n + 2 else n - 1 - a
        assert pn == pytest.approx(k * m * G * DT, rel=1e-4)


def test_compressed_chain_carries_the_force_everywhere():
    """Fig. 13(a): a chain of touching discs pressed by F against a fixed
    wall carries F dt on every contact once converged."""
    F = 2.5
    wl, f = cases.chain(n=8, force=F)
    s, st = _one_step(wl, f_ext=f, order=O.ORDER_RANDOM, criterion=O.CRIT_GLOBAL_REL, alpha=1e-15,
                      max_sweeps=50000)
    assert st["converged"]
    assert s.nc == 8
    assert np.allclose(s.impulses[:, 0], F * DT, rtol=1e-9, atol=0)


def test_chain_iterations_grow_diffusively():
    """Sec. 4.3: forces relax diffusively, so the sweeps needed grow ~ n^2
    (loose check: doubling the chain needs well over twice the sweeps)."""
    sweeps = []
    for n in (8, 16):
        wl, f = cases.chain(n=n, force=1.0)
        s, st = _one_step(wl, f_ext=f, order=O.ORDER_RANDOM, criterion=O.CRIT_LOCAL, alpha=1e-10,
                          max_sweeps=200000)
        assert st["converged"]
        sweeps.append(st["sweeps"])
    assert sweeps[1] > 2.5 * sweeps[0]


# --- Coulomb friction (Eqs. 6-11) --------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_incline_frozen_rotation_stick_below_tan_mu(dim):
    mu = 0.4
    th = math.atan(0.9 * mu)
    wl = cases.incline(th, mu, dim=dim, frozen=True)
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    m = 1.0 / wl.inv_m[0]
    P = s.impulses[0]
    assert P[0] == pytest.approx(m * G * math.cos(th) * DT, rel=1e-13)
    pt = abs(P[1]) if dim == 2 else float(np.linalg.norm(P[1:]))
    assert pt == pytest.approx(m * G * math.sin(th) * DT, rel=1e-13)
    assert np.max(np.abs(s.v)) < 1e-15      # stuck


@pytest.mark.parametrize("dim", [2, 3])
def test_incline_frozen_rotation_slides_above_tan_mu(dim):
    mu = 0.4
    th = math.atan(1.1 * mu)
    wl = cases.incline(th, mu, dim=dim, frozen=True)
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    P = s.impulses[0]
    pt = abs(P[1]) if dim == 2 else float(np.linalg.norm(P[1:]))
    assert pt == pytest.approx(mu * P[0], rel=1e-14)
    # sliding: a = g (sin th - mu cos th) along the slope, friction opposing
    assert s.v[0] == pytest.approx(G * (math.sin(th) - mu * math.cos(th)) * DT, rel=1e-12)
    # the tangential impulse opposes the motion: on the particle it points to -x
    force_on_particle_x = -(P[1] if dim == 2 else P[1])
    assert force_on_particle_x < 0


@pytest.mark.parametrize("dim,factor,roll_frac", [(2, 3.0, 2.0 / 3.0), (3, 3.5, 5.0 / 7.0)])
def test_incline_free_rotation_rolls_until_threshold(dim, factor, roll_frac):
    """A free disc rolls without slipping while tan(theta) <= 3 mu (sphere:
    7 mu / 2): then v = (2/3) g sin(theta) dt (sphere 5/7) and the contact
    point is at rest; beyond the threshold it slips."""
    mu = 0.2
    th = math.atan(0.9 * factor * mu)
    wl = cases.incline(th, mu, dim=dim, frozen=False)
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    r = wl.r[0]
    assert s.v[0] == pytest.approx(roll_frac * G * math.sin(th) * DT, rel=1e-12)
    if dim == 2:
        # contact point (below the centre, arm -r e_y): v_x + w r = 0
        assert abs(s.v[0] + s.w[0] * r) < 1e-15
    else:
        # arm -r e_z: v + w x (-r e_z) -> x component v_x - w_y r
        assert abs(s.v[0] - s.w[1] * r) < 1e-15
    P = s.impulses[0]
    pt = abs(P[1]) if dim == 2 else float(np.linalg.norm(P[1:]))
    assert pt < mu * P[0]
    th2 = math.atan(1.1 * factor * mu)
    wl2 = cases.incline(th2, mu, dim=dim, frozen=False)
    s2, _ = _one_step(wl2, alpha=1e-15, max_sweeps=100)
    P2 = s2.impulses[0]
    pt2 = abs(P2[1]) if dim == 2 else float(np.linalg.norm(P2[1:]))
    assert pt2 == pytest.approx(mu * P2[0], rel=1e-14)
    slip = (s2.v[0] + s2.w[0] * r) if dim == 2 else (s2.v[0] - s2.w[1] * r)
    assert slip > 1e-9


PHI = 0.7   # an azimuth off both floor axes


def _tangential(P):
    """(P_t along the slope's downhill direction, across it, its z part)."""
    c, s = math.cos(PHI), math.sin(PHI)
    return P[1] * c + P[2] * s, -P[1] * s + P[2] * c, P[3]


def test_oblique_incline_3d_stick_keeps_the_downhill_direction():
    """A sphere (rotation frozen) on a slope whose downhill direction is at
    azimuth phi: below tan(theta) = mu it sticks, with the whole tangential
    impulse m g sin(theta) dt along the slope and none across it."""
    mu = 0.4
    th = math.atan(0.9 * mu)
    wl = cases.incline(th, mu, dim=3, frozen=True, azimuth=PHI)
    s, _ = _one_step(wl, alpha=1e-15, max_sweeps=100)
    m = 1.0 / wl.inv_m[0]
    P = s.impulses[0]
    along, across, z = _tangential(P)
    assert P[0] == pytest.approx(m * G * math.cos(th) * DT, rel=1e-13)
    assert abs(along) == pytest.approx(m * G * math.sin(th) * DT, rel=1e-13)
    assert abs(across) <= 1e-15 * abs(along) and z == 0.0
    assert np.max(np.abs(s.v)) < 1e-15


def test_oblique_incline_3d_slides_along_the_trial_velocity():
    """Above tan(theta) = mu the sphere slides downhill: |P_t| = mu P_n,
    P_t parallel to the trial tangential velocity (Eqs. 9-11 with an
    isotropic tangential mass), and v = g (sin(theta) - mu cos(theta)) dt
    along (cos phi, sin phi)."""
    mu = 0.4
    th = math.atan(1.1 * mu)
    wl = cases.incline(th, mu, dim=3, frozen=True, azimuth=PHI)
    s, _ = _one_step(wl, alpha=1e-15, max_sweeps=100)
    P = s.impulses[0]
    along, across, z = _tangential(P)
    assert math.hypot(along, across) == pytest.approx(mu * P[0], rel=1e-14)
    assert abs(across) <= 1e-14 * abs(along) and z == 0.0
    speed = G * (math.sin(th) - mu * math.cos(th)) * DT
    v = np.asarray(s.v).reshape(-1)[:3]   # particle 0: (v_x, v_y, v_z)
    assert v[0] == pytest.approx(speed * math.cos(PHI), rel=1e-12)
    assert v[1] == pytest.approx(speed * math.sin(PHI), rel=1e-12)
    assert abs(v[2]) < 1e-15


def test_oblique_incline_3d_rolls_about_the_cross_slope_axis():
    """A free sphere below tan(theta) = 7 mu / 2 rolls without slipping:
    v = (5/7) g sin(theta) dt downhill and the contact point (arm -r e_z) is
    at rest, v_x - r w_y = 0 and v_y + r w_x = 0, so w is about the axis
    across the slope."""
    mu = 0.2
    th = math.atan(0.9 * 3.5 * mu)
    wl = cases.incline(th, mu, dim=3, frozen=False, azimuth=PHI)
    s, _ = _one_step(wl, alpha=1e-15, max_sweeps=100)
    r = wl.r[0]
    v = np.asarray(s.v).reshape(-1)[:3]    # particle 0: (v_x, v_y, v_z)
    wv = np.asarray(s.w).reshape(-1)[:3]   # (w_x, w_y, w_z)
    speed = 5.0 / 7.0 * G * math.sin(th) * DT
    assert v[0] == pytest.approx(speed * math.cos(PHI), rel=1e-12)
    assert v[1] == pytest.approx(speed * math.sin(PHI), rel=1e-12)
    assert abs(v[0] - r * wv[1]) < 1e-15
    assert abs(v[1] + r * wv[0]) < 1e-15
    assert abs(wv[2]) < 1e-15


# --- glancing collision of touching particles (Fig. 2, Eqs. 3-11) -----------

def _glancing(dim, mu):
    """Particles a and b touching along an oblique unit normal e, approaching
    with a tangential relative velocity and spinning; no gravity, no walls.
    The centre offset and its length are exact in binary (3-4-5 and 1-2-2-3
    triangles), so the gap is exactly 0."""
    if dim == 2:
        ra, rb = 1.5, 1.0
        off = np.array([1.5, 2.0])              # length 2.5 = ra + rb
        xa = np.array([5.0, 5.0])
        va, vb = [0.3, -0.1], [-0.2, 0.1]
        w = [0.4, -0.3]
        lo, hi = (0.0, 0.0, 0.0), (20.0, 20.0, 1.0)
    else:
        ra, rb = 1.75, 1.25
        off = np.array([1.0, 2.0, 2.0])         # length 3 = ra + rb
        xa = np.array([5.0, 5.0, 5.0])
        va, vb = [0.3, -0.1, 0.2], [-0.2, 0.4, -0.3]
        w = [[0.1, 0.0, -0.2], [0.0, 0.3, 0.1]]
        lo, hi = (0.0, 0.0, 0.0), (20.0, 20.0, 20.0)
    e = off / (ra + rb)
    xb = xa + off
    wl = cases._wl("glancing", dim, [xa, xb], [ra, rb], v=[va, vb], w=w, dt=DT, mu=mu,
                   gravity=(0.0, 0.0, 0.0), box_lo=lo, box_hi=hi)
    return wl, e


def _point_velocity(dim, v, w, arm):
    """Velocity of the material point at `arm` from the centre: v + w x arm."""
    if dim == 2:
        return v + w * np.array([-arm[1], arm[0]])
    return v + np.cross(w, arm)


def _contact_velocity(wl, e, v, w):
    d = wl.dim
    v = np.asarray(v).reshape(2, d)
    w = np.asarray(w).reshape(2, -1) if d == 3 else np.asarray(w).reshape(2)
    pa = _point_velocity(d, v[0], w[0], wl.r[0] * e)
    pb = _point_velocity(d, v[1], w[1], -wl.r[1] * e)
    return pb - pa


def _momenta(wl, x, v, w):
    """Linear momentum and angular momentum about the origin."""
    d = wl.dim
    m = 1.0 / wl.inv_m
    I = 1.0 / wl.inv_I
    x = np.asarray(x).reshape(2, d)
    v = np.asarray(v).reshape(2, d)
    p = (m[:, None] * v).sum(axis=0)
    if d == 2:
        w = np.asarray(w).reshape(2)
        L = float((m * (x[:, 0] * v[:, 1] - x[:, 1] * v[:, 0])).sum() + (I * w).sum())
        return p, np.array([L])
    w = np.asarray(w).reshape(2, 3)
    L = (m[:, None] * np.cross(x, v)).sum(axis=0) + (I[:, None] * w).sum(axis=0)
    return p, L


@pytest.mark.parametrize("dim", [2, 3])
def test_glancing_collision_sticks_at_the_contact_point(dim):
    """With ample friction the single contact sticks: afterwards the two
    material points at the contact have the same velocity (normal: Eq. 4 with
    gap 0; tangential: the stick solution of Eq. 5), while linear momentum
    and angular momentum about the origin are those of before (an equal and
    opposite impulse pair at one point)."""
    wl, e = _glancing(dim, mu=10.0)
    p0, L0 = _momenta(wl, wl.x, wl.v, wl.w)
    u0 = _contact_velocity(wl, e, wl.v, wl.w)
    assert float(u0 @ e) < 0.0                       # approaching
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    assert s.impulses.shape[0] == 1 and st["converged"]
    u = _contact_velocity(wl, e, s.v, s.w)
    assert np.max(np.abs(u)) <= 1e-15 * 1e2 * np.max(np.abs(u0))
    p1, L1 = _momenta(wl, wl.x, s.v, s.w)
    assert np.max(np.abs(p1 - p0)) <= 1e-15 * np.max(np.abs(p0)) * 10
    assert np.max(np.abs(L1 - L0)) <= 1e-14 * (np.max(np.abs(L0)) + 1.0)
    P = s.impulses[0]
    pt = abs(P[1]) if dim == 2 else float(np.linalg.norm(P[1:]))
    assert 0.0 < pt < 10.0 * P[0]


@pytest.mark.parametrize("dim", [2, 3])
def test_glancing_collision_slides_against_the_tangential_velocity(dim):
    """With little friction the contact slides: the normal relative velocity
    of the contact points vanishes, |P_t| = mu P_n, and the tangential
    relative velocity keeps its direction and shrinks (Eqs. 9-11 with an
    isotropic tangential mass); the momenta are unchanged."""
    mu = 0.05
    wl, e = _glancing(dim, mu=mu)
    p0, L0 = _momenta(wl, wl.x, wl.v, wl.w)
    u0 = _contact_velocity(wl, e, wl.v, wl.w)
    u0t = u0 - (u0 @ e) * e
    s, st = _one_step(wl, alpha=1e-15, max_sweeps=100)
    assert s.impulses.shape[0] == 1 and st["converged"]
    u = _contact_velocity(wl, e, s.v, s.w)
    ut = u - (u @ e) * e
    assert abs(float(u @ e)) <= 1e-14 * np.max(np.abs(u0))
    P = s.impulses[0]
    pt = abs(P[1]) if dim == 2 else float(np.linalg.norm(P[1:]))
    assert pt == pytest.approx(mu * P[0], rel=1e-13)
    cosang = float(ut @ u0t) / (np.linalg.norm(ut) * np.linalg.norm(u0t))
    assert cosang == pytest.approx(1.0, abs=1e-13)
    assert 0.0 < np.linalg.norm(ut) < np.linalg.norm(u0t)
    p1, L1 = _momenta(wl, wl.x, s.v, s.w)
    assert np.max(np.abs(p1 - p0)) <= 1e-15 * np.max(np.abs(p0)) * 10
    assert np.max(np.abs(L1 - L0)) <= 1e-14 * (np.max(np.abs(L0)) + 1.0)


# --- perfectly inelastic collision (Sec. 2.1, Eq. 4) -------------------------

@pytest.mark.parametrize("r1,r2,v1,v2", [(1.0, 1.0, 2.0, -2.0), (1.2, 0.8, 3.0, -0.5)])
def test_head_on_collision_closes_gap_then_moves_together(r1, r2, v1, v2):
    wl = cases.head_on(v1, v2, r1=r1, r2=r2)
    m1, m2 = 1.0 / wl.inv_m[0], 1.0 / wl.inv_m[1]
    p0 = m1 * v1 + m2 * v2
    s = system(wl, alpha=1e-15, max_sweeps=100)
    s.step()
    vx = s.v.reshape(2, 2)[:, 0]
    x = s.x.reshape(2, 2)
    gap = (x[1, 0] - x[0, 0]) - (r1 + r2)
    assert abs(gap) < 1e-13                          # Eq. 4: the new gap is zero
    assert m1 * vx[0] + m2 * vx[1] == pytest.approx(p0, rel=1e-14)
    s.step()                                         # touching now: no rebound
    vx = s.v.reshape(2, 2)[:, 0]
    vc = p0 / (m1 + m2)
    assert vx[0] == pytest.approx(vc, rel=1e-12, abs=1e-14)
    assert vx[1] == pytest.approx(vc, rel=1e-12, abs=1e-14)


# --- invariants ----------------------------------------------------------------

def _gas(n=300, L=60.0, seed=3, dim=2):
    from paper_1104_3516_gb300 import workloads as W
    r = W.uniform(seed, n, 0.8, 1.2)
    x = W.rsa(dim, n, r, (0.0,) * dim, (L,) * dim, (1,) * dim, seed)
    v = W.normal(seed, n * dim, 1.0).reshape(n, dim)
    inv_m, inv_I = W.masses(dim, r)
    w = np.zeros(n) if dim == 2 else np.zeros((n, 3))
    return W.Workload(name="gas", dim=dim, x=x, v=v, w=w, r=r, inv_m=inv_m, inv_I=inv_I, dt=2e-2,
                      gravity=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(L, L, L), periodic=(1, 1, 1))


@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_conserved_without_walls(dim):
    """Each contact applies +P and -P, so total momentum is conserved and the
    perfectly inelastic contacts never add kinetic energy."""
    wl = _gas(dim=dim)
    m = 1.0 / wl.inv_m
    s = system(wl, alpha=1e-10, max_sweeps=500)
    p0 = (m[:, None] * s.v.reshape(-1, dim)).sum(axis=0)
    scale = float((m[:, None] * np.abs(s.v.reshape(-1, dim))).sum())

    def ke():
        v = s.v.reshape(-1, dim)
        I = 1.0 / wl.inv_I
        wr = s.w.reshape(len(m), -1)
        return 0.5 * float((m[:, None] * v * v).sum()) + 0.5 * float((I[:, None] * wr * wr).sum())

    e_prev = ke()
    touched = 0
    for _ in range(15):
        st = s.step()
        touched += int(np.count_nonzero(s.impulses[:, 0]))
        e = ke()
        assert e <= e_prev * (1 + 1e-12)
        e_prev = e
    p1 = (m[:, None] * s.v.reshape(-1, dim)).sum(axis=0)
    assert touched > 0
    assert np.all(np.abs(p1 - p0) <= 1e-13 * scale)


def test_free_fall_is_semi_implicit_euler():
    """Eqs. 1-2: v(t+dt) = v + g dt, then r(t+dt) = r + v(t+dt) dt, so after k
    steps y = y0 - g dt^2 k (k + 1) / 2 (an explicit update would give k(k-1)/2)."""
    wl = cases.resting_disc()
    wl.x[0, 1] = 5.0
    s = system(wl)
    k = 7
    for _ in range(k):
        s.step()
    assert s.v[1] == pytest.approx(-G * DT * k, rel=1e-14)
    assert s.x[1] == pytest.approx(5.0 - G * DT * DT * k * (k + 1) / 2, rel=1e-14)


# --- convergence tests (Sec. 2.1) ----------------------------------------------

def test_free_spin_and_periodic_wrap():
    """Eq. 2 without contacts: a spinning disc's orientation advances by
    omega dt per step with omega unchanged, and a disc crossing the periodic
    x boundary re-enters at the other side (x + v dt - L)."""
    L = 10.0
    wl = cases._wl("spin", 2, [[9.875, 5.0]], [1.0], v=[[50.0, 0.0]], w=[2.0], dt=DT, mu=0.3,
                   gravity=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(L, 10.0, 1.0), periodic=(1, 0, 0))
    s = system(wl, alpha=1e-15, max_sweeps=10)
    x = [float(s.x[0])]
    for k in range(1, 4):
        s.step()
        assert s.nc == 0
        assert s.w[0] == 2.0
        assert s.theta[0] == pytest.approx(k * 2.0 * DT, rel=1e-15)
        x.append(float(s.x[0]))
        assert 0.0 <= x[-1] < L
    # 9.875 -> 9.925 -> 9.975 -> 10.025 - L = 0.025
    assert x[1] == pytest.approx(9.925, rel=1e-15)
    assert x[2] == pytest.approx(9.975, rel=1e-15)
    assert x[3] == pytest.approx(0.025, rel=1e-12)


def test_colour_and_random_orders_agree_on_a_settled_pile():
    """The colour order is a sequential order of the same scheme (Sec. 2.1):
    on a 1000-disc pile resting on the floor both orders converge (1e-10) to
    the same floor force, equal to the pile's weight, and the same height;
    the forces themselves need not agree (hyperstatic network, Sec. 4.4)."""
    from paper_1104_3516_gb300 import workloads as W
    wl = W.dense_biaxial_discs(n=1000)
    wl.wall_mask = 0b0100
    out = {}
    for order in (O.ORDER_COLOUR, O.ORDER_RANDOM):
        s = system(wl, alpha=1e-10, max_sweeps=200000, order=order)
        st = s.step()
        assert st["converged"]
        out[order] = (st["wall_force"][2], float(np.max(s.x.reshape(-1, 2)[:, 1] + wl.r)))
    (fc, hc), (fr, hr) = out[O.ORDER_COLOUR], out[O.ORDER_RANDOM]
    assert fc == pytest.approx(fr, rel=1e-6)
    assert fc == pytest.approx(float(np.sum(1.0 / wl.inv_m)), rel=1e-4)
    assert hc == pytest.approx(hr, rel=1e-6)


def test_squared_global_test_matches_plain_test_at_sqrt_alpha():
    """Test (II) compares the squared ratio with alpha: equivalent to the
    plain ratio against sqrt(alpha)."""
    wl = cases.column(n=5)
    _, st_sq = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_GLOBAL_SQ, alpha=1e-12, max_sweeps=10000)
    _, st_pl = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_GLOBAL_REL, alpha=1e-6, max_sweeps=10000)
    assert st_sq["sweeps"] == st_pl["sweeps"] and st_sq["converged"] and st_pl["converged"]
    _, st_tight = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_GLOBAL_REL, alpha=1e-12, max_sweeps=10000)
    assert st_tight["sweeps"] > st_pl["sweeps"]


def test_zero_alpha_never_converges_and_hits_the_cap():
    wl = cases.column(n=4)
    _, st = _one_step(wl, alpha=0.0, max_sweeps=37)
    assert st["sweeps"] == 37 and not st["converged"]


def test_warm_start_reuses_the_previous_forces():
    """A static column stepped twice: with the forces carried over the second
    solve needs only a few sweeps; from zero forces it needs as many again."""
    wl = cases.column(n=5)
    s = system(wl, alpha=1e-13, max_sweeps=20000, order=O.ORDER_RANDOM)
    st1 = s.step()
    st2 = s.step()
    assert st1["sweeps"] > 10
    assert 4 * st2["sweeps"] < st1["sweeps"]
    s_cold = system(wl, alpha=1e-13, max_sweeps=20000, order=O.ORDER_RANDOM, warm_start=0)
    s_cold.step()
    st_cold = s_cold.step()
    assert st_cold["sweeps"] > 4 * st2["sweeps"]


# --- mixed parallel / sequential update (Sec. 2.3) -----------------------------

def test_parallel_fraction_zero_is_the_sequential_scheme():
    wl = cases.column(n=5)
    a, st_a = _one_step(wl, order=O.ORDER_COLOUR, alpha=1e-13, max_sweeps=5000)
    b, st_b = _one_step(wl, order=O.ORDER_COLOUR, alpha=1e-13, max_sweeps=5000, parallel_p=0.0)
    assert st_a["sweeps"] == st_b["sweeps"]
    assert np.array_equal(a.impulses, b.impulses)


def test_jacobi_update_needs_more_sweeps_than_gauss_seidel():
    """Sec. 4.3: the parallel (Jacobi) update diffuses information more slowly
    (D_s / D_p ~ 1.5), so the chain needs more sweeps; both reach F dt."""
    F = 1.0
    out = {}
    for p in (0.0, 1.0):
        wl, f = cases.chain(n=12, force=F)
        s, st = _one_step(wl, f_ext=f, order=O.ORDER_RANDOM, criterion=O.CRIT_LOCAL, alpha=1e-16,
                          max_sweeps=200000, parallel_p=p)
        assert st["converged"]
        assert np.allclose(s.impulses[:, 0], F * DT, rtol=1e-5)
        out[p] = st["sweeps"]
    assert out[1.0] > 1.2 * out[0.0]


def _splitmix64(x):
    """splitmix64 (Steele, Lea and Flood, OOPSLA 2014), the generator the
    parallel subset is drawn with: restated here to predict the draws."""
    M = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def _drawn_parallel(a, b, seed, p, sweep):
    """Whether contact (a, b) is in the re-drawn parallel subset of iteration
    step `sweep` (0-based): a uniform number from splitmix64 of the key mixed
    with the seed and the step number, below p."""
    M = (1 << 64) - 1
    x = ((a << 32) | b) ^ ((seed * 0xD1B54A32D192ED03) & M) ^ (((sweep + 1) * 0x9E3779B97F4A7C15) & M)
    return (_splitmix64(x) >> 11) * (1.0 / 9007199254740992.0) < p


@pytest.mark.parametrize("seed", [3, 11, 12345])
def test_redrawn_parallel_subset_follows_the_stack_recursion(seed):
    """Sec. 2.3 with the parallel subset drawn afresh in every iteration
    step.  Two discs stacked on the floor, forces from zero, in units of
    m g dt: the disc-disc contact B is updated before the floor contact A,
    and always sees the old A (B_k = A_(k-1) / 2: it comes first, and a
    parallel A's change lands at the end of the sweep).  A sees the new B of
    its sweep (A_k = 1 + B_k) only if neither contact is parallel; a parallel
    A works from the sweep's start and a parallel B's change lands at the
    end, so otherwise A_k = 1 + B_(k-1).  The draws, predicted from the
    generator's definition, must reproduce the oracle's impulses sweep by
    sweep, and differ from sweep to sweep."""
    wl = cases.stack2()
    wl.seed = seed
    unit = G * DT / wl.inv_m[0]
    p = 0.5
    A, B = 0.0, 0.0
    draws = []
    for k in range(1, 9):
        parA = _drawn_parallel(0, 4, seed, p, k - 1)
        parB = _drawn_parallel(0, 1, seed, p, k - 1)
        draws.append((parA, parB))
        Bk = A / 2.0
        A = 1.0 + (B if (parA or parB) else Bk)
        B = Bk
        s, _ = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=k, warm_start=0,
                         parallel_p=p, parallel_redraw=1)
        assert s.contacts.tolist() == [[0, 1], [0, 4]]
        assert s.impulses[1, 0] == pytest.approx(A * unit, rel=1e-12)
        assert s.impulses[0, 0] == pytest.approx(B * unit, rel=1e-12, abs=1e-18)
    assert len(set(draws)) > 1              # the subset changes between steps


def test_redrawn_subset_limits_are_the_fixed_schemes():
    """p = 0 and p = 1 draw the same subsets in every step, so both
    readings give the sequential and the Jacobi scheme, bit for bit."""
    F = 1.0
    for p in (0.0, 1.0):
        wl, f = cases.chain(n=12, force=F)
        a, st_a = _one_step(wl, f_ext=f, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=60, parallel_p=p)
        b, st_b = _one_step(wl, f_ext=f, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=60, parallel_p=p,
                            parallel_redraw=1)
        assert np.array_equal(a.impulses, b.impulses)


# --- observables of Sec. 4.4 ---------------------------------------------------

def test_column_observables_closed_form():
    """A static column: every force is vertical (orientation bin of pi/2), and
    the stress in a stripe of width 2 r equals (load x branch) / (L_x x 2 r):
    the floor contact carries n m g with branch r, the contact below disc k
    (from the top) carries k m g with branch 2 r."""
    n = 6
    wl = cases.column(n=n)
    s, st = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_GLOBAL_REL, alpha=1e-15, max_sweeps=20000)
    hist = O.force_orientation(s.impulses, s.normal[: s.nc], nbins=18)
    assert hist.sum() == n and hist[9] == n
    m, r = 1.0 / wl.inv_m[0], wl.r[0]
    Lx = wl.box_hi[0] - wl.box_lo[0]
    sig = O.stress_profile(s.x, wl.r, wl.n, s.contacts, s.normal[: s.nc], s.gap[: s.nc], s.impulses, DT, 1, 0.0,
                           2 * r, n + 1, Lx)
    expect = np.zeros(n + 1)
    expect[0] = n * m * G * r / (Lx * 2 * r)
    for k in range(1, n):       # contact between disc k-1 and k (from the bottom) lies at y = 2 k r
        expect[k] = (n - k) * m * G * 2 * r / (Lx * 2 * r)
    assert np.allclose(sig, expect, rtol=1e-9, atol=0)


# --- force-controlled walls (the pressure walls of Fig. 10) ------------------------

def test_pressed_column_carries_the_push():
    """A lid of mass M pushed with force F onto a column resting on a fixed
    floor, no gravity: the lid's momentum F dt (Eq. 1) is stopped by the
    rigid column in the step, so every contact carries F dt, the floor and
    the lid both see the force F, and nothing moves."""
    F = 2.0
    wl = cases.pressed_column(n=5, push=F, lid_mass=50.0)
    s = system(wl, order=O.ORDER_RANDOM, alpha=1e-14, max_sweeps=20000)
    for _ in range(3):
        st = s.step()
        assert st["converged"]
        assert np.allclose(s.impulses[:, 0], F * DT, rtol=1e-9, atol=0)
        assert np.allclose(s.impulses[:, 1], 0.0, atol=1e-15)
        assert st["wall_force"][2] == pytest.approx(F, rel=1e-9)
        assert st["wall_force"][3] == pytest.approx(F, rel=1e-9)
        assert abs(s.p.wall_vel[3 * 3 + 1]) <= 1e-12
        assert np.abs(s.v).max() <= 1e-12
    assert s.wall_pos[3] == pytest.approx(wl.wall_pos[3], abs=1e-14)


def test_free_lid_accelerates_with_its_push():
    """With no contact the lid follows Eq. 1-2 alone: after k steps it has
    moved down by (F/M) dt^2 k (k + 1) / 2."""
    F, M = 3.0, 7.0
    wl = cases.pressed_column(n=2, push=F, lid_mass=M, lid_gap=2.0)
    s = system(wl, order=O.ORDER_RANDOM)
    k = 6
    for _ in range(k):
        s.step()
    assert s.wall_pos[3] == pytest.approx(wl.wall_pos[3] - (F / M) * DT * DT * k * (k + 1) / 2, rel=0, abs=1e-13)


def test_contacts_on_a_force_controlled_wall_conflict():
    """On a kinematic wall contacts never conflict; on a force-controlled
    wall (a body) they must all get different colours."""
    n = 6
    pairs = np.array([[i, n + 2] for i in range(n)], dtype=np.int32)
    c0, K0 = O.colour_greedy(n, pairs, seed=5)
    c1, K1 = O.colour_greedy(n, pairs, seed=5, dyn_walls=1 << 2)
    assert K0 == 1 and K1 == n and len(set(c1.tolist())) == n


# --- domain-wise update of the parallel algorithm (Sec. 3.1, Sec. 4.3) -----------

def test_domains_sharing_no_particle_give_gauss_seidel():
    """Two columns in two slabs share no particle, so each domain's sweep is
    the Gauss-Seidel sweep of its column: same sweeps, same impulses (up to
    the rounding of summing the domains' velocity changes)."""
    wl = cases.two_columns(n=4)
    a, st_a = _one_step(wl, order=O.ORDER_COLOUR, alpha=1e-13, max_sweeps=5000)
    b, st_b = _one_step(wl, order=O.ORDER_COLOUR, alpha=1e-13, max_sweeps=5000, domains=(2, 1, 1))
    assert st_a["sweeps"] == st_b["sweeps"]
    assert np.array_equal(a.contacts, b.contacts)
    assert np.allclose(b.impulses, a.impulses, rtol=1e-13, atol=1e-18)
    assert np.allclose(b.v, a.v, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_stack_split_between_two_domains_is_a_jacobi_pair(k):
    """Two discs on the floor (floor contact A, disc-disc contact B), forces
    from zero, in units of m g dt.  One domain, colour order (B first, its
    particles have more contacts): Gauss-Seidel gives B_k = A_{k-1} / 2,
    A_k = 1 + B_k, i.e. A_k = 2 - 2^(1-k), B_k = 1 - 2^(1-k).  A and B in
    different domains see each other's impulse of the previous sweep only
    (Sec. 3.1): A_k = 1 + B_{k-1}, B_k = A_{k-1} / 2, i.e.
    A_k = 2 - 2^(1 - ceil(k/2)), B_k = 1 - 2^(-floor(k/2))."""
    wl = cases.stack2()
    unit = G * DT / wl.inv_m[0]
    gs, _ = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=k, warm_start=0)
    jac, _ = _one_step(wl, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=k, warm_start=0,
                       domains=(1, 3, 1))
    # contact 0 is (0, 1) = B, contact 1 is (0, wall 2) = A
    assert gs.contacts.tolist() == [[0, 1], [0, 4]]
    A_gs, B_gs = 2.0 - 2.0 ** (1 - k), 1.0 - 2.0 ** (1 - k)
    A_j, B_j = 2.0 - 2.0 ** (1 - math.ceil(k / 2)), 1.0 - 2.0 ** (-(k // 2))
    assert gs.impulses[1, 0] == pytest.approx(A_gs * unit, rel=1e-12)
    assert gs.impulses[0, 0] == pytest.approx(B_gs * unit, rel=1e-12, abs=1e-18)
    assert jac.impulses[1, 0] == pytest.approx(A_j * unit, rel=1e-12)
    assert jac.impulses[0, 0] == pytest.approx(B_j * unit, rel=1e-12, abs=1e-18)


def test_contact_domains_follow_the_middle_of_the_gap():
    """The domain of a contact is the slab of the middle of its gap: the
    chain's contacts sit at x = 2 k r, one per slab of width 2 r."""
    n = 6
    wl, _ = cases.chain_slabs(n=n)
    p = params(wl, domains=(n, 1, 1))
    pairs = O.detect_brute(p, wl.x, wl.r, wl.wall_pos)
    normal, gap, _, _ = O.contact_geometry(p, wl.x, wl.r, wl.inv_m, wl.inv_I, wl.wall_pos, pairs)
    dom, nd = O.contact_domains(p, wl.x, wl.r, pairs, normal, gap)
    assert nd == n
    expect = [b if b < n else 0 for a, b in pairs.tolist()]   # (k-1, k) at x = 2 k r; the wall contact at 0
    assert dom.tolist() == expect


def test_every_contact_in_its_own_domain_is_the_parallel_update():
    """With one contact per domain nothing is sequential: every contact is
    computed from the velocities of the sweep start and applied at its end,
    which is the mixed update of Sec. 2.3 with p = 1 (Jacobi)."""
    n = 6
    wl, f = cases.chain_slabs(n=n, force=1.0)
    kw = dict(f_ext=f, order=O.ORDER_COLOUR, criterion=O.CRIT_NONE, max_sweeps=40, warm_start=0)
    dom, _ = _one_step(wl, domains=(n, 1, 1), **kw)
    jac, _ = _one_step(wl, parallel_p=1.0, **kw)
    seq, _ = _one_step(wl, **kw)
    assert np.allclose(dom.impulses, jac.impulses, rtol=1e-12, atol=1e-18)
    assert np.allclose(dom.v, jac.v, rtol=0, atol=1e-14)
    assert not np.allclose(dom.impulses, seq.impulses, rtol=1e-3)


def test_domain_boundaries_slow_the_chain_like_a_parallel_fraction():
    """Sec. 4.3, Fig. 13(b): a chain of n discs pressed against a wall,
    forces from zero, random sequential order within each of N_p domains.
    Boundaries act as parallel update, so the sweeps to reach the squared
    global test at 1e-12 grow with N_p as D_s / D_eff with
    D_eff = D_p p + D_s (1 - p), p = N_p / n.  The fitted ratio D_s / D_p
    lies near the paper's values (1.53 fitted, ~1.59 from q_s / q_p)."""
    n = 24
    mean = {}
    for Np in (1, 4, 12):
        sw = []
        for seed in range(4):
            wl, f = cases.chain_slabs(n=n, force=1.0)
            s, st = _one_step(wl, f_ext=f, order=O.ORDER_RANDOM, criterion=O.CRIT_GLOBAL_SQ, alpha=1e-12,
                              max_sweeps=200000, domains=(Np, 1, 1), seed=seed, warm_start=0)
            assert st["converged"]
            sw.append(st["sweeps"])
        mean[Np] = float(np.mean(sw))
    assert mean[1] < mean[4] < mean[12]
    ratios = []
    for Np in (4, 12):
        p = Np / n
        nt = mean[Np] / mean[1]            # = 1 / (1 - p + p D_p / D_s)
        ratios.append(p / (1.0 / nt - 1.0 + p))
    assert all(1.35 < q < 1.85 for q in ratios), ratios
