"""Tiny hand-built systems with closed-form answers (shared by the oracle pin
tests and the GPU parity tests).  Pure input construction: no CD arithmetic.
"""
import math

import numpy as np

from paper_1104_3516_gb300.workloads import Workload, masses

G = 1.0
DT = 1e-3


def _wl(name, dim, x, r, v=None, w=None, inv_I=None, **kw):
    x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
    r = np.asarray(r, dtype=np.float64)
    n = r.shape[0]
    inv_m, iI = masses(dim, r)
    if inv_I is not None:
        iI = np.asarray(inv_I, dtype=np.float64)
    v = np.zeros((n, dim)) if v is None else np.asarray(v, dtype=np.float64).reshape(n, dim)
    if w is None:
        w = np.zeros(n) if dim == 2 else np.zeros((n, 3))
    return Workload(name=name, dim=dim, x=x, v=v, w=np.asarray(w, dtype=np.float64), r=r, inv_m=inv_m,
                    inv_I=iI, **kw)


def resting_disc(dim=2, radius=1.0, mu=0.3):
    """One particle touching the floor (gap 0), at rest, gravity 1."""
    if dim == 2:
        return _wl("resting_disc", 2, [[0.0, radius]], [radius], dt=DT, mu=mu, gravity=(0.0, -G, 0.0),
                   box_lo=(-10.0, 0.0, 0.0), box_hi=(10.0, 10.0, 1.0), wall_mask=0b0100)
    return _wl("resting_sphere", 3, [[0.0, 0.0, radius]], [radius], dt=DT, mu=mu, gravity=(0.0, 0.0, -G),
               box_lo=(-10.0, -10.0, 0.0), box_hi=(10.0, 10.0, 10.0), wall_mask=0b010000)


def column(n=6, radius=1.0, mu=0.3):
    """n equal discs stacked vertically on the floor, all gaps exactly 0."""
    y = radius + 2.0 * radius * np.arange(n)
    x = np.stack([np.zeros(n), y], axis=1)
    return _wl("column", 2, x, np.full(n, radius), dt=DT, mu=mu, gravity=(0.0, -G, 0.0),
               box_lo=(-5.0, 0.0, 0.0), box_hi=(5.0, 2.0 * radius * n + 5.0, 1.0), wall_mask=0b0100)


def chain(n=8, radius=1.0, force=1.0):
    """n equal discs in a row along x touching each other, the first touching
    the fixed wall x = 0; a force `force` pushes the last one towards the wall.
    No gravity.  Returns (workload, f_ext)."""
    xs = radius + 2.0 * radius * np.arange(n)
    x = np.stack([xs, np.zeros(n)], axis=1)
    wl = _wl("chain", 2, x, np.full(n, radius), dt=DT, mu=0.3, gravity=(0.0, 0.0, 0.0),
             box_lo=(0.0, -5.0, 0.0), box_hi=(2.0 * radius * n + 5.0, 5.0, 1.0), wall_mask=0b0001)
    f = np.zeros((n, 2))
    f[-1, 0] = -force
    return wl, f


def incline(theta, mu, dim=2, frozen=True, radius=1.0, azimuth=0.0):
    """One particle resting on the floor with gravity tilted by theta:
    g = (sin theta, -cos theta) (2D) or (sin theta cos phi, sin theta sin phi,
    -cos theta) (3D, phi = azimuth: the slope's downhill direction in the
    floor plane)."""
    if dim == 2:
        inv_I = np.zeros(1) if frozen else None
        return _wl("incline", 2, [[0.0, radius]], [radius], inv_I=inv_I, dt=DT, mu=mu,
                   gravity=(G * math.sin(theta), -G * math.cos(theta), 0.0), box_lo=(-10.0, 0.0, 0.0),
                   box_hi=(10.0, 10.0, 1.0), wall_mask=0b0100)
    inv_I = np.zeros(1) if frozen else None
    gx = G * math.sin(theta) * math.cos(azimuth)
    gy = G * math.sin(theta) * math.sin(azimuth) if azimuth != 0.0 else 0.0
    return _wl("incline3", 3, [[0.0, 0.0, radius]], [radius], inv_I=inv_I, dt=DT, mu=mu,
               gravity=(gx, gy, -G * math.cos(theta)), box_lo=(-10.0, -10.0, 0.0),
               box_hi=(10.0, 10.0, 10.0), wall_mask=0b010000)


def head_on(v1, v2, r1=1.0, r2=1.0, gap=None):
    """Two discs on the x axis approaching each other; no gravity, no walls."""
    if gap is None:
        gap = 0.5 * (v1 - v2) * DT
    x = [[0.0, 0.0], [r1 + r2 + gap, 0.0]]
    return _wl("head_on", 2, x, [r1, r2], v=[[v1, 0.0], [v2, 0.0]], dt=DT, mu=0.3, gravity=(0.0, 0.0, 0.0),
               box_lo=(-20.0, -20.0, 0.0), box_hi=(20.0, 20.0, 1.0))


def colliding_gas(n=40, seed=1110, vsig=2.0, dt=0.01, phi=0.55, mu=0.3):
    """A loose lattice of discs in a box with floor and side walls, gravity 1,
    fast random velocities and a long time step, so that within a few steps
    many pairs collide (open, sticking and sliding contacts side by side)."""
    from paper_1104_3516_gb300.workloads import settling_discs
    wl = settling_discs(seed=seed, n=n, phi=phi, mu=mu, vsig=vsig, steps=5)
    wl.dt = dt
    return wl


def periodic_gas(n=36, seed=1111, vsig=2.0, dt=0.01, phi=0.55, mu=0.3):
    """The same gas in a box periodic in x and y: no walls, no gravity (total
    momentum is then conserved by every step)."""
    wl = colliding_gas(n=n, seed=seed, vsig=vsig, dt=dt, phi=phi, mu=mu)
    top = float(np.max(wl.x[:, 1] + wl.r)) + 0.3
    wl.box_lo = (0.0, 0.0, 0.0)
    wl.box_hi = (float(wl.box_hi[0]), top, 1.0)
    wl.periodic = (1, 1, 0)
    wl.wall_mask = 0
    wl.gravity = (0.0, 0.0, 0.0)
    return wl


def leaning_column(offsets=(0.2, -0.6, 0.3, -0.25, 0.65), radius=1.0, mu=0.3, rotations=True):
    """Equal discs stacked on the floor, each touching the one below with
    the horizontal offset given (gaps exactly 0 up to rounding), gravity 1:
    every contact carries weight; the larger offsets make contacts slide."""
    x = [[0.0, radius]]
    for dx in offsets:
        px, py = x[-1]
        x.append([px + dx, py + math.sqrt((2.0 * radius) ** 2 - dx * dx)])
    n = len(x)
    inv_I = None if rotations else np.zeros(n)
    return _wl("leaning_column", 2, x, np.full(n, radius), inv_I=inv_I, dt=DT, mu=mu, gravity=(0.0, -G, 0.0),
               box_lo=(-10.0, 0.0, 0.0), box_hi=(10.0, 2.0 * radius * n + 5.0, 1.0), wall_mask=0b0100)


def pressed_column(n=5, radius=1.0, push=2.0, lid_mass=50.0, mu=0.3, lid_gap=0.0):
    """n equal discs stacked on a fixed floor under a force-controlled lid
    (wall 3, mass lid_mass, pushed down with force `push`), no gravity; the
    lid starts at rest lid_gap above the top disc."""
    y = radius + 2.0 * radius * np.arange(n)
    x = np.stack([np.zeros(n), y], axis=1)
    top = float(y[-1] + radius) + lid_gap
    wl = _wl("pressed_column", 2, x, np.full(n, radius), dt=DT, mu=mu, gravity=(0.0, 0.0, 0.0),
             box_lo=(-5.0, 0.0, 0.0), box_hi=(5.0, top + 5.0, 1.0), wall_mask=0b1100)
    wp = np.zeros(6)
    wp[3] = top
    wl.wall_pos = wp
    wl.wall_push = np.array([0.0, 0.0, 0.0, push, 0.0, 0.0])
    wl.wall_mass = np.array([0.0, 0.0, 0.0, lid_mass, 0.0, 0.0])
    return wl


def stack2(radius=1.0, mu=0.3):
    """Two equal discs stacked on the floor (gaps 0), gravity 1; the box
    [-5, 5] x [0, 4.5] cut into 3 slabs along y puts the floor contact
    (middle of its gap at y = 0) and the disc-disc contact (y = 2 r) in
    different domains."""
    return _wl("stack2", 2, [[0.0, radius], [0.0, 3.0 * radius]], [radius, radius], dt=DT, mu=mu,
               gravity=(0.0, -G, 0.0), box_lo=(-5.0, 0.0, 0.0), box_hi=(5.0, 4.5 * radius, 1.0), wall_mask=0b0100)


def two_columns(n=4, radius=1.0, mu=0.3):
    """Two columns of n discs on the floor at x = -3 and x = +3: two slabs
    along x separate them completely."""
    y = radius + 2.0 * radius * np.arange(n)
    x = np.concatenate([np.stack([np.full(n, -3.0), y], axis=1), np.stack([np.full(n, 3.0), y], axis=1)])
    return _wl("two_columns", 2, x, np.full(2 * n, radius), dt=DT, mu=mu, gravity=(0.0, -G, 0.0),
               box_lo=(-6.0, 0.0, 0.0), box_hi=(6.0, 2.0 * radius * n + 5.0, 1.0), wall_mask=0b0100)


def chain_slabs(n=8, radius=1.0, force=1.0):
    """The chain of :func:`chain` in the box [-r, (2 n - 1) r] along x, so
    that n equal slabs along x are centred on the contact points 2 k r
    (k = 0: the wall contact); with N_p slabs, N_p dividing n, every slab
    holds n / N_p contacts.  Returns (workload, f_ext)."""
    wl, f = chain(n=n, radius=radius, force=force)
    wl.box_lo = (-radius, -5.0, 0.0)
    wl.box_hi = ((2.0 * n - 1.0) * radius, 5.0, 1.0)
    return wl, f


def floor_row(radii, spacing=3.0, mu=0.3):
    """Discs of the given radii resting on the floor (gaps 0), `spacing`
    apart along x so that no two touch; gravity 1."""
    r = np.asarray(radii, dtype=np.float64)
    n = r.shape[0]
    x = np.stack([spacing * np.arange(n), r], axis=1)
    return _wl("floor_row", 2, x, r, dt=DT, mu=mu, gravity=(0.0, -G, 0.0), box_lo=(-5.0, 0.0, 0.0),
               box_hi=(spacing * n + 5.0, 10.0, 1.0), wall_mask=0b0100)
