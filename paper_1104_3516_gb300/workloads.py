"""Seeded synthetic packings shaped like the paper's workloads.

Input generation only: nothing here computes a contact force, an impulse or
any step of the Contact Dynamics method.  Both the CUDA library and the CPU
oracle consume these arrays unchanged, so this module is the only code the
two share.

Each builder returns a :class:`Workload`: particle arrays (numpy, FP64) plus
the physical parameters of the run.  Masses follow density 1: a disc of radius
r has m = pi r^2 (areal mass) and I = m r^2 / 2; a sphere m = 4/3 pi r^3 and
I = 2/5 m r^2.  Particle ids are sorted by a coarse spatial grid (rows of
height 2 r_max, then x) so that touching particles have nearby ids.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen", "cd_workloads.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libcd_workloads.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _gen():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            d, i64, u64 = C.c_double, C.c_int64, C.c_uint64
            lib.wl_uniform.argtypes = [u64, i64, d, d, P(d)]
            lib.wl_normal.argtypes = [u64, i64, d, P(d)]
            lib.wl_rsa.restype = i64
            lib.wl_rsa.argtypes = [i64, i64, P(d), P(d), P(d), P(i64), d, u64, i64, P(d)]
            lib.wl_deposit2d.restype = i64
            lib.wl_deposit2d.argtypes = [i64, P(d), d, d, u64, P(d)]
            _lib = lib
    return _lib


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _seed(seed: int, stream: int) -> int:
    return (int(seed) * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03) & (2**64 - 1)


def uniform(seed: int, n: int, lo: float, hi: float, stream: int = 0) -> np.ndarray:
    out = np.zeros(max(n, 1))
    _gen().wl_uniform(C.c_uint64(_seed(seed, stream)), n, lo, hi, _p(out))
    return out[:n]


def normal(seed: int, n: int, sigma: float, stream: int = 1) -> np.ndarray:
    out = np.zeros(max(n, 1))
    _gen().wl_normal(C.c_uint64(_seed(seed, stream)), n, sigma, _p(out))
    return out[:n]


@dataclasses.dataclass
class Workload:
    """Particles plus run parameters; walls are indexed k = 2*axis + side."""
    name: str
    dim: int
    x: np.ndarray          # (n, dim)
    v: np.ndarray          # (n, dim)
    w: np.ndarray          # (n,) in 2D, (n, 3) in 3D
    r: np.ndarray
    inv_m: np.ndarray
    inv_I: np.ndarray
    dt: float = 1e-3
    mu: float = 0.3
    gravity: tuple = (0.0, -1.0, 0.0)
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (0, 0, 0)
    wall_mask: int = 0
    wall_pos: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(6))
    wall_vel: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((6, 3)))
    wall_push: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(6))   # force-controlled walls
    wall_mass: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(6))   # (mass 0: kinematic)
    delta: float = 0.24
    alpha: float = 1e-6
    max_sweeps: int = 1000
    steps: int = 1
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    @property
    def f_ext(self):
        return None


def masses(dim: int, r: np.ndarray):
    if dim == 2:
        m = math.pi * r * r
        I = 0.5 * m * r * r
    else:
        m = (4.0 / 3.0) * math.pi * r ** 3
        I = 0.4 * m * r * r
    return 1.0 / m, 1.0 / I


def spatial_order(x: np.ndarray, cell: float) -> np.ndarray:
    """Permutation sorting particles by grid row (then higher axes), then x."""
    D = x.shape[1]
    keys = [x[:, 0]]
    for k in range(1, D):
        keys.append(np.floor(x[:, k] / cell))
    return np.lexsort(tuple(keys))


def _finish(name, dim, x, r, v=None, w=None, order=True, **kw) -> Workload:
    n = r.shape[0]
    if order and n > 0:
        perm = spatial_order(x, 2.0 * float(r.max()))
        x, r = x[perm], r[perm]
        if v is not None:
            v = v[perm]
        if w is not None:
            w = w[perm]
    inv_m, inv_I = masses(dim, r)
    if v is None:
        v = np.zeros((n, dim))
    if w is None:
        w = np.zeros(n) if dim == 2 else np.zeros((n, 3))
    return Workload(name=name, dim=dim, x=np.ascontiguousarray(x), v=np.ascontiguousarray(v),
                    w=np.ascontiguousarray(w), r=np.ascontiguousarray(r), inv_m=inv_m, inv_I=inv_I, **kw)


def rsa(dim, n, r, lo, hi, periodic, seed, min_gap=0.0, max_attempts=None):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    per = np.asarray(periodic, dtype=np.int64)
    x = np.zeros((max(n, 1), dim))
    max_attempts = max_attempts or 2000 * max(n, 1)
    got = _gen().wl_rsa(dim, n, _p(np.ascontiguousarray(r)), _p(lo), _p(hi), _p(per, C.c_int64), min_gap,
                        C.c_uint64(_seed(seed, 7)), max_attempts, _p(x))
    if got < n:
        raise RuntimeError(f"random sequential addition placed {got} of {n} particles")
    return x[:n]


def deposit2d(n, r, Lx, ymax, seed):
    x = np.zeros((max(n, 1), 2))
    got = _gen().wl_deposit2d(n, _p(np.ascontiguousarray(r)), Lx, ymax, C.c_uint64(_seed(seed, 11)), _p(x))
    if got < n:
        raise RuntimeError(f"deposition placed {got} of {n} discs below height {ymax}")
    return x[:n]


# --------------------------------------------------------------------------
# The five workload shapes.  Sizes default to the full configurations; the
# `n` arguments shrink them for fast tests.
# --------------------------------------------------------------------------

def dilute_discs(seed=1105, n=1000, width=40.0, phi=0.40, mu=0.3, steps=200) -> Workload:
    """1000 frictional discs, r ~ U[0.8, 1.2], RSA at packing fraction 0.40
    in a box 40 wide with floor and side walls, open top (gravity 1 in -y)."""
    r = uniform(seed, n, 0.8, 1.2)
    area = float(np.sum(math.pi * r * r))
    height = area / (width * phi)
    x = rsa(2, n, r, (0.0, 0.0), (width, height), (0, 0), seed)
    wp = np.zeros(6)
    wp[1] = width
    wp[3] = height + 2.4
    return _finish("dilute_discs_2d", 2, x, r, mu=mu, gravity=(0.0, -1.0, 0.0), box_lo=(0.0, 0.0, 0.0),
                   box_hi=(width, height + 2.4, 1.0), periodic=(0, 0, 0), wall_mask=0b0111, wall_pos=wp,
                   steps=steps, seed=seed)


def dense_biaxial_discs(seed=1106, n=100_000, phi=0.80, mu=0.3, steps=100, wall_speed=1e-3) -> Workload:
    """N discs, r ~ U[0.8, 1.2], box width sqrt(sum(pi r^2) / 0.80) (the
    square box at packing fraction 0.80), periodic in x, floor fixed and the
    top wall pushed down at 1e-3.  The discs are gravity-deposited so every
    disc rests on two supports (a loaded static network; gravity 1 in -y).
    Deposition is looser than 0.80, so the pile stands slightly taller than
    wide; the top wall starts touching the highest disc."""
    r = uniform(seed, n, 0.8, 1.2)
    area = float(np.sum(math.pi * r * r))
    L = math.sqrt(area / phi)
    x = deposit2d(n, r, L, 2.0 * L, seed)
    top = float(np.max(x[:, 1] + r))
    wp = np.zeros(6)
    wp[2] = 0.0
    wp[3] = top
    wv = np.zeros((6, 3))
    wv[3, 1] = -wall_speed
    return _finish("dense_biaxial_discs_2d", 2, x, r, mu=mu, gravity=(0.0, -1.0, 0.0), box_lo=(0.0, 0.0, 0.0),
                   box_hi=(L, top, 1.0), periodic=(1, 0, 0), wall_mask=0b1100, wall_pos=wp, wall_vel=wv,
                   steps=steps, seed=seed)


def sphere_gas(seed=1107, n=1_000_000, floor=100.0, phi=0.3, mu=0.5, vsig=0.1, steps=50) -> Workload:
    """Spheres r ~ U[0.8, 1.2], RSA gas at packing fraction 0.3 over a
    floor x floor base with floor and four side walls, velocities N(0, 0.1).
    The fraction is taken over the region the sphere centres can reach."""
    r = uniform(seed, n, 0.8, 1.2)
    vol = float(np.sum((4.0 / 3.0) * math.pi * r ** 3))
    # packing fraction over the region the centres can reach (inside the walls)
    height = vol / ((floor - 2.4) ** 2 * phi) + 2.4
    x = rsa(3, n, r, (0.0, 0.0, 0.0), (floor, floor, height), (0, 0, 0), seed)
    v = normal(seed, 3 * n, vsig).reshape(n, 3)
    wp = np.zeros(6)
    wp[1] = floor
    wp[3] = floor
    wp[5] = height + 2.4
    # gravity along -z; the floor is wall 4 (z low)
    return _finish("sphere_gas_3d", 3, x, r, v=v, mu=mu, gravity=(0.0, 0.0, -1.0), box_lo=(0.0, 0.0, 0.0),
                   box_hi=(floor, floor, height + 2.4), periodic=(0, 0, 0), wall_mask=0b011111, wall_pos=wp,
                   steps=steps, seed=seed)


def jittered_lattice(n, r, width, phi, seed):
    """Triangular lattice filling a box `width` wide row by row, with the
    spacing a of packing fraction phi and each site jittered uniformly by up
    to (a - 2 r_max) / 2 per axis, so no two discs overlap."""
    rmax = float(r.max())
    area = float(np.sum(math.pi * r * r))
    a = math.sqrt(2.0 * area / (n * phi * math.sqrt(3.0)))
    if a < 2.0 * rmax:
        raise RuntimeError(f"packing fraction {phi} too high for a jittered lattice")
    nx = max(1, int(math.floor((width - 2.0 * rmax - 0.5 * a) / a)) + 1)
    j = np.arange(n)
    row, col = j // nx, j % nx
    x = rmax + col * a + 0.5 * a * (row % 2)
    y = rmax + row * a * math.sqrt(3.0) / 2.0
    jit = 0.5 * (a - 2.0 * rmax)
    x = x + uniform(seed, n, -jit, jit, stream=21)
    y = y + uniform(seed, n, -jit, jit, stream=22)
    return np.stack([x, y], axis=1)


def settling_discs(seed=1109, n=10_000, phi=0.5, mu=0.3, vsig=0.05, steps=200, width=None) -> Workload:
    """Discs r ~ U[0.8, 1.2] on a jittered triangular lattice at packing
    fraction phi in a square box with floor and side walls, initial
    velocities N(0, vsig), gravity 1: a loose packing that settles."""
    r = uniform(seed, n, 0.8, 1.2)
    area = float(np.sum(math.pi * r * r))
    L = math.sqrt(area / phi) if width is None else width
    x = jittered_lattice(n, r, L, phi, seed)
    H = float(np.max(x[:, 1] + r)) + 0.5
    v = normal(seed, 2 * n, vsig).reshape(n, 2) if vsig > 0 else None
    wp = np.zeros(6)
    wp[1] = L
    wp[3] = H
    return _finish("settling_discs_2d", 2, x, r, v=v, mu=mu, gravity=(0.0, -1.0, 0.0), box_lo=(0.0, 0.0, 0.0),
                   box_hi=(L, H, 1.0), periodic=(0, 0, 0), wall_mask=0b0111, wall_pos=wp, steps=steps,
                   seed=seed)


def pressure_column(seed=1112, n=8000, width_diameters=20, pressure=0.25, mu=0.3, lid_mass=None,
                    steps=200) -> Workload:
    """The medium test system of Fig. 10: n discs with 20% polydispersity
    (r ~ U[0.8, 1.2]) in a box periodic in x, width_diameters mean diameters
    wide, between a fixed floor and a force-controlled lid (wall 3) pressing
    with `pressure` times the width; no gravity.  The discs are deposited
    first (every disc resting on two supports), the lid starts on the
    highest one.  lid_mass defaults to the mass of one layer of discs."""
    r = uniform(seed, n, 0.8, 1.2)
    Lx = 2.0 * float(np.mean(r)) * width_diameters
    area = float(np.sum(math.pi * r * r))
    x = deposit2d(n, r, Lx, 4.0 * area / Lx, seed)
    top = float(np.max(x[:, 1] + r))
    wp = np.zeros(6)
    wp[3] = top
    push = np.zeros(6)
    push[3] = pressure * Lx
    mass = np.zeros(6)
    mass[3] = lid_mass if lid_mass is not None else float(width_diameters) * math.pi
    wl = _finish("pressure_column_2d", 2, x, r, mu=mu, gravity=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0),
                 box_hi=(Lx, top + 2.0, 1.0), periodic=(1, 0, 0), wall_mask=0b1100, wall_pos=wp, steps=steps,
                 seed=seed)
    wl.wall_push = push
    wl.wall_mass = mass
    return wl


def sliding_pyramids(seed=1113, n_pyramids=3334, spacing=8.0, floor_speed=1.0, base_gap=1.0, mu=0.3,
                     steps=200) -> Workload:
    """Pyramids of three discs, r ~ U[0.8, 1.2], on a floor that moves
    sideways at `floor_speed` under them, periodic in x (one pyramid per
    `spacing` of floor), at rest, gravity 1: two base discs stand on the
    floor `base_gap` apart and the third rests on both (all contact gaps 0).
    The floor slides under the base discs all along a 200-step rollout, so
    friction drives the pyramids and, through the top disc's inclined
    contacts, their floor forces and heights: a contact-dominated case
    whose losses depend on mu, with four contacts per nine degrees of
    freedom (no hyperstatic network)."""
    r = uniform(seed, 3 * n_pyramids, 0.8, 1.2).reshape(n_pyramids, 3)
    x = np.zeros((n_pyramids, 3, 2))
    for k in range(n_pyramids):
        r1, r2, r3 = r[k]
        c1 = np.array([k * spacing + r1, r1])
        c2 = np.array([c1[0] + r1 + r2 + base_gap, r2])
        # the top centre: distance r1 + r3 from c1 and r2 + r3 from c2, above them
        a, b = r1 + r3, r2 + r3
        d = float(np.linalg.norm(c2 - c1))
        along = (a * a - b * b + d * d) / (2.0 * d)
        h = math.sqrt(a * a - along * along)
        e = (c2 - c1) / d
        c3 = c1 + along * e + h * np.array([-e[1], e[0]])
        x[k] = [c1, c2, c3]
    L = n_pyramids * spacing
    top = float(np.max(x[:, :, 1] + r))
    wv = np.zeros((6, 3))
    wv[2, 0] = floor_speed
    return _finish("sliding_pyramids_2d", 2, x.reshape(-1, 2), r.reshape(-1), mu=mu, gravity=(0.0, -1.0, 0.0),
                   box_lo=(0.0, 0.0, 0.0), box_hi=(L, top + 10.0, 1.0), periodic=(1, 0, 0), wall_mask=0b0100,
                   wall_pos=np.zeros(6), wall_vel=wv, steps=steps, seed=seed)


def batch_sizes(seed=1108, n_packings=512, nmin=200, nmax=20000) -> np.ndarray:
    """Disc counts log-uniform in [nmin, nmax] per packing."""
    u = uniform(seed, n_packings, 0.0, 1.0, stream=3)
    return np.floor(np.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))).astype(np.int64)


def settled_pile(seed, n, phi=0.5, mu=0.3, steps=100):
    """n discs r ~ U[0.8, 1.2] gravity-deposited into a box of width
    sqrt(sum pi r^2 / phi) (the square box at packing fraction phi),
    periodic in x, floor at y = 0, open top: a settled, loaded pile."""
    r = uniform(seed, n, 0.8, 1.2)
    area = float(np.sum(math.pi * r * r))
    L = math.sqrt(area / phi)
    x = deposit2d(n, r, L, 4.0 * L, seed)
    top = float(np.max(x[:, 1] + r))
    wp = np.zeros(6)
    return _finish("settled_pile_2d", 2, x, r, mu=mu, gravity=(0.0, -1.0, 0.0), box_lo=(0.0, 0.0, 0.0),
                   box_hi=(L, max(L, top + 2.4), 1.0), periodic=(1, 0, 0), wall_mask=0b0100, wall_pos=wp,
                   steps=steps, seed=seed)


def shard_range(n_items, rank, world):
    """The contiguous index range [lo, hi) of the items rank `rank` of
    `world` takes: the ranks' ranges are disjoint, in rank order, and cover
    all items (sizes differ by at most one)."""
    return (n_items * rank) // world, (n_items * (rank + 1)) // world


def batched_settling(seed=1108, n_packings=512, nmin=200, nmax=20000, steps=100, shard=None):
    """Independent packings: disc counts log-uniform in [nmin, nmax], mu ~
    U[0.1, 0.6] each, every packing settled under gravity in its box sized
    to packing fraction 0.5 (see settled_pile).  Packing b depends only on
    (seed, b), so `shard = (rank, world)` builds just that rank's packings
    (shard_range): the same ones a single process builds at those indices."""
    sizes = batch_sizes(seed, n_packings, nmin, nmax)
    mus = uniform(seed, n_packings, 0.1, 0.6, stream=4)
    out = []
    lo, hi = (0, n_packings) if shard is None else shard_range(n_packings, shard[0], shard[1])
    for b in range(lo, hi):
        w = settled_pile(seed=_seed(seed, 100 + b) & 0xFFFFFFFF, n=int(sizes[b]), phi=0.5, mu=float(mus[b]),
                         steps=steps)
        w.name = "batched_settling_2d"
        out.append(w)
    return out
