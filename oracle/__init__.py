"""FP64 CPU oracle of the Contact Dynamics time step (arXiv:1104.3516).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(the CUDA library and its Python binding) never imports this package.

This module is argument marshalling around ``cd_oracle.c`` (plain C, compiled
with ``-O2 -ffp-contract=off``).  Every function cites the part of the paper
it restates:

* :func:`detect_brute` / :func:`detect_cells` -- contact detection, Sec. 3.2
  (cell method) with the margin of Eq. 12 / Sec. 3.1 (l = 2.2 r_max).
* :func:`contact_geometry` -- normal, gap and pair mass matrix, Sec. 2.1,
  Fig. 1, Eq. 5.
* :func:`colour_greedy` -- greedy colouring of the contact graph (the order
  the GPU sweeps in; not in the paper, which sweeps sequentially).
* :func:`solve` -- iterative Gauss-Seidel force calculation, Sec. 2.1 and
  Fig. 2 (Eqs. 3-11), convergence tests (I)/(II); mixed parallel update of
  Sec. 2.3; domain-wise update of Sec. 3.1 (with :func:`contact_domains`).
* :func:`step` -- one time step, Fig. 3 with Eqs. 1-2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libcd_oracle.so")
_lock = threading.Lock()
_lib = None

CRIT_NONE, CRIT_GLOBAL_REL, CRIT_GLOBAL_SQ, CRIT_LOCAL = -1, 0, 1, 2
ORDER_COLOUR, ORDER_RANDOM, ORDER_FIXED = 0, 1, 2


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int64),
        ("dt", C.c_double),
        ("mu", C.c_double),
        ("gravity", C.c_double * 3),
        ("box_lo", C.c_double * 3),
        ("box_hi", C.c_double * 3),
        ("periodic", C.c_int64 * 3),
        ("wall_mask", C.c_int64),
        ("wall_vel", C.c_double * 18),
        ("delta", C.c_double),
        ("alpha", C.c_double),
        ("criterion", C.c_int64),
        ("max_sweeps", C.c_int64),
        ("order", C.c_int64),
        ("warm_start", C.c_int64),
        ("seed", C.c_uint64),
        ("parallel_p", C.c_double),
        ("rotations", C.c_int64),
        ("wall_push", C.c_double * 6),
        ("wall_mass", C.c_double * 6),
        ("domains", C.c_int64 * 3),
        ("parallel_redraw", C.c_int64),
    ]


class SolveStats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64),
        ("converged", C.c_int64),
        ("residual", C.c_double),
        ("r_avg", C.c_double),
        ("r_avg_prev", C.c_double),
        ("n_colours", C.c_int64),
        ("wall_force", C.c_double * 6),
    ]

    def as_dict(self):
        return {
            "sweeps": int(self.sweeps),
            "converged": bool(self.converged),
            "residual": float(self.residual),
            "r_avg": float(self.r_avg),
            "r_avg_prev": float(self.r_avg_prev),
            "n_colours": int(self.n_colours),
            "wall_force": [float(v) for v in self.wall_force],
        }


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_lib`` (no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared",
            "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.POINTER
            d, i32, i64 = C.c_double, C.c_int32, C.c_longlong
            _lib.ora_splitmix64.restype = C.c_uint64
            _lib.ora_splitmix64.argtypes = [C.c_uint64]
            for name in ("ora_detect_brute", "ora_detect_cells"):
                f = getattr(_lib, name)
                f.restype = i64
                f.argtypes = [P(Params), i64, P(d), P(d), P(d), i64, P(i32)]
            _lib.ora_contact_geometry.restype = None
            _lib.ora_contact_geometry.argtypes = [P(Params), i64, P(d), P(d), P(d), P(d), P(d), i64, P(i32),
                                                  P(d), P(d), P(d), P(d)]
            _lib.ora_colour_greedy.restype = C.c_int
            _lib.ora_colour_greedy.argtypes = [i64, i64, P(i32), C.c_uint64, C.c_int64, P(i32)]
            _lib.ora_colour_repair.restype = C.c_int
            _lib.ora_colour_repair.argtypes = [i64, i64, P(i32), C.c_int64, P(i32)]
            _lib.ora_solve.restype = C.c_int
            _lib.ora_solve.argtypes = [P(Params), i64, P(d), P(d), P(d), P(d), P(d), i64, P(i32), P(d), P(d),
                                       P(d), P(d), P(i32), P(i32), P(i32), i64, P(d), P(d),
                                       P(SolveStats)]
            _lib.ora_contact_domains.restype = i64
            _lib.ora_contact_domains.argtypes = [P(Params), i64, P(d), P(d), i64, P(i32), P(d), P(d), P(i32)]
            _lib.ora_step.restype = C.c_int
            _lib.ora_step.argtypes = [P(Params), i64, P(d), P(d), P(d), P(d), P(d), P(d), P(d), P(d), P(d),
                                      i64, P(i64), P(i32), P(d), i64, C.c_int, P(i32), P(d), P(d),
                                      P(SolveStats)]
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(dim=2, dt=1e-3, mu=0.3, gravity=(0.0, -1.0, 0.0), box_lo=(0, 0, 0), box_hi=(1, 1, 1),
                periodic=(0, 0, 0), wall_mask=0, wall_vel=None, delta=0.24, alpha=1e-6,
                criterion=CRIT_GLOBAL_REL, max_sweeps=1000, order=ORDER_COLOUR, warm_start=1, seed=0,
                parallel_p=0.0, rotations=1, wall_push=None, wall_mass=None, domains=(1, 1, 1),
                parallel_redraw=0) -> Params:
    p = Params()
    p.dim = dim
    p.dt = dt
    p.mu = mu
    for k in range(3):
        p.gravity[k] = gravity[k]
        p.box_lo[k] = box_lo[k]
        p.box_hi[k] = box_hi[k]
        p.periodic[k] = int(periodic[k])
    p.wall_mask = int(wall_mask)
    wv = np.zeros(18) if wall_vel is None else np.asarray(wall_vel, dtype=np.float64).reshape(18)
    for k in range(18):
        p.wall_vel[k] = float(wv[k])
    p.delta = delta
    p.alpha = alpha
    p.criterion = criterion
    p.max_sweeps = max_sweeps
    p.order = order
    p.warm_start = int(warm_start)
    p.seed = int(seed) & (2**64 - 1)
    p.parallel_p = parallel_p
    p.parallel_redraw = int(parallel_redraw)
    p.rotations = int(rotations)
    wp = np.zeros(6) if wall_push is None else np.asarray(wall_push, dtype=np.float64).reshape(6)
    wm = np.zeros(6) if wall_mass is None else np.asarray(wall_mass, dtype=np.float64).reshape(6)
    for k in range(6):
        p.wall_push[k] = float(wp[k])
        p.wall_mass[k] = float(wm[k])
    for k in range(3):
        p.domains[k] = int(domains[k])
    return p


def splitmix64(x: int) -> int:
    return int(lib().ora_splitmix64(C.c_uint64(int(x) & (2**64 - 1))))


def detect_brute(p: Params, x, r, wall_pos, cap=None):
    """All contact candidates by brute force over pairs (Sec. 3.2 baseline)."""
    x, r, wp = _f64(x).reshape(-1), _f64(r), _f64(wall_pos)
    n = r.shape[0]
    cap = cap if cap is not None else max(16, 8 * n)
    pairs = np.zeros((cap, 2), dtype=np.int32)
    nc = lib().ora_detect_brute(C.byref(p), n, _ptr(x, C.c_double), _ptr(r, C.c_double), _ptr(wp, C.c_double),
                                cap, _ptr(pairs, C.c_int32))
    if nc > cap:
        return detect_brute(p, x, r, wall_pos, cap=int(nc))
    return pairs[:nc].copy()


def detect_cells(p: Params, x, r, wall_pos, cap=None):
    """Cell-method contact detection (Sec. 3.2)."""
    x, r, wp = _f64(x).reshape(-1), _f64(r), _f64(wall_pos)
    n = r.shape[0]
    cap = cap if cap is not None else max(16, 8 * n)
    pairs = np.zeros((cap, 2), dtype=np.int32)
    nc = lib().ora_detect_cells(C.byref(p), n, _ptr(x, C.c_double), _ptr(r, C.c_double), _ptr(wp, C.c_double),
                                cap, _ptr(pairs, C.c_int32))
    if nc > cap:
        return detect_cells(p, x, r, wall_pos, cap=int(nc))
    return pairs[:nc].copy()


def contact_geometry(p: Params, x, r, inv_m, inv_I, wall_pos, pairs):
    """Normal (nc, 3), gap, m_n, m_t of each contact (Sec. 2.1, Eq. 5)."""
    x, r, im, iI, wp = _f64(x).reshape(-1), _f64(r), _f64(inv_m), _f64(inv_I), _f64(wall_pos)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    nc = pairs.shape[0]
    normal = np.zeros((max(nc, 1), 3))
    gap, mn, mt = (np.zeros(max(nc, 1)) for _ in range(3))
    lib().ora_contact_geometry(C.byref(p), r.shape[0], _ptr(x, C.c_double), _ptr(r, C.c_double),
                               _ptr(im, C.c_double), _ptr(iI, C.c_double), _ptr(wp, C.c_double), nc,
                               _ptr(pairs, C.c_int32), _ptr(normal, C.c_double), _ptr(gap, C.c_double),
                               _ptr(mn, C.c_double), _ptr(mt, C.c_double))
    return normal[:nc], gap[:nc], mn[:nc], mt[:nc]


def colour_greedy(n, pairs, seed, dyn_walls=0):
    """Greedy colouring in descending priority (largest degree first, then the
    splitmix64 hash), then the Kempe-chain repair of its highest colour
    (:func:`colour_repair`); dyn_walls: bit k for a force-controlled wall k,
    whose contacts conflict.  Returns (colour, K)."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    nc = pairs.shape[0]
    colour = np.zeros(max(nc, 1), dtype=np.int32)
    K = lib().ora_colour_greedy(n, nc, _ptr(pairs, C.c_int32), C.c_uint64(int(seed) & (2**64 - 1)),
                                int(dyn_walls), _ptr(colour, C.c_int32))
    return colour[:nc], int(K)


def colour_repair(n, pairs, colour, dyn_walls=0):
    """Kempe-chain repair of the highest colour of a proper contact colouring
    (see ora_colour_repair); returns (new colour, K)."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    nc = pairs.shape[0]
    col = np.ascontiguousarray(colour, dtype=np.int32).copy()
    if nc == 0:
        return col, 0
    K = lib().ora_colour_repair(n, nc, _ptr(pairs, C.c_int32), int(dyn_walls), _ptr(col, C.c_int32))
    return col[:nc], int(K)


def solve(p: Params, v_free, w_free, r, inv_m, inv_I, pairs, normal, gap, mn, mt, P0=None, colour=None,
          fixed=None, step_index=0, history=False, domain=None):
    """Gauss-Seidel impulse solve (Sec. 2.1, Fig. 2).

    ``v_free``/``w_free`` are the velocities without contact impulses; returns
    ``(P, v, w, stats[, ravg_history])`` where ``v``/``w`` include the final
    impulses.  P has 2 columns (Pn, Pt) in 2D and 4 (Pn, Ptx, Pty, Ptz) in 3D.
    ``domain`` (one id per contact, see :func:`contact_domains`) selects the
    domain-wise update of Sec. 3.1.
    """
    D = int(p.dim)
    pw = 2 if D == 2 else 4
    v = _f64(v_free).reshape(-1).copy()
    w = _f64(w_free).reshape(-1).copy()
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    nc = pairs.shape[0]
    P = np.zeros((max(nc, 1), pw)) if P0 is None else np.ascontiguousarray(P0, dtype=np.float64).reshape(-1, pw).copy()
    if P.shape[0] == 0:
        P = np.zeros((1, pw))
    col = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.int32)
    dom = None if domain is None else np.ascontiguousarray(domain, dtype=np.int32)
    hist = np.zeros(int(p.max_sweeps) + 1) if history else None
    st = SolveStats()
    normal = np.ascontiguousarray(normal, dtype=np.float64).reshape(-1, 3)
    lib().ora_solve(C.byref(p), _f64(r).shape[0], _ptr(v, C.c_double), _ptr(w, C.c_double),
                    _ptr(_f64(r), C.c_double), _ptr(_f64(inv_m), C.c_double), _ptr(_f64(inv_I), C.c_double),
                    nc, _ptr(pairs, C.c_int32), _ptr(normal, C.c_double), _ptr(_f64(gap), C.c_double),
                    _ptr(_f64(mn), C.c_double), _ptr(_f64(mt), C.c_double), _ptr(col, C.c_int32),
                    _ptr(fx, C.c_int32), _ptr(dom, C.c_int32), step_index, _ptr(P, C.c_double), _ptr(hist, C.c_double), C.byref(st))
    out = (P[:nc].copy(), v, w, st.as_dict())
    if history:
        return out + (hist[: st.sweeps + 1].copy(),)
    return out


def contact_domains(p: Params, x, r, pairs, normal, gap):
    """Domain of every contact for the domain-wise update of Sec. 3.1 (the
    slab grid of ``p.domains`` over the box, by the middle of the gap);
    returns (ids, number of domains)."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    nc = pairs.shape[0]
    out = np.zeros(max(nc, 1), dtype=np.int32)
    normal = np.ascontiguousarray(normal, dtype=np.float64).reshape(-1, 3)
    nd = lib().ora_contact_domains(C.byref(p), _f64(r).shape[0], _ptr(_f64(x).reshape(-1), C.c_double),
                                   _ptr(_f64(r), C.c_double), nc, _ptr(pairs, C.c_int32),
                                   _ptr(normal, C.c_double), _ptr(_f64(gap), C.c_double), _ptr(out, C.c_int32))
    return out[:nc], int(nd)


class OracleSystem:
    """State holder for stepping the oracle over several time steps (Fig. 3)."""

    def __init__(self, p: Params, x, v, w, r, inv_m, inv_I, wall_pos, theta=None, f_ext=None, cap=None,
                 use_cells=True):
        self.p = p
        self.D = int(p.dim)
        self.x = _f64(x).reshape(-1).copy()
        self.v = _f64(v).reshape(-1).copy()
        self.w = _f64(w).reshape(-1).copy()
        self.r = _f64(r).copy()
        self.n = self.r.shape[0]
        self.theta = np.zeros(self.n) if theta is None else _f64(theta).copy()
        self.inv_m = _f64(inv_m).copy()
        self.inv_I = _f64(inv_I).copy()
        self.f_ext = None if f_ext is None else _f64(f_ext).reshape(-1).copy()
        self.wall_pos = _f64(wall_pos).copy()
        self.cap = cap if cap is not None else max(64, 8 * self.n)
        self.pw = 2 if self.D == 2 else 4
        self.pairs = np.zeros((self.cap, 2), dtype=np.int32)
        self.P = np.zeros((self.cap, self.pw))
        self.colour = np.zeros(self.cap, dtype=np.int32)
        self.normal = np.zeros((self.cap, 3))
        self.gap = np.zeros(self.cap)
        self.nc = 0
        self.step_index = 0
        self.use_cells = use_cells

    def step(self):
        st = SolveStats()
        nc = C.c_longlong(self.nc)
        rc = lib().ora_step(C.byref(self.p), self.n, _ptr(self.x, C.c_double), _ptr(self.v, C.c_double),
                            _ptr(self.w, C.c_double), _ptr(self.theta, C.c_double), _ptr(self.r, C.c_double),
                            _ptr(self.inv_m, C.c_double), _ptr(self.inv_I, C.c_double),
                            _ptr(self.f_ext, C.c_double), _ptr(self.wall_pos, C.c_double), self.cap,
                            C.byref(nc), _ptr(self.pairs, C.c_int32), _ptr(self.P, C.c_double),
                            self.step_index, int(self.use_cells), _ptr(self.colour, C.c_int32),
                            _ptr(self.normal, C.c_double), _ptr(self.gap, C.c_double), C.byref(st))
        if rc != 0:
            raise RuntimeError(f"oracle contact capacity {self.cap} exceeded: {nc.value} needed")
        self.nc = int(nc.value)
        self.step_index += 1
        return st.as_dict()

    @property
    def contacts(self):
        return self.pairs[: self.nc].copy()

    @property
    def impulses(self):
        return self.P[: self.nc].copy()


# ---------------------------------------------------------------------------
# Observables of Sec. 4.4 (Figs. 14-15), restated in numpy from the impulses.
# ---------------------------------------------------------------------------

def force_orientation(P, normal, nbins=18):
    """Fig. 14: phi = arctan(R_y / R_x) of every contact force with a nonzero
    impulse, folded into [0, pi), counted in nbins equal bins (2D)."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 2)
    normal = np.asarray(normal, dtype=np.float64).reshape(-1, 3)
    keep = ~((P[:, 0] == 0.0) & (P[:, 1] == 0.0))
    pn, pt = P[keep, 0], P[keep, 1]
    nx, ny = normal[keep, 0], normal[keep, 1]
    rx = pn * nx - pt * ny
    ry = pn * ny + pt * nx
    phi = np.arctan2(ry, rx)
    phi = np.where(phi < 0.0, phi + np.pi, phi)
    phi = np.where(phi >= np.pi, phi - np.pi, phi)
    b = np.floor(phi / (np.pi / nbins)).astype(np.int64)
    b = np.clip(b, 0, nbins - 1)
    return np.bincount(b, minlength=nbins)


def stress_profile(x, r, n_particles, pairs, normal, gap, P, dt, axis, lo, width, nstripes, box_extent,
                   periodic_length=None):
    """Fig. 15: sigma_kk per stripe along axis k, sum of R_k l_k over the
    contacts whose contact point (middle of the gap, Sec. 3.1) lies in the
    stripe, divided by the stripe volume (width x box_extent of the other
    axes); l is the branch vector a -> b, or a's centre -> wall surface."""
    pairs = np.asarray(pairs)
    D = 2 if np.asarray(P).reshape(len(pairs), -1).shape[1] == 2 else 3
    x = np.asarray(x, dtype=np.float64).reshape(-1, D)
    P = np.asarray(P, dtype=np.float64).reshape(len(pairs), -1)
    normal = np.asarray(normal, dtype=np.float64).reshape(-1, 3)
    sig = np.zeros(nstripes)
    for c, (a, b) in enumerate(pairs):
        n = normal[c]
        if D == 2:
            t = np.array([-n[1], n[0], 0.0])
            R = (P[c, 0] * n + P[c, 1] * t) / dt
        else:
            R = (P[c, 0] * n + np.concatenate([P[c, 1:], []])) / dt
        if R[axis] == 0.0:
            continue
        point = x[a, axis] + (r[a] + 0.5 * gap[c]) * n[axis]
        if b < n_particles:
            l = x[b, axis] - x[a, axis]
            if periodic_length:
                if l > 0.5 * periodic_length:
                    l -= periodic_length
                elif l < -0.5 * periodic_length:
                    l += periodic_length
        else:
            l = (r[a] + gap[c]) * n[axis]
        q = np.floor((point - lo) / width)
        if 0 <= q < nstripes:
            sig[int(q)] += R[axis] * l
    return sig / (width * box_extent)
