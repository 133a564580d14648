"""Derivatives of Contact Dynamics time steps at fixed contact states (2D).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the test suite is the
only caller; the product path never imports it.

The paper differentiates nothing.  What this module fixes is the plain
definition of the derivative of one time step, the map

    (x, v, omega, mu)  ->  (x', v', omega')

of Eqs. 1-2 with the impulses of the iterative solve (Sec. 2.1, Fig. 2,
Eqs. 3-11), taken at a fixed contact set and fixed contact states.  Once the
iteration has converged, every contact is in one of three states, read off its
impulse the way the branches of Fig. 2 leave it:

* open: the gap test of Eq. 3 gave P = 0;
* sticking (Eq. 5): the gap closes and the contact points do not slip, i.e.
  the relative velocity after the step has u_n' = -g/dt and u_t' = 0;
* sliding (Eqs. 9-11): u_n' = -g/dt and P_t = s mu P_n with s = +-1.

With the states held fixed these are linear equations in the impulses.  Here
they are assembled densely: H maps body velocities (v_x, v_y, omega per
particle) to contact-frame relative velocities (u_n, u_t) per contact, W =
diag(inv_m, inv_m, inv_I); the retained rows (u_n and u_t of a sticking
contact, u_n of a sliding one) of H (v_free + W H^T P) + u_wall + g/dt = 0 are
solved with numpy's dense solver for the free impulse components, and the
step is completed with Eq. 2.  Every operation of that map is analytic in its
inputs (the branch decisions -- states, periodic images, the wrap of
positions -- are frozen or read from real parts), so evaluating it in complex
arithmetic gives directional derivatives by the complex step
Im f(theta + i h e) / h (Squire and Trapp, SIAM Review 40, 1998) with no
subtractive cancellation.  The tests pin this module against central finite
differences of the oracle's own iteration and against closed forms.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

OPEN, STICK, SLIDE = 0, 1, 2
# A contact whose normal impulse is at most this fraction of the step's
# largest one is taken as open: after an inelastic collision two bodies keep
# touching with zero normal velocity, and the iteration leaves rounding noise
# in P_n; the map has a kink there and the open side is the one linearised.
GRAZING = 1e-9


def classify(P, mu, grazing=GRAZING):
    """State of each 2D contact from its converged impulse (P_n, P_t): open
    when P_n is at most `grazing` times the largest P_n of the step, sliding
    when the tangential impulse sits on the Coulomb bound |P_t| == mu P_n (the
    product rounded once, as the sliding branch forms it), sticking
    otherwise.  Returns (state, s) with P_t = s mu P_n on sliding contacts."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 2)
    pn, pt = P[:, 0], P[:, 1]
    lim = mu * pn
    scale = float(pn.max()) if pn.size else 0.0
    state = np.where(pn <= grazing * scale, OPEN, np.where(np.abs(pt) == lim, SLIDE, STICK))
    sign = np.where(pt < 0.0, -1.0, 1.0)
    return state.astype(np.int64), sign


@dataclass
class Consts:
    """What stays fixed over a rollout: particles, box and parameters."""
    n: int
    r: np.ndarray
    inv_m: np.ndarray
    inv_I: np.ndarray        # already zero where rotations are frozen
    dt: float
    gravity: np.ndarray      # (2,)
    f_ext: np.ndarray | None
    lo: np.ndarray
    hi: np.ndarray
    periodic: np.ndarray
    wall_vel: np.ndarray     # (6, 3)


@dataclass
class StepRecord:
    """The frozen branch decisions of one time step."""
    pairs: np.ndarray        # (nc, 2), wall body ids n + k
    state: np.ndarray        # (nc,) OPEN / STICK / SLIDE
    sign: np.ndarray         # (nc,) s of a sliding contact
    shift: np.ndarray        # (nc, 2) periodic image added to x_b - x_a
    wall_pos: np.ndarray     # (6,) wall planes during the step
    P: np.ndarray            # (nc, 2) the iteration's impulses (for reporting)


def consts_of(sys) -> Consts:
    """Constants of an ``oracle.OracleSystem`` (2D)."""
    p = sys.p
    if int(p.dim) != 2:
        raise ValueError("the frozen-state map is written for 2D discs")
    iI = np.asarray(sys.inv_I, dtype=np.float64) * (1.0 if int(p.rotations) else 0.0)
    return Consts(n=sys.n, r=sys.r.copy(), inv_m=sys.inv_m.copy(), inv_I=iI, dt=float(p.dt),
                  gravity=np.array([p.gravity[0], p.gravity[1]]),
                  f_ext=None if sys.f_ext is None else sys.f_ext.reshape(-1, 2).copy(),
                  lo=np.array([p.box_lo[0], p.box_lo[1]]), hi=np.array([p.box_hi[0], p.box_hi[1]]),
                  periodic=np.array([int(p.periodic[0]), int(p.periodic[1])]),
                  wall_vel=np.array([p.wall_vel[k] for k in range(18)]).reshape(6, 3))


def _images(cs: Consts, x, pairs):
    """Periodic image of each particle pair, chosen as the detection does:
    the separation x_b - x_a is folded once when it exceeds half a period."""
    shift = np.zeros((len(pairs), 2))
    for c, (a, b) in enumerate(pairs):
        if b >= cs.n:
            continue
        for k in range(2):
            if not cs.periodic[k]:
                continue
            L = cs.hi[k] - cs.lo[k]
            d = x[b, k] - x[a, k]
            if d > 0.5 * L:
                shift[c, k] = -L
            elif d < -0.5 * L:
                shift[c, k] = L
    return shift


def record_rollout(sys, steps):
    """Steps the oracle system `steps` times and returns the frozen decisions
    of every step (the system is left after the last step)."""
    cs = consts_of(sys)
    recs = []
    for _ in range(steps):
        x = sys.x.reshape(-1, 2).copy()
        wall = sys.wall_pos.copy()
        sys.step()
        pairs = sys.contacts.astype(np.int64)
        P = sys.impulses
        state, sign = classify(P, float(sys.p.mu))
        recs.append(StepRecord(pairs=pairs, state=state, sign=sign, shift=_images(cs, x, pairs), wall_pos=wall,
                               P=P))
    return recs


def step_map(cs: Consts, rec: StepRecord, x, v, w, mu):
    """One time step at the frozen decisions of `rec`, in whatever number
    type the inputs carry (float or complex).  x, v: (n, 2); w: (n,).
    Returns (x', v', w', P)."""
    n, dt = cs.n, cs.dt
    x = np.asarray(x).reshape(n, 2)
    v = np.asarray(v).reshape(n, 2)
    w = np.asarray(w).reshape(n)
    ty = np.result_type(x, v, w, np.asarray(mu), np.float64)
    # Eq. 1: free flight with the explicit external forces
    acc = np.where(cs.inv_m[:, None] == 0.0, 0.0, cs.gravity[None, :])
    if cs.f_ext is not None:
        acc = acc + cs.f_ext * cs.inv_m[:, None]
    vf = v + acc * dt
    V = np.zeros(3 * n, dtype=ty)
    V[0::3], V[1::3], V[2::3] = vf[:, 0], vf[:, 1], w
    Winv = np.zeros(3 * n)
    Winv[0::3], Winv[1::3], Winv[2::3] = cs.inv_m, cs.inv_m, cs.inv_I

    nc = len(rec.pairs)
    H = np.zeros((2 * nc, 3 * n), dtype=ty)
    const = np.zeros(2 * nc, dtype=ty)      # wall velocity terms and g / dt on the normal rows
    for c, (a, b) in enumerate(rec.pairs):
        if b < n:
            d = x[b] - x[a] + rec.shift[c]
            dist = np.sqrt(d[0] * d[0] + d[1] * d[1])
            nv = d / dist
            g = dist - (cs.r[a] + cs.r[b])
        else:
            k = int(b - n)
            axis = k // 2
            nv = np.zeros(2, dtype=ty)
            nv[axis] = 1.0 if (k & 1) else -1.0
            g = (x[a, axis] - rec.wall_pos[k]) - cs.r[a] if (k & 1) == 0 else (rec.wall_pos[k] - x[a, axis]) - cs.r[a]
        t = np.array([-nv[1], nv[0]], dtype=ty)
        # u_n = n . (v_b - v_a);  u_t = t . (v_b - v_a) - r_a w_a - r_b w_b
        H[2 * c, 3 * a:3 * a + 2] = -nv
        H[2 * c + 1, 3 * a:3 * a + 2] = -t
        H[2 * c + 1, 3 * a + 2] = -cs.r[a]
        if b < n:
            H[2 * c, 3 * b:3 * b + 2] = nv
            H[2 * c + 1, 3 * b:3 * b + 2] = t
            H[2 * c + 1, 3 * b + 2] = -cs.r[b]
        else:
            vw = cs.wall_vel[int(b - n), :2]
            const[2 * c] += nv[0] * vw[0] + nv[1] * vw[1]
            const[2 * c + 1] += t[0] * vw[0] + t[1] * vw[1]
        const[2 * c] += g / dt

    rows, cols = [], []
    Phi = np.zeros((2 * nc, 2 * nc), dtype=ty)
    m = 0
    for c in range(nc):
        if rec.state[c] == STICK:
            rows += [2 * c, 2 * c + 1]
            Phi[2 * c, m] = 1.0
            Phi[2 * c + 1, m + 1] = 1.0
            m += 2
        elif rec.state[c] == SLIDE:
            rows.append(2 * c)
            Phi[2 * c, m] = 1.0
            Phi[2 * c + 1, m] = rec.sign[c] * mu
            m += 1
    Phi = Phi[:, :m]
    P = np.zeros(2 * nc, dtype=ty)
    if m > 0:
        A = (H * Winv[None, :]) @ H.T
        K = (A @ Phi)[rows, :]
        rhs = -(H @ V + const)[rows]
        p = np.linalg.solve(K, rhs)
        P = Phi @ p
    Vn = V + Winv * (H.T @ P)
    vn = np.stack([Vn[0::3], Vn[1::3]], axis=1)
    wn = Vn[2::3]
    # Eq. 2, with the periodic wrap decided on the real part
    xn = x + vn * dt
    for k in range(2):
        if cs.periodic[k]:
            L = cs.hi[k] - cs.lo[k]
            xr = xn[:, k].real
            xn[:, k] = xn[:, k] - L * (xr >= cs.hi[k]) + L * (xr < cs.lo[k])
    return xn, vn, wn, P.reshape(nc, 2)


def rollout_map(cs: Consts, recs, x0, v0, w0, mu, with_forces=False):
    """The frozen-state map over all recorded steps; with_forces also
    returns the wall forces of the last step (sum of the normal impulses on
    wall k over dt, 6 values)."""
    x, v, w = np.asarray(x0).reshape(cs.n, 2), np.asarray(v0).reshape(cs.n, 2), np.asarray(w0).reshape(cs.n)
    P = None
    for rec in recs:
        x, v, w, P = step_map(cs, rec, x, v, w, mu)
    if not with_forces:
        return x, v, w
    F = np.zeros(6, dtype=np.result_type(x, v, w, np.float64))
    if recs:
        for c, (a, b) in enumerate(recs[-1].pairs):
            if b >= cs.n:
                F[int(b - cs.n)] += P[c, 0] / cs.dt
    return x, v, w, F


def directional_derivatives(cs: Consts, recs, x0, v0, w0, mu, weights, directions, h=1e-30, wall_weights=None):
    """d/de of L = <c_x, x_T> + <c_v, v_T> + <c_w, w_T> (+ <c_F, F_T> with
    F_T the wall forces of the last step) along each direction
    e = (e_x, e_v, e_w, e_mu) by the complex step.  `weights` = (c_x, c_v,
    c_w); `wall_weights` = c_F (6 values) or None; `directions` a list of
    4-tuples."""
    cx, cv, cw = (np.asarray(a, dtype=np.float64) for a in weights)
    cF = None if wall_weights is None else np.asarray(wall_weights, dtype=np.float64).reshape(6)
    out = []
    for ex, ev, ew, emu in directions:
        x, v, w, F = rollout_map(cs, recs, np.asarray(x0).reshape(cs.n, 2) + 1j * h * np.asarray(ex).reshape(cs.n, 2),
                                 np.asarray(v0).reshape(cs.n, 2) + 1j * h * np.asarray(ev).reshape(cs.n, 2),
                                 np.asarray(w0).reshape(cs.n) + 1j * h * np.asarray(ew).reshape(cs.n),
                                 mu + 1j * h * emu, with_forces=True)
        L = np.sum(cx.reshape(cs.n, 2) * x) + np.sum(cv.reshape(cs.n, 2) * v) + np.sum(cw.reshape(cs.n) * w)
        if cF is not None:
            L = L + np.sum(cF * F)
        out.append(L.imag / h)
    return np.array(out)


def jacobian_condition(cs: Consts, rec: StepRecord, x, mu):
    """2-norm condition number of the retained-row matrix of one step (the
    conditioning of the frozen-state system; infinite when hyperstatic)."""
    n = cs.n
    xr = np.asarray(x, dtype=np.float64).reshape(n, 2)
    # assemble with zero velocities: only the matrix is wanted
    nc = len(rec.pairs)
    H = np.zeros((2 * nc, 3 * n))
    for c, (a, b) in enumerate(rec.pairs):
        if b < n:
            d = xr[b] - xr[a] + rec.shift[c]
            nv = d / np.sqrt(d @ d)
        else:
            k = int(b - n)
            nv = np.zeros(2)
            nv[k // 2] = 1.0 if (k & 1) else -1.0
        t = np.array([-nv[1], nv[0]])
        H[2 * c, 3 * a:3 * a + 2] = -nv
        H[2 * c + 1, 3 * a:3 * a + 2] = -t
        H[2 * c + 1, 3 * a + 2] = -cs.r[a]
        if b < n:
            H[2 * c, 3 * b:3 * b + 2] = nv
            H[2 * c + 1, 3 * b:3 * b + 2] = t
            H[2 * c + 1, 3 * b + 2] = -cs.r[b]
    Winv = np.zeros(3 * n)
    Winv[0::3], Winv[1::3], Winv[2::3] = cs.inv_m, cs.inv_m, cs.inv_I
    rows, m = [], 0
    Phi = np.zeros((2 * nc, 2 * nc))
    for c in range(nc):
        if rec.state[c] == STICK:
            rows += [2 * c, 2 * c + 1]
            Phi[2 * c, m] = 1.0
            Phi[2 * c + 1, m + 1] = 1.0
            m += 2
        elif rec.state[c] == SLIDE:
            rows.append(2 * c)
            Phi[2 * c, m] = 1.0
            Phi[2 * c + 1, m] = rec.sign[c] * mu
            m += 1
    if m == 0:
        return 1.0
    K = ((H * Winv[None, :]) @ H.T @ Phi[:, :m])[rows, :]
    return float(np.linalg.cond(K))
