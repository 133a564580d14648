"""Turns a Workload into oracle calls (test-side glue, argument marshalling)."""
import numpy as np

import oracle as O


def params(wl, **over):
    kw = dict(dim=wl.dim, dt=wl.dt, mu=wl.mu, gravity=wl.gravity, box_lo=wl.box_lo, box_hi=wl.box_hi,
              periodic=wl.periodic, wall_mask=wl.wall_mask, wall_vel=np.asarray(wl.wall_vel).reshape(18),
              delta=wl.delta, alpha=wl.alpha, max_sweeps=wl.max_sweeps, seed=wl.seed,
              wall_push=np.asarray(wl.wall_push).reshape(6), wall_mass=np.asarray(wl.wall_mass).reshape(6))
    kw.update(over)
    return O.make_params(**kw)


def system(wl, f_ext=None, use_cells=True, cap=None, **over):
    p = params(wl, **over)
    return O.OracleSystem(p, wl.x, wl.v, wl.w, wl.r, wl.inv_m, wl.inv_I, np.asarray(wl.wall_pos, dtype=np.float64),
                          f_ext=f_ext, cap=cap, use_cells=use_cells)
