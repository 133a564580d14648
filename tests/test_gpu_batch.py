"""Batched packings: every packing of a batch must get exactly what the
oracle computes for that packing alone (contact set, colours, impulses sweep
by sweep, its own convergence stop), although all packings share the GPU's
colour phases."""
import numpy as np
import pytest

import oracle as O
from gpu_common import impulse_err, needs_gpu, oracle_crit
from oracle_adapter import system as osystem
from paper_1104_3516_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, needs_gpu]


def batch_2d():
    return [
        W.settling_discs(seed=21, n=300, mu=0.1, vsig=0.3),
        W.settling_discs(seed=22, n=1500, mu=0.55, vsig=0.2),
        W.dense_biaxial_discs(seed=23, n=800, wall_speed=0.3),
        W.dilute_discs(seed=24, n=400, width=30.0),
        W.settling_discs(seed=25, n=60, mu=0.3, vsig=0.5),
    ]


def batch_3d():
    return [W.sphere_gas(seed=31, n=400, floor=12.0, vsig=0.6, mu=0.2),
            W.sphere_gas(seed=32, n=900, floor=14.0, vsig=0.4, mu=0.6)]


def split(contacts, offsets, npk, n_total):
    """Per-packing contacts in local ids (walls n_b + k)."""
    out = []
    pairs = contacts["pairs"]
    for b in range(npk):
        lo, hi = offsets[b], offsets[b + 1]
        sel = (pairs[:, 0] >= lo) & (pairs[:, 0] < hi)
        pb = pairs[sel].astype(np.int64).copy()
        a_l = pb[:, 0] - lo
        wall = pb[:, 1] >= n_total
        b_l = np.where(wall, (hi - lo) + (pb[:, 1] - n_total) % 6, pb[:, 1] - lo)
        out.append({"pairs": np.stack([a_l, b_l], axis=1), "impulse": contacts["impulse"][sel],
                    "colour": contacts["colour"][sel]})
    return out


def run(batch, steps, **kw):
    from paper_1104_3516_gb300 import cd
    g = cd.CDSystem(batch[0], device="cuda:0", batch=batch, **kw)
    sts = [g.step(1) for _ in range(steps)]
    return g, sts


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("k", [1, 9])
def test_batch_sweep_by_sweep_equals_each_packing_alone(which, k):
    from paper_1104_3516_gb300 import cd
    batch = batch_2d() if which == "2d" else batch_3d()
    g, sts = run(batch, 1, criterion=cd.CD_CONV_NONE, max_sweeps=k)
    n_total = sum(b.n for b in batch)
    parts = split(g.contacts(), g.offsets, len(batch), n_total)
    s = g.state()
    for b, wl in enumerate(batch):
        o = osystem(wl, criterion=O.CRIT_NONE, max_sweeps=k, order=O.ORDER_COLOUR)
        o.step()
        assert np.array_equal(parts[b]["pairs"], o.contacts), b
        assert np.array_equal(parts[b]["colour"], o.colour[: o.nc]), b
        assert impulse_err(parts[b]["impulse"], o.impulses) <= 1e-12, b
        v = s["v"][g.offsets[b]: g.offsets[b + 1]].reshape(-1)
        assert float(np.abs(v - o.v).max()) <= 1e-12 * max(float(np.abs(o.v).max()), 1e-300), b


def test_batch_convergence_is_per_packing():
    from paper_1104_3516_gb300 import cd
    batch = batch_2d()
    g, sts = run(batch, 3, criterion=cd.CD_CONV_GLOBAL_REL, max_sweeps=400, alpha=1e-7)
    stats = g.packing_stats()
    n_total = sum(b.n for b in batch)
    parts = split(g.contacts(), g.offsets, len(batch), n_total)
    sweeps = []
    for b, wl in enumerate(batch):
        o = osystem(wl, criterion=O.CRIT_GLOBAL_REL, max_sweeps=400, alpha=1e-7, order=O.ORDER_COLOUR)
        for _ in range(3):
            ost = o.step()
        assert stats[b]["sweeps"] == ost["sweeps"], b
        assert stats[b]["converged"] == ost["converged"], b
        assert impulse_err(parts[b]["impulse"], o.impulses) <= 1e-12, b
        assert np.allclose(stats[b]["wall_pos"], o.wall_pos, rtol=0, atol=0), b
        # wall force = sum(P_n) / dt over the wall's contacts: within n_wall impulse bounds
        wf_o = np.array(ost["wall_force"])
        n_w = np.array([np.count_nonzero(o.contacts[:, 1] == wl.n + k) for k in range(6)])
        bound = n_w * 1e-12 * float(np.abs(o.impulses).max()) / wl.dt
        assert np.all(np.abs(np.array(stats[b]["wall_force"]) - wf_o) <= bound), b
        sweeps.append(stats[b]["sweeps"])
    assert len(set(sweeps)) > 1          # packings stop at different sweeps
    assert sts[-1]["last"]["sweeps"] == max(sweeps)
