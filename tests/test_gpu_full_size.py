"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (one persistent block per SM, max_contacts as
there): the 1e5-disc dense pile (FP64 and FP32), the 1e6-sphere gas, and the
512-packing batch.  The oracle follows the same colour order for a bounded
number of sweeps (it is single-threaded); contact sets and colours are
compared whole, impulses and velocities element by element.  For the batch,
the oracle solves sampled packings alone, which every packing of a batch must
reproduce exactly."""
import numpy as np
import pytest

import oracle as O
from gpu_common import impulse_err, needs_gpu
from oracle_adapter import system as osystem
from paper_1104_3516_gb300 import workloads as W
from test_gpu_batch import split

pytestmark = [pytest.mark.gpu, needs_gpu]


def compare(wl, sweeps, precision, max_contacts, tol):
    from paper_1104_3516_gb300 import cd
    g = cd.CDSystem(wl, device="cuda:0", precision=precision, criterion=cd.CD_CONV_NONE, max_sweeps=sweeps,
                    max_contacts=max_contacts, timing=1)
    st = g.step(1)
    o = osystem(wl, criterion=O.CRIT_NONE, max_sweeps=sweeps, order=O.ORDER_COLOUR, cap=max_contacts)
    o.step()
    c = g.contacts()
    assert st["last"]["n_contacts"] == o.nc
    assert np.array_equal(c["pairs"], o.contacts)
    assert np.array_equal(c["colour"], o.colour[: o.nc])
    if precision == cd.CD_FP64:
        assert np.array_equal(c["normal"], o.normal[: o.nc])
        assert np.array_equal(c["gap"], o.gap[: o.nc])
    assert impulse_err(c["impulse"], o.impulses) <= tol
    s = g.state()
    vs = max(float(np.abs(o.v).max()), 1e-300)
    assert float(np.abs(s["v"].reshape(-1) - o.v).max()) <= tol * vs
    return st


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4)])
def test_dense_pile_1e5_discs(precision, tol):
    """The 2D benchmark configuration: 100,000 discs, mu 0.3, periodic x,
    top wall, 20 sweeps of the first step."""
    wl = W.dense_biaxial_discs(n=100_000)
    st = compare(wl, 20, precision, 4 * wl.n, tol)
    assert st["last"]["n_colours"] >= 7 and st["last"]["n_contacts"] > 200_000


def test_sphere_gas_1e6():
    """The 3D configuration: 1,000,000 spheres, mu 0.5, rotations, 4 side
    walls and a floor; 3 sweeps of the first step."""
    wl = W.sphere_gas(n=1_000_000)
    st = compare(wl, 3, 0, 8 * wl.n, 1e-12)
    assert st["last"]["n_contacts"] > 500_000


def test_batch_512_packings_sampled():
    """The batched configuration: 512 gravity-settled piles (200-20,000 discs,
    mu U[0.1, 0.6]); 10 sweeps; packings 0, 17, 255 and 511 against the
    oracle alone, and every packing's contacts belong to it."""
    from paper_1104_3516_gb300 import cd
    batch = W.batched_settling(seed=1108, n_packings=512)
    n_total = sum(b.n for b in batch)
    g = cd.CDSystem(batch[0], device="cuda:0", batch=batch, criterion=cd.CD_CONV_NONE, max_sweeps=10,
                    max_contacts=6 * n_total)
    g.step(1)
    c = g.contacts()
    parts = split(c, g.offsets, len(batch), n_total)
    assert sum(len(p["pairs"]) for p in parts) == len(c["pairs"])
    s = g.state()
    for b in (0, 17, 255, 511):
        wl = batch[b]
        o = osystem(wl, criterion=O.CRIT_NONE, max_sweeps=10, order=O.ORDER_COLOUR, cap=6 * wl.n)
        o.step()
        assert np.array_equal(parts[b]["pairs"], o.contacts), b
        assert np.array_equal(parts[b]["colour"], o.colour[: o.nc]), b
        assert impulse_err(parts[b]["impulse"], o.impulses) <= 1e-12, b
        v = s["v"][g.offsets[b]: g.offsets[b + 1]].reshape(-1)
        assert float(np.abs(v - o.v).max()) <= 1e-12 * max(float(np.abs(o.v).max()), 1e-300), b
