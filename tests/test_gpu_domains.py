"""The domain-wise update of the parallel algorithm (Sec. 3.1) on the GPU
against the oracle: a contact belongs to the slab of the middle of its gap;
every domain sweeps its own contacts in the colour order while the other
domains' contacts keep the impulses of the previous sweep.  Closed form on a
two-disc stack, sweep-by-sweep parity (FP64 1e-12, FP32 1e-4) on dense and
settling packings and a 3D gas, stopping sweeps, warm-started trajectories,
the chain of Fig. 13(a), and the configurations it refuses."""
import math

import numpy as np
import pytest

import oracle as O
import oracle_cases as cases
from gpu_common import gpu_system, impulse_err, needs_gpu, run_pair
from paper_1104_3516_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, needs_gpu]

FP64_TOL = 1e-12
FP32_TOL = 1e-4


def check_state(g, o, tol):
    s = g.state()
    vs = max(float(np.abs(o.v).max()), 1e-300)
    assert float(np.abs(s["v"].reshape(-1) - o.v).max()) <= tol * vs
    ws = max(float(np.abs(o.w).max()), 1e-300)
    assert float(np.abs(s["w"].reshape(-1) - o.w).max()) <= tol * ws


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_stack_split_between_domains_is_a_jacobi_pair(k):
    """Floor contact A and disc-disc contact B in different slabs: A_k =
    2 - 2^(1 - ceil(k/2)), B_k = 1 - 2^(-floor(k/2)) in units of m g dt."""
    from paper_1104_3516_gb300 import cd
    wl = cases.stack2()
    g, o, gst, ost = run_pair(wl, criterion=cd.CD_CONV_NONE, max_sweeps=k, warm_start=0, domains=(1, 3, 1))
    unit = cases.G * cases.DT / wl.inv_m[0]
    c = g.contacts()
    assert c["pairs"].tolist() == [[0, 1], [0, 4]]
    A, B = 2.0 - 2.0 ** (1 - math.ceil(k / 2)), 1.0 - 2.0 ** (-(k // 2))
    assert c["impulse"][1, 0] == pytest.approx(A * unit, rel=1e-12)
    assert c["impulse"][0, 0] == pytest.approx(B * unit, rel=1e-12, abs=1e-18)
    assert impulse_err(c["impulse"], o.impulses) <= FP64_TOL


CASES = {
    "dense_deposit": (W.dense_biaxial_discs(n=5000), [(4, 2, 1), (9, 5, 1)]),
    "settling_discs": (W.settling_discs(n=3000, vsig=0.3), [(3, 3, 1)]),
    "sphere_gas": (W.sphere_gas(n=3000, floor=20.0, vsig=0.5), [(2, 2, 2), (3, 1, 4)]),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("k", [1, 2, 7, 40])
def test_domains_fp64_sweep_by_sweep(name, k):
    from paper_1104_3516_gb300 import cd
    wl, doms = CASES[name]
    for dom in doms:
        g, o, gst, ost = run_pair(wl, criterion=cd.CD_CONV_NONE, max_sweeps=k, domains=dom)
        c = g.contacts()
        assert np.array_equal(c["pairs"], o.contacts)
        assert gst[0]["last"]["sweeps"] == k == ost[0]["sweeps"]
        assert impulse_err(c["impulse"], o.impulses) <= FP64_TOL, dom
        check_state(g, o, FP64_TOL)


@pytest.mark.parametrize("name", ["dense_deposit", "sphere_gas"])
def test_domains_fp32_sweep_by_sweep(name):
    from paper_1104_3516_gb300 import cd
    wl, doms = CASES[name]
    g, o, gst, ost = run_pair(wl, criterion=cd.CD_CONV_NONE, max_sweeps=40, precision=cd.CD_FP32, domains=doms[0])
    assert impulse_err(g.contacts()["impulse"], o.impulses) <= FP32_TOL


def test_domains_stop_at_the_oracle_sweep_over_warm_started_steps():
    from paper_1104_3516_gb300 import cd
    wl, _ = CASES["dense_deposit"]
    g, o, gst, ost = run_pair(wl, steps=3, criterion=cd.CD_CONV_GLOBAL_REL, max_sweeps=1000, alpha=1e-6,
                              domains=(5, 3, 1))
    for a, b in zip(gst, ost):
        assert a["last"]["sweeps"] == b["sweeps"]
    assert impulse_err(g.contacts()["impulse"], o.impulses) <= 1e-12
    check_state(g, o, 1e-12)


def test_domains_sharing_no_particle_equal_gauss_seidel():
    """Slabs that cut no particle's contacts leave the Gauss-Seidel sweep
    unchanged."""
    from paper_1104_3516_gb300 import cd
    wl = cases.two_columns(n=4)
    kw = dict(criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-13, max_sweeps=5000)
    a = gpu_system(wl, **kw)
    sa = a.step(1)
    b = gpu_system(wl, domains=(2, 1, 1), **kw)
    sb = b.step(1)
    assert sa["last"]["sweeps"] == sb["last"]["sweeps"]
    assert impulse_err(b.contacts()["impulse"], a.contacts()["impulse"]) <= 1e-13


def test_chain_needs_more_sweeps_with_more_domains():
    """Fig. 13(a, b): the chain pressed against a wall, forces from zero, in
    1, 4 and 12 domains; the GPU stops at the oracle's sweep (colour order)
    and the sweeps grow with the number of domain boundaries."""
    from paper_1104_3516_gb300 import cd
    n = 24
    sweeps = {}
    for Np in (1, 4, 12):
        wl, f = cases.chain_slabs(n=n, force=1.0)
        g, o, gst, ost = run_pair(wl, f_ext=f, criterion=cd.CD_CONV_GLOBAL_SQ, alpha=1e-12, max_sweeps=200000,
                                  warm_start=0, domains=(Np, 1, 1))
        assert gst[0]["last"]["sweeps"] == ost[0]["sweeps"]
        assert gst[0]["last"]["converged"]
        assert impulse_err(g.contacts()["impulse"], o.impulses) <= 1e-12
        sweeps[Np] = ost[0]["sweeps"]
    assert sweeps[1] < sweeps[4] < sweeps[12]


@pytest.mark.parametrize("kw", [dict(parallel_p=0.3), dict(tape_steps=2)])
def test_domains_refuse_other_schedules(kw):
    from paper_1104_3516_gb300 import cd
    wl, _ = CASES["dense_deposit"]
    with pytest.raises(cd.CDError):
        gpu_system(wl, domains=(2, 2, 1), **kw)


def test_domains_refuse_batches_and_force_controlled_walls():
    from paper_1104_3516_gb300 import cd
    batch = W.batched_settling(seed=5, n_packings=2, nmin=200, nmax=300)
    with pytest.raises(cd.CDError):
        gpu_system(batch[0], batch=batch, domains=(2, 1, 1))
    with pytest.raises(cd.CDError):
        gpu_system(cases.pressed_column(n=3), domains=(1, 2, 1))
    with pytest.raises(cd.CDError):
        gpu_system(cases.column(n=3), domains=(-1, 1, 1))
