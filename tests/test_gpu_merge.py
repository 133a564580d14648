"""Merging of the last colours into one sweep phase (params.merge_last_colour):
the contacts of the M last colours (M = 3, else 2) form chains through shared
particles, each chain goes whole to one block, which updates the chains'
contacts colour by colour with a block barrier between them.  The update
order is the colour order, so impulses and states must be bit-identical to
the run without merging and to the two-colour merge (FP64 and FP32, 2D and
3D, at the benchmark's full size), the oracle must still match sweep by
sweep, and the merge must actually happen where the last class is small."""
import numpy as np
import pytest

import oracle as O
from gpu_common import gpu_system, impulse_err, needs_gpu, run_pair
from paper_1104_3516_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, needs_gpu]

CASES = {
    "dense_deposit": W.dense_biaxial_discs(n=5000),
    "settling_discs": W.settling_discs(n=3000, vsig=0.3),
    "sphere_gas": W.sphere_gas(n=3000, floor=20.0, vsig=0.5),
}


def pair(wl, steps=1, merge=1, **kw):
    a = gpu_system(wl, merge_last_colour=0, **kw)
    b = gpu_system(wl, merge_last_colour=merge, **kw)
    sa = [a.step(1) for _ in range(steps)]
    sb = [b.step(1) for _ in range(steps)]
    return a, b, sa, sb


def identical(a, b):
    ca, cb = a.contacts(), b.contacts()
    assert np.array_equal(ca["pairs"], cb["pairs"])
    assert np.array_equal(ca["colour"], cb["colour"])
    assert np.array_equal(ca["impulse"], cb["impulse"])
    xa, xb = a.state(), b.state()
    for k in ("x", "v", "w"):
        assert np.array_equal(xa[k], xb[k]), k


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("merge", [1, 2])
def test_merged_phase_is_bit_identical(name, precision, merge):
    from paper_1104_3516_gb300 import cd
    a, b, sa, sb = pair(CASES[name], steps=2, merge=merge, criterion=cd.CD_CONV_NONE, max_sweeps=40,
                        precision=precision)
    identical(a, b)
    for x, y in zip(sa, sb):
        K = y["last"]["n_colours"]
        assert x["last"]["n_phases"] == x["last"]["n_colours"]
        assert y["last"]["n_phases"] in ((K, K - 1, K - 2) if merge == 1 else (K, K - 1))


def test_merge_happens_on_the_dense_deposit():
    """Three colours merge where the last class is small; merge_last_colour 2
    keeps to two.  The chains of both are checked by the bit-identity above."""
    from paper_1104_3516_gb300 import cd
    g = gpu_system(CASES["dense_deposit"], merge_last_colour=1, criterion=cd.CD_CONV_NONE, max_sweeps=5)
    st = g.step(1)
    c = g.contacts()
    cnt = np.bincount(c["colour"])
    assert 4 * cnt[-1] <= cnt[-3]
    assert st["last"]["n_phases"] == st["last"]["n_colours"] - 2
    g2 = gpu_system(CASES["dense_deposit"], merge_last_colour=2, criterion=cd.CD_CONV_NONE, max_sweeps=5)
    st2 = g2.step(1)
    assert st2["last"]["n_phases"] == st2["last"]["n_colours"] - 1
    assert np.array_equal(g.contacts()["impulse"], g2.contacts()["impulse"])


def test_merged_phase_matches_the_oracle_sweep_by_sweep():
    from paper_1104_3516_gb300 import cd
    wl = CASES["dense_deposit"]
    for k in (1, 7, 40):
        g, o, gst, ost = run_pair(wl, criterion=cd.CD_CONV_NONE, max_sweeps=k, merge_last_colour=1)
        assert gst[0]["last"]["n_phases"] == gst[0]["last"]["n_colours"] - 2
        assert impulse_err(g.contacts()["impulse"], o.impulses) <= 1e-12
        s = g.state()
        vs = max(float(np.abs(o.v).max()), 1e-300)
        assert float(np.abs(s["v"].reshape(-1) - o.v).max()) <= 1e-12 * vs


def test_merged_phase_stops_at_the_same_sweep():
    from paper_1104_3516_gb300 import cd
    a, b, sa, sb = pair(CASES["dense_deposit"], steps=3, criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-6,
                        max_sweeps=1000)
    for x, y in zip(sa, sb):
        assert x["last"]["sweeps"] == y["last"]["sweeps"]
    assert impulse_err(b.contacts()["impulse"], a.contacts()["impulse"]) <= 1e-13


def test_merged_phase_full_size_pile():
    """The 1e5-disc pile of the benchmark: 20 sweeps, merged and not."""
    from paper_1104_3516_gb300 import cd
    wl = W.dense_biaxial_discs(n=100_000)
    a, b, sa, sb = pair(wl, criterion=cd.CD_CONV_NONE, max_sweeps=20, max_contacts=4 * wl.n)
    identical(a, b)
    assert sb[0]["last"]["n_phases"] == sb[0]["last"]["n_colours"] - 2


def test_merge_parameter_is_checked():
    from paper_1104_3516_gb300 import cd
    for bad in (-1, 5):
        with pytest.raises(cd.CDError):
            gpu_system(CASES["dense_deposit"], merge_last_colour=bad)


@pytest.mark.parametrize("cap, merged_later", [(5, False), (80, True)])
def test_automatic_merge_follows_the_previous_solve(cap, merged_later):
    """merge_last_colour 4 merges on a system's first step (no solve yet)
    and afterwards only if the previous solve took at least 64 sweeps; the
    bits equal the unmerged run's either way."""
    from paper_1104_3516_gb300 import cd
    a, b, sa, sb = pair(CASES["dense_deposit"], steps=3, merge=4, criterion=cd.CD_CONV_NONE, max_sweeps=cap)
    identical(a, b)
    k = [s["last"]["n_colours"] for s in sb]
    assert sb[0]["last"]["n_phases"] == k[0] - 2
    for s, kk in zip(sb[1:], k[1:]):
        assert s["last"]["n_phases"] == (kk - 2 if merged_later else kk)


@pytest.mark.parametrize("kw", [dict(parallel_p=0.3), dict(domains=(2, 2, 1))])
def test_merge_is_ignored_by_other_schedules(kw):
    from paper_1104_3516_gb300 import cd
    g = gpu_system(CASES["dense_deposit"], merge_last_colour=1, criterion=cd.CD_CONV_NONE, max_sweeps=3, **kw)
    st = g.step(1)
    assert st["last"]["n_phases"] == st["last"]["n_colours"]
