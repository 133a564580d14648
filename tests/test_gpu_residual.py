"""The convergence tests of Sec. 2.1 on the CUDA path (through the C ABI)
against values derived by hand from their definitions: the same closed forms
that pin the oracle's residual (tests/test_oracle_residual.py), here without
the oracle in between."""
import math

import numpy as np
import pytest

import oracle_cases as cases
from gpu_common import gpu_system, needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]

G, DT = cases.G, cases.DT


def _stack_ravg(k):
    # two discs stacked on the floor, B (disc-disc) before A (floor), from zero:
    # R^k = (A_k + B_k) / 2 = (3 - 2^(2-k)) / 2 in units of m g dt
    return 0.0 if k == 0 else (3.0 - 2.0 ** (2 - k)) / 2.0


def _stack_ratio(k):
    return 1.0 if k == 1 else 1.0 / (3.0 * (2.0 ** (k - 1) - 1.0))


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_gpu_stack_residual_sequence_closed_form(k):
    from paper_1104_3516_gb300 import cd
    wl = cases.stack2()
    unit = G * DT / wl.inv_m[0]
    g = gpu_system(wl, criterion=cd.CD_CONV_NONE, max_sweeps=k, warm_start=0)
    st = g.step(1)["last"]
    assert g.contacts()["pairs"].tolist() == [[0, 1], [0, 4]]
    assert st["sweeps"] == k
    assert st["r_avg"] == pytest.approx(_stack_ravg(k) * unit, rel=1e-13)
    assert st["residual"] == pytest.approx(_stack_ratio(k), rel=1e-10)


@pytest.mark.parametrize("crit,alpha,expect", [("rel", 1e-6, 20), ("rel", 1e-3, 10), ("sq", 1e-6, 10),
                                               ("sq", 1e-10, 17)])
def test_gpu_stack_stops_at_the_closed_form_sweep(crit, alpha, expect):
    from paper_1104_3516_gb300 import cd
    c = cd.CD_CONV_GLOBAL_REL if crit == "rel" else cd.CD_CONV_GLOBAL_SQ
    g = gpu_system(cases.stack2(), criterion=c, alpha=alpha, max_sweeps=1000, warm_start=0)
    st = g.step(1)["last"]
    assert st["converged"] and st["sweeps"] == expect
    power = 2 if crit == "sq" else 1
    assert st["residual"] == pytest.approx(_stack_ratio(expect) ** power, rel=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_gpu_resting_particle_residual_is_one_then_stops(dim):
    from paper_1104_3516_gb300 import cd
    wl = cases.resting_disc(dim=dim)
    mgdt = G * DT / wl.inv_m[0]
    st1 = gpu_system(wl, criterion=cd.CD_CONV_NONE, max_sweeps=1).step(1)["last"]
    assert st1["residual"] == 1.0
    assert st1["r_avg"] == pytest.approx(mgdt, rel=1e-15)
    g = gpu_system(wl, criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-6, max_sweeps=100)
    a = g.step(1)["last"]
    b = g.step(1)["last"]   # warm start from m g dt: R^0 = R^1, one sweep
    assert a["sweeps"] == 2 and a["converged"]
    assert b["sweeps"] == 1 and b["converged"] and b["residual"] <= 1e-15


@pytest.mark.parametrize("dim,azimuth", [(2, 0.0), (3, 0.7)])
def test_gpu_residual_averages_the_impulse_magnitude(dim, azimuth):
    from paper_1104_3516_gb300 import cd
    wl = cases.incline(math.atan(0.2), mu=0.4, dim=dim, azimuth=azimuth)
    st = gpu_system(wl, criterion=cd.CD_CONV_NONE, max_sweeps=1).step(1)["last"]
    assert st["r_avg"] == pytest.approx(G * DT / wl.inv_m[0], rel=1e-14)


def _row_gpu(radii, warm, max_sweeps=1, alpha=1e-6):
    """Discs resting on the floor, floor contacts only, warm impulse m g dt
    where `warm`, else zero; one local-test solve of the given contact list
    from the free velocities."""
    from paper_1104_3516_gb300 import cd
    wl = cases.floor_row(radii)
    wl.v = wl.v.copy()
    wl.v[:, 1] -= G * DT
    pairs = np.array([[i, wl.n + 2] for i in range(wl.n)], dtype=np.int32)
    P0 = np.zeros((wl.n, 2))
    P0[:, 0] = np.where(warm, G * DT / wl.inv_m, 0.0)
    g = gpu_system(wl, criterion=cd.CD_CONV_LOCAL, alpha=alpha, max_sweeps=max_sweeps)
    g.set_contacts(pairs, P0)
    return g.solve_contacts()


def test_gpu_local_test_ninety_percent_rule():
    a = _row_gpu([1.0] * 9 + [0.02], [True] * 9 + [False])
    assert a["converged"] and a["sweeps"] == 1 and a["residual"] == 0.1
    b = _row_gpu([1.0] * 8 + [0.02] * 2, [True] * 8 + [False] * 2)
    assert not b["converged"] and b["residual"] == 0.2
    c = _row_gpu([1.0] * 8 + [0.02] * 2, [True] * 8 + [False] * 2, max_sweeps=10)
    assert c["converged"] and c["sweeps"] == 2
    d = _row_gpu([1.0] * 20, [True] * 19 + [False])
    assert not d["converged"] and d["sweeps"] == 1


def test_gpu_nan_impulses_never_pass_the_global_tests():
    """A NaN starting impulse (given through cd_set_contacts) spreads through
    the velocities: every R_avg is NaN and must not pass tests (II), which
    count only 0/0 (both averages zero) as converged; the solve runs to the
    cap with a NaN residual."""
    from paper_1104_3516_gb300 import cd
    wl = cases.floor_row([1.0] * 4)
    wl.v = wl.v.copy()
    wl.v[:, 1] -= G * DT
    pairs = np.array([[i, wl.n + 2] for i in range(wl.n)], dtype=np.int32)
    P0 = np.zeros((wl.n, 2))
    P0[1, 0] = np.nan
    for crit in (cd.CD_CONV_GLOBAL_REL, cd.CD_CONV_GLOBAL_SQ):
        g = gpu_system(wl, criterion=crit, alpha=1e-6, max_sweeps=50)
        g.set_contacts(pairs, P0)
        st = g.solve_contacts()
        assert not st["converged"] and st["sweeps"] == 50
        assert math.isnan(st["residual"])
