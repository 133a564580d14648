"""The helpers the GPU parity tests use to classify and report impulses,
checked on hand-made impulses and on the oracle's own output (no GPU)."""
import numpy as np

from gpu_common import branch, near_switch, switch_report
from oracle_adapter import system
from paper_1104_3516_gb300 import workloads as W


def test_branch_of_hand_made_impulses():
    P = np.array([[0.0, 0.0], [1.0, 0.1], [1.0, 0.3], [2.0, -0.6]])
    assert branch(P, 0.3).tolist() == [0, 1, 2, 2]
    P3 = np.array([[1.0, 0.18, 0.24, 0.0], [1.0, 0.0, 0.1, 0.0]])   # |P_t| = 0.3, 0.1
    assert branch(P3, 0.3).tolist() == [2, 1]


def test_near_switch_counts_hand_made_impulses():
    mu = 0.3
    P = np.array([
        [1e-12, 0.0],                    # closed, 5e-13 of the scale above the opening switch
        [1.0, mu * (1.0 - 1e-11)],       # sticking 1e-11 below the cone
        [1.0, mu],                       # on the cone: the slide branch, not counted
        [2.0, 0.1],                      # far from both switches
        [0.0, 0.0],                      # open
    ])
    assert near_switch(P, mu) == (1, 1)
    rep = switch_report(P, P, mu)
    assert rep == {"contacts": 5, "near_open": 1, "near_slide": 1, "branch_differs": 0}
    Q = P.copy()
    Q[1, 1] = mu                         # one side slides where the other sticks
    assert switch_report(Q, P, mu)["branch_differs"] == 1


def test_oracle_pile_has_every_branch():
    """A settled pile after one step of 200 sweeps holds open, sticking and
    sliding contacts: the parity cases exercise all three branches."""
    wl = W.dense_biaxial_discs(n=600)
    s = system(wl, max_sweeps=200)
    s.step()
    b = branch(s.impulses, wl.mu)
    counts = np.bincount(b, minlength=3)
    assert counts.sum() == s.nc and np.all(counts > 0)
