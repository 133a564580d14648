"""Block shapes of the persistent sweep grid keep the Gauss-Seidel order, so
every shape the autotuner may pick gives the same impulses; the autotuner
returns one of its candidates with a timing for each."""
import numpy as np
import pytest

from gpu_common import needs_gpu
from paper_1104_3516_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_block_shapes_give_identical_impulses_and_the_tuner_picks_one():
    from paper_1104_3516_gb300 import autotune, cd
    wl = W.dense_biaxial_discs(seed=5, n=3000, wall_speed=0.3)
    ref = None
    for t, b in autotune.BLOCK_SHAPES:
        g = cd.CDSystem(wl, device="cuda:0", criterion=cd.CD_CONV_NONE, max_sweeps=25, sweep_threads=t,
                        sweep_blocks_per_sm=b)
        g.step(2)
        P = g.contacts()["impulse"]
        v = g.state()["v"]
        if ref is None:
            ref = (P, v)
        else:
            assert np.array_equal(P, ref[0]) and np.array_equal(v, ref[1]), (t, b)
    best, table = autotune.tune(wl, sweeps=10, steps=1)
    assert best in [c for c, _ in table] and len(table) >= 5
    assert all(ms > 0 for _, ms in table)
    with pytest.raises(cd.CDError):
        cd.CDSystem(wl, device="cuda:0", sweep_threads=384)
