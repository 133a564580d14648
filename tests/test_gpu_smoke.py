"""The package's smoke check (one small CD step on cuda:0 against the oracle)
runs as part of the GPU suite."""
import pytest

from gpu_common import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def test_smoke_entry_point():
    import __graft_entry__ as ge
    ge.smoke()
