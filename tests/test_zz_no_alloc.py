"""The allocation-free detection entry point against the regular one.

cd_detect_contacts_noalloc serves callers that cannot call cudaMalloc (their
device memory is owned by someone else); its scratch is a fixed device array
inside the library.  Its output must equal cd_detect_contacts' (bit-exact, the
detection bar), including on a second call in a row that reuses the shared
scratch left by the first.  Collected last (file name) so a failure here does
not hide any other result.
"""
import numpy as np
import pytest

from gpu_common import gpu_system, needs_gpu
from paper_1104_3516_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, needs_gpu]


def _noalloc(wl, max_contacts, buffers=None, outputs=True):
    """One call on the workload; `buffers` (pairs, normal, gap) lets a test
    keep the output tensors, `outputs=False` passes none (size query)."""
    import torch
    from paper_1104_3516_gb300 import cd
    dev = torch.device("cuda:0")
    dd = dict(dtype=torch.float64, device=dev)
    pos = torch.as_tensor(np.ascontiguousarray(wl.x).reshape(-1), **dd)
    rad = torch.as_tensor(wl.r, **dd)
    im = torch.as_tensor(wl.inv_m, **dd)
    iI = torch.as_tensor(wl.inv_I, **dd)
    if buffers is None:
        buffers = (torch.full((max_contacts, 2), -1, dtype=torch.int32, device=dev),
                   torch.zeros((max_contacts, 3), **dd), torch.zeros(max_contacts, **dd))
    pairs, normal, gap = buffers if outputs else (None, None, None)
    p = cd.make_params(wl)
    nc = cd.cd_detect_contacts_noalloc(p, wl.n, pos, rad, im, iI, max_contacts, pairs, normal, gap,
                                       torch.cuda.current_stream(dev).cuda_stream)
    if not outputs:
        return nc
    return pairs[:nc].cpu().numpy(), normal[:nc].cpu().numpy(), gap[:nc].cpu().numpy()


def _periodic_gas_3d():
    """A 3D gas periodic along x and y, with the floor only."""
    wl = W.sphere_gas(n=3000, floor=20.0, vsig=0.5)
    wl.periodic = (1, 1, 0)
    wl.wall_mask = 0b010000
    return wl


def test_noalloc_detection_equals_workspace_detection_on_two_calls_in_a_row():
    cases = [W.dense_biaxial_discs(n=5000), W.sphere_gas(n=3000, floor=20.0, vsig=0.5), _periodic_gas_3d()]
    for wl in cases:
        g = gpu_system(wl)
        g.detect_contacts()
        ref = g.contacts()
        for _ in range(2):
            pairs, normal, gap = _noalloc(wl, 65536)
            assert np.array_equal(pairs, ref["pairs"])
            assert np.array_equal(normal, ref["normal"])
            assert np.array_equal(gap, ref["gap"])


def test_noalloc_limits_are_reported():
    from paper_1104_3516_gb300 import cd
    wl = W.dense_biaxial_discs(n=2000)
    with pytest.raises(cd.CDError) as e:
        _noalloc(wl, 65537)
    assert e.value.status == cd.CD_ERR_INVALID_ARG and "65536" in str(e.value)
    g = gpu_system(wl)
    needed = g.detect_contacts()
    import torch
    dev = torch.device("cuda:0")
    bufs = (torch.full((10, 2), -1, dtype=torch.int32, device=dev),
            torch.zeros((10, 3), dtype=torch.float64, device=dev), torch.zeros(10, dtype=torch.float64, device=dev))
    big_pairs = torch.full((20, 2), -1, dtype=torch.int32, device=dev)
    bufs_in_big = (big_pairs[:10], bufs[1], bufs[2])
    with pytest.raises(cd.CDError) as e:
        _noalloc(wl, 10, buffers=bufs_in_big)
    assert e.value.status == cd.CD_ERR_CAPACITY
    assert e.value.needed == needed
    assert torch.all(big_pairs[10:] == -1)        # nothing written past max_contacts
    # a size query: no outputs, max_contacts 0
    with pytest.raises(cd.CDError) as e:
        _noalloc(wl, 0, outputs=False)
    assert e.value.status == cd.CD_ERR_CAPACITY and e.value.needed == needed
    # undersized or mistyped outputs are refused before the call
    with pytest.raises(ValueError):
        _noalloc(wl, 10, buffers=(bufs[0][:5], bufs[1], bufs[2]))
    with pytest.raises(ValueError):
        _noalloc(wl, 10, buffers=(bufs[0].to(torch.int64), bufs[1], bufs[2]))
    big = W.settling_discs(n=16385)
    with pytest.raises(cd.CDError) as e:
        _noalloc(big, 1000)
    assert e.value.status == cd.CD_ERR_INVALID_ARG and "16384" in str(e.value)
