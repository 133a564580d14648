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


def _noalloc(wl, max_contacts):
    import torch
    from paper_1104_3516_gb300 import cd
    dev = torch.device("cuda:0")
    dd = dict(dtype=torch.float64, device=dev)
    pos = torch.as_tensor(np.ascontiguousarray(wl.x).reshape(-1), **dd)
    rad = torch.as_tensor(wl.r, **dd)
    im = torch.as_tensor(wl.inv_m, **dd)
    iI = torch.as_tensor(wl.inv_I, **dd)
    pairs = torch.full((max_contacts, 2), -1, dtype=torch.int32, device=dev)
    normal = torch.zeros((max_contacts, 3), **dd)
    gap = torch.zeros(max_contacts, **dd)
    p = cd.make_params(wl)
    nc = cd.cd_detect_contacts_noalloc(p, wl.n, pos, rad, im, iI, max_contacts, pairs, normal, gap,
                                       torch.cuda.current_stream(dev).cuda_stream)
    return pairs[:nc].cpu().numpy(), normal[:nc].cpu().numpy(), gap[:nc].cpu().numpy()


def test_noalloc_detection_equals_workspace_detection_on_two_calls_in_a_row():
    cases = [W.dense_biaxial_discs(n=5000), W.sphere_gas(n=3000, floor=20.0, vsig=0.5)]
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
    with pytest.raises(cd.CDError) as e:
        _noalloc(wl, 10)
    assert e.value.status == cd.CD_ERR_CAPACITY
    big = W.settling_discs(n=16385)
    with pytest.raises(cd.CDError) as e:
        _noalloc(big, 1000)
    assert e.value.status == cd.CD_ERR_INVALID_ARG and "16384" in str(e.value)
