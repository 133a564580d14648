"""Helpers for the GPU parity tests: run the same seeded input through the CUDA
library (via the C ABI binding) and through the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from oracle_adapter import system as oracle_system


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def gpu_system(wl, **kw):
    from paper_1104_3516_gb300 import cd
    return cd.CDSystem(wl, device="cuda:0", **kw)


def p_scale(P):
    return max(float(np.abs(P).max()) if P.size else 0.0, 1e-300)


def impulse_err(P_gpu, P_ref):
    """max |P_gpu - P_ref| / max(|P_ref|): the relative-to-scale error used by
    every impulse tolerance (open contacts have P = 0, so a per-contact
    relative error is meaningless there)."""
    if P_ref.size == 0:
        return 0.0
    return float(np.abs(P_gpu - P_ref).max()) / p_scale(P_ref)


def oracle_crit(gpu_crit):
    from paper_1104_3516_gb300 import cd
    return {cd.CD_CONV_NONE: O.CRIT_NONE, cd.CD_CONV_GLOBAL_REL: O.CRIT_GLOBAL_REL,
            cd.CD_CONV_GLOBAL_SQ: O.CRIT_GLOBAL_SQ, cd.CD_CONV_LOCAL: O.CRIT_LOCAL}[gpu_crit]


def run_pair(wl, steps=1, criterion=None, max_sweeps=None, alpha=None, precision=0, warm_start=1, f_ext=None,
             use_cells=True, max_contacts=None, tile_cells=0, **gpu_kw):
    """Steps the workload on the GPU and in the oracle (colour order, same
    seed); returns (gpu_system, oracle_system, gpu_stats, oracle_stats)."""
    from paper_1104_3516_gb300 import cd
    criterion = cd.CD_CONV_GLOBAL_REL if criterion is None else criterion
    ms = wl.max_sweeps if max_sweeps is None else max_sweeps
    al = wl.alpha if alpha is None else alpha
    g = gpu_system(wl, criterion=criterion, max_sweeps=ms, alpha=al, precision=precision, warm_start=warm_start,
                   f_ext=f_ext, max_contacts=max_contacts, tile_cells=tile_cells, **gpu_kw)
    o = oracle_system(wl, f_ext=f_ext, use_cells=use_cells, criterion=oracle_crit(criterion), max_sweeps=ms,
                      alpha=al, warm_start=warm_start, order=O.ORDER_COLOUR,
                      cap=max_contacts or max(64, 8 * wl.n), tile_cells=tile_cells,
                      parallel_p=gpu_kw.get("parallel_p", 0.0), domains=gpu_kw.get("domains", (1, 1, 1)))
    gst, ost = [], []
    for _ in range(steps):
        gst.append(g.step(1))
        ost.append(o.step())
    return g, o, gst, ost


needs_gpu = pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")
