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


def branch(P, mu, rel=1e-12):
    """Branch of the single-contact solve (Fig. 2) each final impulse lies on:
    0 open (P_n = 0), 1 stick (|P_t| below mu P_n), 2 slide (|P_t| = mu P_n
    within `rel`)."""
    P = np.asarray(P, dtype=np.float64)
    pn = P[:, 0]
    pt = np.abs(P[:, 1]) if P.shape[1] == 2 else np.linalg.norm(P[:, 1:], axis=1)
    lim = mu * pn
    out = np.ones(pn.shape[0], dtype=np.int64)
    out[pt >= lim * (1.0 - rel)] = 2
    out[pn <= 0.0] = 0
    return out


def near_switch(P, mu, rel=1e-10):
    """Contacts whose impulse lies within `rel` (relative) of a switch of the
    single-contact solve, counted from the oracle's impulses: closed contacts
    with 0 < P_n <= rel max P_n (near the gap test's switch to open), and
    sticking contacts with mu P_n - |P_t| <= rel mu P_n (near the Coulomb
    switch to sliding).  Returns (near_open, near_slide)."""
    P = np.asarray(P, dtype=np.float64)
    if P.shape[0] == 0:
        return 0, 0
    pn = P[:, 0]
    pt = np.abs(P[:, 1]) if P.shape[1] == 2 else np.linalg.norm(P[:, 1:], axis=1)
    scale = max(float(pn.max()), 1e-300)
    lim = mu * pn
    near_open = int(np.count_nonzero((pn > 0.0) & (pn <= rel * scale)))
    slack = lim - pt
    # (a slack within 1e-12 of mu P_n is the slide branch itself, as in branch())
    near_slide = int(np.count_nonzero((pn > 0.0) & (slack > 1e-12 * lim) & (slack <= rel * lim)))
    return near_open, near_slide


def switch_report(P_gpu, P_ref, mu, branch_rel=1e-12):
    """What the sweep-by-sweep parity tests record beside the impulse bound
    (no contact is excluded from it): the contacts near a switch, and those
    whose final branch differs between the two sides (`branch_rel`: how close
    to the cone counts as sliding; an FP32 slide lies on the FP32 cone, ~1e-8
    from the FP64 one)."""
    no, ns = near_switch(P_ref, mu)
    differ = (int(np.count_nonzero(branch(P_gpu, mu, branch_rel) != branch(P_ref, mu, branch_rel)))
              if len(P_ref) else 0)
    return {"contacts": int(len(P_ref)), "near_open": no, "near_slide": ns, "branch_differs": differ}


def oracle_crit(gpu_crit):
    from paper_1104_3516_gb300 import cd
    return {cd.CD_CONV_NONE: O.CRIT_NONE, cd.CD_CONV_GLOBAL_REL: O.CRIT_GLOBAL_REL,
            cd.CD_CONV_GLOBAL_SQ: O.CRIT_GLOBAL_SQ, cd.CD_CONV_LOCAL: O.CRIT_LOCAL}[gpu_crit]


def run_pair(wl, steps=1, criterion=None, max_sweeps=None, alpha=None, precision=0, warm_start=1, f_ext=None,
             use_cells=True, max_contacts=None, **gpu_kw):
    """Steps the workload on the GPU and in the oracle (colour order, same
    seed); returns (gpu_system, oracle_system, gpu_stats, oracle_stats)."""
    from paper_1104_3516_gb300 import cd
    criterion = cd.CD_CONV_GLOBAL_REL if criterion is None else criterion
    ms = wl.max_sweeps if max_sweeps is None else max_sweeps
    al = wl.alpha if alpha is None else alpha
    g = gpu_system(wl, criterion=criterion, max_sweeps=ms, alpha=al, precision=precision, warm_start=warm_start,
                   f_ext=f_ext, max_contacts=max_contacts, **gpu_kw)
    o = oracle_system(wl, f_ext=f_ext, use_cells=use_cells, criterion=oracle_crit(criterion), max_sweeps=ms,
                      alpha=al, warm_start=warm_start, order=O.ORDER_COLOUR,
                      cap=max_contacts or max(64, 8 * wl.n),
                      parallel_p=gpu_kw.get("parallel_p", 0.0), parallel_redraw=gpu_kw.get("parallel_redraw", 0),
                      domains=gpu_kw.get("domains", (1, 1, 1)))
    gst, ost = [], []
    for _ in range(steps):
        gst.append(g.step(1))
        ost.append(o.step())
    return g, o, gst, ost


needs_gpu = pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")
