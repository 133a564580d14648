"""Autotuner for the persistent sweep grid.

Times short solves of the caller's own system under candidate launch
configurations and returns the fastest: the block shape of the cooperative
sweep grid (threads per block x blocks per SM).  Every candidate keeps the
Gauss-Seidel order, so choosing among them changes only the speed.

Everything runs through the CUDA library (``cd.CDSystem``); each trial is
timed with the CUDA events the library records around the sweep kernel.
"""
from __future__ import annotations

from . import cd

BLOCK_SHAPES = [(512, 1), (256, 2), (256, 1), (128, 4), (128, 2)]
ORDER_KEEPING = [dict(sweep_threads=t, sweep_blocks_per_sm=b) for t, b in BLOCK_SHAPES]


def tune(wl, batch=None, precision=cd.CD_FP64, sweeps=40, steps=2, device="cuda", candidates=None,
         max_contacts=None):
    """Returns (best parameter dict, table of (parameters, ms per sweep)).

    Each candidate system is built over the workload (or the batch), stepped
    once untimed, then `steps` steps of exactly `sweeps` sweeps are timed; the
    figure is the sweep kernel's device time per sweep.  Candidates the
    device or the system cannot run (a schedule a batch does not support, a
    shape that does not fit) are skipped."""
    cands = list(candidates) if candidates is not None else list(ORDER_KEEPING)
    table = []
    for kw in cands:
        extra = dict(kw)
        if max_contacts is not None:
            extra["max_contacts"] = max_contacts
        try:
            g = cd.CDSystem(wl, device=device, batch=batch, precision=precision, criterion=cd.CD_CONV_NONE,
                            max_sweeps=sweeps, timing=1, **extra)
            g.step(1)
            st = g.step(steps)
        except cd.CDError:
            continue
        ms = st["phase_ms"]["sweep"] / (steps * max(st["last"]["sweeps"], 1))
        table.append((dict(kw), ms))
        del g
    if not table:
        raise RuntimeError("no candidate configuration could run")
    best = min(table, key=lambda t: t[1])[0]
    return best, table
