"""Readers of the hand-derived golden files under tests/golden/ (shared by the
oracle pins and the GPU parity tests).  Pure input handling: no CD
arithmetic."""
import os

import numpy as np

from paper_1104_3516_gb300.workloads import Workload, masses

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_hand_case(name="detect_hand_2d.txt"):
    """Particles (x..., r), expected pairs and parameters of a golden file:
    `disc x y r` (2D) or `sphere x y z r` (3D) lines, `expect a b`, `param`."""
    disc, expect, prm = [], [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("disc", "sphere"):
                disc.append([float(t) for t in tok[1:]])
            elif tok[0] == "expect":
                expect.append((int(tok[1]), int(tok[2])))
            elif tok[0] == "param":
                prm[tok[1]] = [float(t) for t in tok[2:]]
    return np.array(disc), expect, prm


def hand_geometry(prm):
    """(dim, box_lo, box_hi, periodic, wall_mask, wall_pos) of a golden file,
    the box and periodic flags padded to three axes."""
    dim = int(prm.get("dim", [2])[0])
    box = prm["box"]
    per = [int(v) for v in prm["periodic"]]
    if dim == 2:
        lo, hi, per3 = (box[0], box[2], 0.0), (box[1], box[3], 1.0), (per[0], per[1], 0)
    else:
        lo, hi, per3 = (box[0], box[2], box[4]), (box[1], box[3], box[5]), tuple(per)
    wp = np.array(prm.get("wall_pos", [0.0] * 6), dtype=np.float64)
    return dim, lo, hi, per3, int(prm["wall_mask"][0]), wp


def hand_workload(name):
    """The golden file's particles as a Workload at rest (no gravity), and the
    expected pairs."""
    disc, expect, prm = load_hand_case(name)
    dim, lo, hi, per3, mask, wp = hand_geometry(prm)
    x = disc[:, :dim].copy()
    r = disc[:, dim].copy()
    n = r.shape[0]
    inv_m, inv_I = masses(dim, r)
    w = np.zeros(n) if dim == 2 else np.zeros((n, 3))
    wl = Workload(name=name, dim=dim, x=x, v=np.zeros((n, dim)), w=w, r=r, inv_m=inv_m, inv_I=inv_I,
                  gravity=(0.0, 0.0, 0.0), box_lo=lo, box_hi=hi, periodic=per3, wall_mask=mask,
                  delta=float(prm["delta"][0]))
    wl.wall_pos = wp
    return wl, expect
