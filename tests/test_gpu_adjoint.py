"""GPU parity of the adjoint (cd_adjoint_step) with the oracle's complex-step
derivatives of the frozen-state step map, the closed forms of single
contacts, conservation of momentum, central differences of the GPU's own
forward rollout, and the checkpointed torch.autograd rollout."""
import copy

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from oracle_adapter import system as oracle_system
from oracle_cases import DT, G, colliding_gas, head_on, leaning_column, periodic_gas, resting_disc

from gpu_common import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]

FWD_ALPHA = 1e-15
ADJ_ALPHA = 1e-13
MAX_SWEEPS = 200000


def gpu_grad(wl, steps, weights, tape=None, wall_weights=None):
    """Steps the workload on the GPU (recording every step) and
    back-propagates L = <c_x, x_T> + <c_v, v_T> + <c_w, w_T>; returns
    (dL/dx0, dL/dv0, dL/dw0, dL/dmu, per-step adjoint stats newest first)."""
    import torch
    from paper_1104_3516_gb300 import cd
    g = cd.CDSystem(wl, device="cuda:0", criterion=cd.CD_CONV_GLOBAL_REL, alpha=FWD_ALPHA, max_sweeps=MAX_SWEEPS,
                    tape_steps=tape or steps)
    g.step(steps)
    cx, cv, cw = (torch.as_tensor(np.asarray(c, dtype=np.float64).reshape(-1), device="cuda:0") for c in weights)
    gx, gv, gw = cx, cv, cw
    gmu, stats = 0.0, []
    wall = wall_weights
    for _ in range(steps):
        gx, gv, gw, st = g.adjoint_step(gx, gv, gw, ADJ_ALPHA, MAX_SWEEPS, dL_dwall_force=wall)
        wall = None
        assert st["converged"] == 1, st
        gmu += st["dL_dmu"]
        stats.append(st)
    return (gx.cpu().numpy().reshape(wl.n, 2), gv.cpu().numpy().reshape(wl.n, 2), gw.cpu().numpy(), gmu, stats)


def oracle_recs(wl, steps):
    s = oracle_system(wl, criterion=O.CRIT_GLOBAL_REL, alpha=FWD_ALPHA, max_sweeps=MAX_SWEEPS,
                      order=O.ORDER_COLOUR)
    recs = A.record_rollout(s, steps)
    return s, recs


def directions(wl, k, seed, xscale=1.0):
    rng = np.random.default_rng(seed)
    return [(xscale * rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape),
             rng.standard_normal(wl.w.shape), float(rng.standard_normal())) for _ in range(k)]


def project(grad, e):
    gx, gv, gw, gmu = grad
    ex, ev, ew, em = e
    return float(np.sum(gx * ex) + np.sum(gv * ev) + np.sum(gw * ew) + gmu * em)


def check_parity(wl, steps, seed=3, ndir=32, xscale=1.0, tol=1e-9, wall_weights=None):
    rng = np.random.default_rng(seed)
    weights = (rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape), rng.standard_normal(wl.w.shape))
    gx, gv, gw, gmu, stats = gpu_grad(wl, steps, weights, wall_weights=wall_weights)
    s, recs = oracle_recs(wl, steps)
    # the contact states of every step agree (stats are newest first)
    for st, rec in zip(stats, reversed(recs)):
        cnt = np.bincount(rec.state, minlength=3)
        assert (st["n_contacts"], st["n_open"], st["n_stick"], st["n_slide"]) == \
            (len(rec.pairs), cnt[A.OPEN], cnt[A.STICK], cnt[A.SLIDE])
    cs = A.consts_of(s)
    dirs = directions(wl, ndir, seed + 1, xscale)
    ref = A.directional_derivatives(cs, recs, wl.x, wl.v, wl.w, wl.mu, weights, dirs, wall_weights=wall_weights)
    got = np.array([project((gx, gv, gw, gmu), e) for e in dirs])
    scale = max(np.abs(ref).max(), 1.0)
    err = np.abs(got - ref).max() / scale
    assert err <= tol, (err, got[:4], ref[:4])
    return stats, recs


def test_gpu_adjoint_one_step_of_collisions():
    wl = colliding_gas(n=300, phi=0.62, vsig=3.0, dt=0.05)
    stats, recs = check_parity(wl, 1)
    assert stats[0]["n_stick"] >= 5 and stats[0]["n_slide"] >= 5


def test_gpu_adjoint_over_steps_with_touching_contacts():
    """Six steps of a fast gas under gravity: contacts left touching after
    collisions (taken as open), sticking and sliding ones, walls."""
    wl = colliding_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    stats, _ = check_parity(wl, 6)
    assert sum(s["n_slide"] for s in stats) > 10 and sum(s["n_stick"] for s in stats) > 10


def test_gpu_adjoint_with_wall_forces():
    """A loss on the last step's wall forces as well as the final state."""
    wl = colliding_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    check_parity(wl, 4, wall_weights=[0.3, -0.7, 1.0, 0.0, 0.0, 0.0])


def test_gpu_floor_force_closed_form():
    """dF/dv_y = -m/dt and dF/dy = -m/dt^2 for a disc pressed on the floor."""
    wl = resting_disc(radius=1.0, mu=0.3)
    wl.v = np.array([[0.0, -0.01]])
    m = 1.0 / wl.inv_m[0]
    z2, z1 = np.zeros((1, 2)), np.zeros(1)
    gx, gv, gw, gmu, st = gpu_grad(wl, 1, (z2, z2, z1), wall_weights=[0, 0, 1.0, 0, 0, 0])
    assert st[0]["n_stick"] == 1
    assert gv[0, 1] == pytest.approx(-m / DT, rel=1e-12)
    assert gx[0, 1] == pytest.approx(-m / DT ** 2, rel=1e-12)
    assert abs(gmu) <= 1e-12 * m


def test_gpu_adjoint_sliding_pyramids_matches_the_oracle():
    """Six pyramids on the sideways-moving floor, 200 steps, a loss on the
    final state and on the last step's wall forces: the GPU's reverse pass
    equals the oracle's complex-step derivative on 32 directions of (x0, v0,
    omega0, mu), contact states equal step by step, and sliding contacts are
    present in every step."""
    from paper_1104_3516_gb300 import workloads as W
    wl = W.sliding_pyramids(n_pyramids=6)
    stats, recs = check_parity(wl, 200, wall_weights=[0.0, 0.0, 1.0, 0.0, 0.0, 0.0], xscale=1e-3)
    assert all(s["n_slide"] >= 6 for s in stats)


def test_gpu_adjoint_periodic_gas():
    wl = periodic_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    check_parity(wl, 6)


def test_gpu_adjoint_leaning_column():
    wl = leaning_column(mu=0.18)
    check_parity(wl, 4, xscale=1e-3)


def test_gpu_momentum_gradient_is_the_mass():
    """No walls, no gravity: d(sum m v_x)/dv0 = (m, 0), and nothing else
    (positions, spins, friction) changes total momentum."""
    wl = periodic_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    m = 1.0 / wl.inv_m
    cv = np.stack([m, np.zeros_like(m)], axis=1)
    gx, gv, gw, gmu, _ = gpu_grad(wl, 6, (np.zeros_like(wl.x), cv, np.zeros_like(wl.w)))
    assert np.abs(gv[:, 0] - m).max() <= 1e-12 * m.max()
    assert np.abs(gv[:, 1]).max() <= 1e-12 * m.max()
    assert np.abs(gx).max() <= 1e-9 * m.max() / wl.dt
    assert np.abs(gw).max() <= 1e-12 * m.max()
    assert abs(gmu) <= 1e-12 * m.max()


def test_gpu_rolling_disc_closed_form():
    r = 0.9
    wl = resting_disc(radius=r, mu=1.0)
    wl.v = np.array([[1e-3, 0.0]])
    wl.w = np.array([2e-4])
    z2, z1 = np.zeros((1, 2)), np.zeros(1)
    gx, gv, gw, gmu, st = gpu_grad(wl, 1, (z2, np.array([[1.0, 0.0]]), z1))
    assert st[0]["n_stick"] == 1
    assert gv[0, 0] == pytest.approx(2.0 / 3.0, rel=1e-12)
    assert gw[0] == pytest.approx(-r / 3.0, rel=1e-12)
    gx, gv, gw, gmu, _ = gpu_grad(wl, 1, (z2, z2, np.ones(1)))
    assert gv[0, 0] == pytest.approx(-2.0 / (3.0 * r), rel=1e-12)
    assert gw[0] == pytest.approx(1.0 / 3.0, rel=1e-12)
    gx, gv, gw, gmu, _ = gpu_grad(wl, 1, (z2, np.array([[0.0, 1.0]]), z1))
    assert gx[0, 1] == pytest.approx(-1.0 / DT, rel=1e-12)


@pytest.mark.parametrize("rotations", [0, 1])
def test_gpu_sliding_disc_friction_derivative(rotations):
    r = 1.1
    wl = resting_disc(radius=r, mu=0.3)
    wl.v = np.array([[1.0, 0.0]])
    if not rotations:
        wl.inv_I = np.zeros(1)
    z2, z1 = np.zeros((1, 2)), np.zeros(1)
    gx, gv, gw, gmu, st = gpu_grad(wl, 1, (z2, np.array([[1.0, 0.0]]), z1))
    assert st[0]["n_slide"] == 1
    assert gmu == pytest.approx(-G * DT, rel=1e-12)
    assert gv[0, 0] == pytest.approx(1.0, rel=1e-12)
    gx, gv, gw, gmu, _ = gpu_grad(wl, 1, (z2, z2, np.ones(1)))
    assert gmu == pytest.approx(-2.0 * G * DT / r if rotations else 0.0, rel=1e-12, abs=1e-300)


def test_gpu_inelastic_collision_closed_form():
    r1, r2 = 1.0, 1.3
    wl = head_on(1.0, -1.0, r1=r1, r2=r2)
    m1, m2 = 1.0 / wl.inv_m[0], 1.0 / wl.inv_m[1]
    M = m1 + m2
    z2, z1 = np.zeros((2, 2)), np.zeros(2)
    c = np.zeros((2, 2))
    c[0, 0] = 1.0
    gx, gv, gw, gmu, _ = gpu_grad(wl, 1, (z2, c, z1))
    assert gv[0, 0] == pytest.approx(m1 / M, rel=1e-12)
    assert gv[1, 0] == pytest.approx(m2 / M, rel=1e-12)
    assert gx[1, 0] == pytest.approx(m2 / (M * DT), rel=1e-12)
    assert gx[0, 0] == pytest.approx(-m2 / (M * DT), rel=1e-12)
    gx, gv, gw, gmu, _ = gpu_grad(wl, 1, (c, z2, z1))
    assert gv[0, 0] == pytest.approx(DT * m1 / M, rel=1e-12)


def test_gpu_adjoint_matches_finite_differences_of_the_gpu_forward():
    """Central differences (h = 1e-6) of the GPU's own rollout of the leaning
    column against the adjoint, on 8 seeded directions."""
    from paper_1104_3516_gb300 import cd
    wl = leaning_column(mu=0.18)
    steps, h = 4, 1e-6
    rng = np.random.default_rng(11)
    weights = (rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape), rng.standard_normal(wl.w.shape))
    grad = gpu_grad(wl, steps, weights)[:4]

    def loss(x, v, w, mu):
        w2 = copy.copy(wl)
        w2.x, w2.v, w2.w, w2.mu = x, v, w, mu
        g = cd.CDSystem(w2, device="cuda:0", criterion=cd.CD_CONV_GLOBAL_REL, alpha=FWD_ALPHA,
                        max_sweeps=MAX_SWEEPS)
        g.step(steps)
        s = g.state()
        return float(np.sum(weights[0] * s["x"]) + np.sum(weights[1] * s["v"]) + np.sum(weights[2] * s["w"]))

    for e in directions(wl, 8, 12, xscale=1e-3):
        ex, ev, ew, em = e
        fd = (loss(wl.x + h * ex, wl.v + h * ev, wl.w + h * ew, wl.mu + h * em)
              - loss(wl.x - h * ex, wl.v - h * ev, wl.w - h * ew, wl.mu - h * em)) / (2 * h)
        d = project(grad, e)
        assert abs(fd - d) <= 1e-5 * max(abs(d), 1.0), (fd, d)


def test_checkpointed_rollout_equals_the_full_tape():
    """torch.autograd through 7 steps with checkpoints every 3 gives the same
    gradients, bit for bit, as recording all 7 (the recomputed steps repeat
    the forward exactly), and leaves the system in the post-rollout state."""
    import torch
    from paper_1104_3516_gb300 import autodiff, cd
    wl = colliding_gas(n=100, phi=0.62, vsig=3.0, dt=0.02)
    out = []
    for k in (3, 7):
        g = cd.CDSystem(wl, device="cuda:0", criterion=cd.CD_CONV_GLOBAL_REL, alpha=FWD_ALPHA,
                        max_sweeps=MAX_SWEEPS, tape_steps=k)
        dd = dict(dtype=torch.float64, device="cuda:0")
        x0 = torch.as_tensor(wl.x, **dd).requires_grad_()
        v0 = torch.as_tensor(wl.v, **dd).requires_grad_()
        w0 = torch.as_tensor(wl.w, **dd).requires_grad_()
        mu = torch.tensor(wl.mu, dtype=torch.float64, requires_grad=True)
        xT, vT, wT, FT = autodiff.rollout(g, x0, v0, w0, mu, 7, checkpoint_every=k, alpha=ADJ_ALPHA,
                                          max_sweeps=MAX_SWEEPS)
        L = (xT[:, 1].sum() + (vT ** 2).sum() + wT.sum()).cpu() + FT[2] / 15.0
        L.backward()
        after = g.state()
        assert np.array_equal(after["x"], xT.detach().cpu().numpy())
        out.append((x0.grad.cpu().numpy(), v0.grad.cpu().numpy(), w0.grad.cpu().numpy(), float(mu.grad)))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_gpu_adjoint_settling_10k_against_finite_differences():
    """The differentiated settling rollout at full size: 10,000 discs, 200
    steps, checkpoints every 20; L = floor pressure of the last step + the
    packing height (top of the highest disc).  The autograd gradient with
    respect to (v0, mu) is checked by central differences (h = 1e-6) of the
    GPU's own rollout on 32 seeded directions.  A direction whose one-sided
    differences disagree has a kink (a contact changing state or the top disc
    changing) inside +-h and is reported, not compared; the smooth ones must
    agree to 1e-5."""
    import torch
    from paper_1104_3516_gb300 import autodiff, cd, workloads as W
    wl = W.settling_discs(n=10_000)
    steps, every, h = 200, 20, 1e-6
    width = float(wl.wall_pos[1] - wl.wall_pos[0])
    kw = dict(criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-13, max_sweeps=20000)

    def loss_of(v0, mu):
        w2 = copy.copy(wl)
        w2.v, w2.mu = v0, mu
        g = cd.CDSystem(w2, device="cuda:0", **kw)
        st = g.step(steps)
        y = g.state()["x"][:, 1]
        return st["last"]["wall_force"][2] / width + float(np.max(y + wl.r))

    g = cd.CDSystem(wl, device="cuda:0", tape_steps=every, **kw)
    dd = dict(dtype=torch.float64, device="cuda:0")
    x0 = torch.as_tensor(wl.x, **dd)
    v0 = torch.as_tensor(wl.v, **dd).requires_grad_()
    w0 = torch.as_tensor(wl.w, **dd)
    mu = torch.tensor(wl.mu, dtype=torch.float64, requires_grad=True)
    xT, vT, wT, FT = autodiff.rollout(g, x0, v0, w0, mu, steps, checkpoint_every=every, alpha=1e-13,
                                      max_sweeps=200000)
    r = torch.as_tensor(wl.r, **dd)
    L = FT[2] / width + torch.max(xT[:, 1] + r).cpu()
    L.backward()
    gv, gmu = v0.grad.cpu().numpy(), float(mu.grad)
    L0 = loss_of(wl.v, wl.mu)
    assert abs(L0 - float(L.detach())) <= 1e-12 * abs(L0)
    rng = np.random.default_rng(2024)
    smooth, kinked = 0, 0
    for _ in range(32):
        ev, em = rng.standard_normal(wl.v.shape), float(rng.standard_normal())
        Lp = loss_of(wl.v + h * ev, wl.mu + h * em)
        Lm = loss_of(wl.v - h * ev, wl.mu - h * em)
        d = float(np.sum(gv * ev) + gmu * em)
        scale = max(abs(d), 1.0)
        if abs((Lp - L0) - (L0 - Lm)) / h > 1e-4 * scale:
            kinked += 1
            continue
        smooth += 1
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - d) <= 1e-5 * scale, (fd, d)
    print(f"settling 10k: {smooth} smooth directions agree, {kinked} kinked")
    assert smooth >= 16


def test_gpu_adjoint_sliding_pyramids_10k_against_finite_differences(record_property):
    """A friction-dominated rollout at full size: 3,334 pyramids of three
    discs (10,002 discs) on a floor moving sideways under them, 200 steps,
    checkpoints every 20.  The base discs slide on the floor throughout, so
    the packing height H and the floor pressure F of the last step both
    depend on mu.  Every rollout sweeps 150 times per step (a step converges
    to 1e-13 in ~40, and a test on the mean impulse of 3,334 independent
    pyramids would stop at a different sweep in each perturbed run).

    dH/d(v0, mu) from autograd is checked by central differences D(h) of the
    GPU's own rollout on the pure-mu direction and 16 seeded directions, at
    h = 1e-4 (H carries ~3e-12 of rounding noise, ~1e-8 in D(h) there): to
    1e-5 of max(|d|, |D|).  A direction has a kink within +-h, and is
    reported, not compared, if a perturbed rollout ends in other contact
    states than the unperturbed one, if another disc is the highest (H is a
    maximum), or if D(h) and D(h / 2) differ by more than 1e-5.  A random
    perturbation of all 20,004 initial velocities by 1e-4 moves some contact
    of some pyramid across a switch in most directions (the detector counts
    any pyramid, not only the highest one, which alone sets H), so the test
    asks for the pure-mu direction and at least four more smooth ones.

    F carries ~4e-9 of rounding noise from the trajectory (measured on this
    rollout: residuals of a cubic fit over mu +- 4e-4), and its nearest kink
    lies at mu + 4e-4, so its difference quotient cannot resolve 1e-5: dF/dmu
    is held to 1e-4 (central differences at 1e-4 and 2e-4, Richardson-
    extrapolated, R = (4 D(h) - D(2 h)) / 3), and to 1e-9 against the
    oracle's complex-step derivative on six pyramids (test above)."""
    import torch
    from paper_1104_3516_gb300 import autodiff, cd, workloads as W
    wl = W.sliding_pyramids(n_pyramids=3334)
    steps, every, h = 200, 20, 1e-4
    width = float(wl.box_hi[0] - wl.box_lo[0])
    kw = dict(criterion=cd.CD_CONV_NONE, max_sweeps=150)

    def run(v0, mu):
        """(F, H, contact states at the end, highest disc) of a rollout from (v0, mu)."""
        w2 = copy.copy(wl)
        w2.v, w2.mu = v0, mu
        g = cd.CDSystem(w2, device="cuda:0", **kw)
        st = g.step(steps)
        y = g.state()["x"][:, 1]
        c = g.contacts()
        pn, pt = c["impulse"][:, 0], np.abs(c["impulse"][:, 1])
        state = np.where(pn <= 0, 0, np.where(pt >= (1 - 1e-12) * mu * pn, 2, 1))
        return (st["last"]["wall_force"][2] / width, float(np.max(y + wl.r)), (c["pairs"], state),
                int(np.argmax(y + wl.r)))

    g = cd.CDSystem(wl, device="cuda:0", tape_steps=every, **kw)
    dd = dict(dtype=torch.float64, device="cuda:0")
    x0 = torch.as_tensor(wl.x, **dd)
    v0 = torch.as_tensor(wl.v, **dd).requires_grad_()
    w0 = torch.as_tensor(wl.w, **dd)
    mu = torch.tensor(wl.mu, dtype=torch.float64, requires_grad=True)
    xT, vT, wT, FT = autodiff.rollout(g, x0, v0, w0, mu, steps, checkpoint_every=every, alpha=1e-13,
                                      max_sweeps=200000)
    r = torch.as_tensor(wl.r, **dd)
    H = torch.max(xT[:, 1] + r)
    F = FT[2] / width
    gv_H, gmu_H = torch.autograd.grad(H, [v0, mu], retain_graph=True)
    gmu_F, = torch.autograd.grad(F, [mu])
    gv_H, gmu_H, gmu_F = gv_H.cpu().numpy(), float(gmu_H), float(gmu_F)
    F0, H0, s0, top0 = run(wl.v, wl.mu)
    assert abs(F0 - float(F.detach())) <= 1e-12 * abs(F0) and abs(H0 - float(H.detach())) <= 1e-12 * abs(H0)
    assert abs(gmu_H) > 1e-3 and abs(gmu_F) > 0.1       # friction matters for both losses
    rng = np.random.default_rng(2025)
    dirs = [(np.zeros_like(wl.v), 1.0)] + [(rng.standard_normal(wl.v.shape), float(rng.standard_normal()))
                                           for _ in range(16)]
    smooth, kinked = 0, 0
    for i, (ev, em) in enumerate(dirs):
        out = {hh: (run(wl.v + hh * ev, wl.mu + hh * em), run(wl.v - hh * ev, wl.mu - hh * em))
               for hh in (h, h / 2)}
        same = all(np.array_equal(o[2][0], s0[0]) and np.array_equal(o[2][1], s0[1]) and o[3] == top0
                   for p in out.values() for o in p)
        DH = [(out[hh][0][1] - out[hh][1][1]) / (2 * hh) for hh in (h, h / 2)]
        d = float(np.sum(gv_H * ev) + gmu_H * em)
        if not same or abs(DH[0] - DH[1]) > 1e-5 * max(abs(d), abs(DH[0])):
            kinked += 1
            assert i > 0, ("the pure-mu direction has a kink", DH, d)
            continue
        smooth += 1
        assert abs(DH[0] - d) <= 1e-5 * max(abs(d), abs(DH[0])), (i, DH, d)
    hF = 1e-4
    DF = [(run(wl.v, wl.mu + hh)[0] - run(wl.v, wl.mu - hh)[0]) / (2 * hh) for hh in (hF, 2 * hF)]
    RF = (4 * DF[0] - DF[1]) / 3
    record_property("dF_dmu", {"autograd": gmu_F, "richardson": RF, "central": DF})
    assert abs(RF - gmu_F) <= 1e-4 * abs(gmu_F), (DF, RF, gmu_F)
    print(f"sliding pyramids 10k: dH/dmu = {gmu_H:.6g}, dF/dmu = {gmu_F:.6g}; {smooth} smooth directions agree, "
          f"{kinked} kinked")
    assert smooth >= 5


def test_gpu_adjoint_compliance():
    """A relative compliance of 1e-12 leaves the derivative of a
    well-posed network unchanged (parity with the rigid oracle holds); on a
    loaded pile, whose contact network is hyperstatic, a compliance of 1e-3
    gives converged, finite gradients through every step."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    wl = leaning_column(mu=0.18)
    rng = np.random.default_rng(3)
    weights = (rng.standard_normal(wl.x.shape), rng.standard_normal(wl.v.shape), rng.standard_normal(wl.w.shape))
    g = cd.CDSystem(wl, device="cuda:0", criterion=cd.CD_CONV_GLOBAL_REL, alpha=FWD_ALPHA, max_sweeps=MAX_SWEEPS,
                    tape_steps=4, adjoint_compliance=1e-12)
    g.step(4)
    gx, gv, gw = (torch.as_tensor(c.reshape(-1), device="cuda:0") for c in weights)
    gmu = 0.0
    for _ in range(4):
        gx, gv, gw, st = g.adjoint_step(gx, gv, gw, ADJ_ALPHA, MAX_SWEEPS)
        gmu += st["dL_dmu"]
    ref = gpu_grad(wl, 4, weights)
    assert np.abs(gv.cpu().numpy().reshape(-1, 2) - ref[1]).max() <= 1e-9 * max(np.abs(ref[1]).max(), 1.0)
    assert abs(gmu - ref[3]) <= 1e-9 * max(abs(ref[3]), 1.0)

    pile = W.settled_pile(7, 400)
    g = cd.CDSystem(pile, device="cuda:0", criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-12, max_sweeps=20000,
                    tape_steps=20, adjoint_compliance=1e-3)
    g.step(20)
    n = pile.n
    gx = torch.zeros(2 * n, dtype=torch.float64, device="cuda:0")
    gx[1::2] = 1.0 / n
    gv, gw = torch.zeros_like(gx), torch.zeros(n, dtype=torch.float64, device="cuda:0")
    hyper = 0
    for _ in range(20):
        gx, gv, gw, st = g.adjoint_step(gx, gv, gw, 1e-10, 200000, dL_dwall_force=[0, 0, 1.0, 0, 0, 0])
        assert st["converged"] == 1 and st["diverged"] == 0, st
        hyper += st["n_rows"] > st["n_dof"]
    assert hyper > 0
    assert torch.isfinite(gv).all() and torch.isfinite(gx).all()


def test_graph_replayed_steps_equal_direct_launches():
    """use_graph = 1 captures one step into a CUDA graph and replays it:
    states, contacts and the tape (hence the adjoint) are bit-identical to
    stepping with direct launches, through contact-set changes and
    checkpoint reloads."""
    import torch
    from paper_1104_3516_gb300 import cd
    wl = colliding_gas(n=300, phi=0.62, vsig=3.0, dt=0.02)
    out = []
    for graph in (0, 1):
        stream = torch.cuda.Stream(device="cuda:0")
        g = cd.CDSystem(wl, device="cuda:0", stream=stream, criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-12,
                        max_sweeps=5000, tape_steps=4, use_graph=graph)
        ck = g.save_checkpoint()
        g.step(3)
        g.load_checkpoint(ck)
        st = g.step(6)
        c = g.contacts()
        s = g.state()
        n = wl.n
        gx = torch.ones(2 * n, dtype=torch.float64, device="cuda:0")
        gv, gw = torch.zeros_like(gx), torch.zeros(n, dtype=torch.float64, device="cuda:0")
        for _ in range(4):
            gx, gv, gw, _ = g.adjoint_step(gx, gv, gw, 1e-13, 100000)
        torch.cuda.synchronize()
        out.append((s["x"], s["v"], s["w"], c["pairs"], c["impulse"], gx.cpu().numpy(), gv.cpu().numpy(),
                    st["total_sweeps"]))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
