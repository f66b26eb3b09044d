"""Learned warm start: training kernels against the FP64 reference MLP, recorded pairs against
the oracle's converged multipliers, and what a trained network gains (Newton updates) while the
results stay those of the plain EPR."""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver
from paper_2508_06911_gb300.warmstart import record_pairs, train

import oracle as O
from oracle import mlp as OM
from parity_util import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def bf16_round(a):
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16  # round to nearest even
    return b.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("dims", [1, 2])
def test_gpu_gradient_matches_fp64_reference(dims):
    import torch

    rng = np.random.default_rng(21 + dims)
    nin, nout, ntot, nw = L.lelbm_mlp_size(dims)
    X = rng.standard_normal((300, nin)).astype(np.float32)
    Y = (0.3 * rng.standard_normal((300, nout))).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    p = L.lelbm_mlp_init(dims, 7, Xd.data_ptr(), Yd.data_ptr(), 300)
    p[:nw] += (0.05 * rng.standard_normal(nw)).astype(np.float32)
    Pd = torch.from_numpy(p).cuda()
    G = torch.zeros(nw, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    loss = L.lelbm_mlp_loss_grad(dims, Pd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), 300, G.data_ptr())
    pr = p.astype(np.float64)
    pr[:nw] = bf16_round(p[:nw])  # the kernels run with BF16 weights
    ref_loss, ref_g = OM.loss_grad(dims, pr, X.astype(np.float64), Y.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    g = G.cpu().numpy().astype(np.float64)
    assert np.abs(g - ref_g).max() <= 2e-4 * np.abs(ref_g).max()
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)


@pytest.mark.parametrize("dims", [1, 2])
def test_inference_matches_fp64_forward(dims):
    """The tensor-core inference lelbm_step runs (standardised inputs and hidden activations
    in BF16, BF16 weights, FP32 accumulation, SiLU in FP32) against the FP64 reference
    forward at the same BF16-rounded weights, element by element, on random features over
    the training range and on features recorded by the plain solver.  BF16 keeps 8 bits:
    every layer's inputs (standardised features, hidden activations) carry up to 2^-9
    relative rounding.  Each output is held to twice the first-order propagation of those
    roundings, |W3| |h2| + |W3| |SiLU'(z2)| |W2| |h1| + ... times 2^-9, computed from the
    reference's own activations (measured: at most a tenth of it), and the mean error to
    0.03 of the output scale ys (measured: 1.4e-3 in 1D, 8e-3 to 1.2e-2 in 2D, whose weights
    give larger sums |W| |h|).  A wrong weight, bias or index is off by O(0.3-1) of ys."""
    import os

    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = np.load(os.path.join(root, "paper_2508_06911_gb300", "weights", f"warmstart_{dims}d.npy"))
    nin, nout, ntot, nw = L.lelbm_mlp_size(dims)
    q = OM.unpack(dims, p)
    rng = np.random.default_rng(40 + dims)
    X_rand = (q["xm"] + q["xs"] * rng.standard_normal((4096, nin))).astype(np.float32)
    w = (W.riemann_1d(n=300, seed_index=5) if dims == 1
         else W.random_smooth_2d(24, 20, seed_index=41, RT_lo=0.25, RT_hi=2.0, umag=1.0))
    s = Solver.riemann1d(w) if dims == 1 else Solver.grid2d(w)
    X_rec, _ = record_pairs(s, steps=1)
    s.close()
    pr = p.astype(np.float64)
    pr[:nw] = bf16_round(p[:nw])
    errs = []
    for name, X in (("random", X_rand), ("recorded", X_rec.cpu().numpy())):
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        Yd = torch.empty((X.shape[0], nout), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        L.lelbm_mlp_infer(dims, p, Xd.data_ptr(), X.shape[0], Yd.data_ptr(), 0)
        got = Yd.cpu().numpy().astype(np.float64)
        ref = OM.forward(dims, pr, X.astype(np.float64))
        err = np.abs(got - ref) / q["ys"]
        # first-order bound of the BF16 roundings of the three layers' inputs (standardised units)
        u = OM.unpack(dims, pr)
        x = (X.astype(np.float64) - u["xm"]) / u["xs"]
        z1 = x @ u["W1"].T + u["b1"]
        h1 = OM.silu(z1)
        z2 = h1 @ u["W2"].T + u["b2"]
        h2 = OM.silu(z2)
        a3 = np.abs(u["W3"])
        d2 = np.abs(OM.silu_grad(z2))
        d1 = np.abs(OM.silu_grad(z1))
        e_h2 = np.abs(h2) @ a3.T
        e_h1 = ((np.abs(h1) @ np.abs(u["W2"]).T) * d2) @ a3.T
        e_x = ((((np.abs(x) @ np.abs(u["W1"]).T) * d1) @ np.abs(u["W2"]).T) * d2) @ a3.T
        bound = 2.0 * 2.0 ** -9 * (e_h2 + e_h1 + e_x) + 1e-6
        print(f"{dims}D inference vs FP64 forward, {name} features ({X.shape[0]}): max {err.max():.3e}, "
              f"mean {err.mean():.3e} of the output scale, max error / bound {(err / bound).max():.2f}")
        assert np.all(np.isfinite(got))
        errs.append((err, bound))
    for err, bound in errs:
        assert err.mean() <= 0.03
        assert np.all(err <= bound)


def test_recorded_targets_are_the_oracle_multipliers():
    import torch

    w = W.riemann_1d(n=40, seed_index=4)
    s = Solver.riemann1d(w)
    nin, nout, _, _ = L.lelbm_mlp_size(1)
    x = torch.full((s.n_cells, nin), float("nan"), dtype=torch.float32, device="cuda")
    y = torch.full((s.n_cells, nout), float("nan"), dtype=torch.float32, device="cuda")
    M0 = s.get_moments()
    torch.cuda.synchronize()
    L.lelbm_step_record(s.h, x.data_ptr(), y.data_ptr())
    s.synchronize()
    Y = y.cpu().numpy()
    pad = int(w.pads[0])
    p = O.params(1, w.K, nu_s=w.nu, Pr=w.Pr)
    # the pads were filled by the step: compare interior cells
    for cell in range(pad, pad + 40, 7):
        co, c, dC, _, _, st = O.cell_populations(p, M0[:, cell])
        assert st == 0
        sig = np.sqrt(co["RT"])
        ref = []
        for kind, con in ((0, co["cf"]), (1, co["cg"])):
            _, lam, _ = O.epr(1, kind, c, dC, co["u"], co["RT"], con, p)
            lam0 = O.maxwell_lambda(1, kind, co["RT"])
            _, order = O.basis(1, kind, np.zeros(1))
            ref += list((lam - lam0) * sig ** order)  # thermal units
        np.testing.assert_allclose(Y[cell], ref, rtol=1e-5, atol=1e-6)
    s.close()


def test_training_lowers_loss_and_newton_work_without_changing_results():
    w = W.riemann_1d_batch(n_batch=256, seed_index=808)
    s = Solver.riemann1d(w)
    X, Y = record_pairs(s, steps=1)
    assert X.shape[0] > 100_000
    params, losses = train(1, X, Y, epochs=3, batch=4096, lr=2e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0] and losses[-1] < 0.2
    s.close()
    # same state, plain start vs learned start (FP64 path): fewer Newton updates, same result
    w2 = W.riemann_1d_batch(n_batch=128, seed_index=809)
    a = Solver.riemann1d(w2)
    b = Solver.riemann1d(w2)
    L.lelbm_set_mlp(b.h, params)
    a.step(1)
    b.step(1)
    ha, hb = np.array(a.stats().newton_hist), np.array(b.stats().newton_hist)
    mean = lambda h: (np.arange(64) * h).sum() / h.sum()
    assert mean(hb) < mean(ha) - 0.3, (mean(ha), mean(hb))
    assert_close(b.get_moments(), a.get_moments(), 1e-12, "learned vs plain start")
    assert b.stats().fallback_mx == 0
    a.close()
    b.close()


@pytest.mark.parametrize("dims,case", [(1, "batch"), (2, "cylinder"), (2, "hotbox")])
def test_shipped_networks_save_newton_updates(dims, case):
    """The trained networks in weights/ take fewer Newton updates than Eq. (IID13) on
    the FP64 path, on states none of them was trained on, with the same results."""
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    params = np.load(os.path.join(here, "..", "paper_2508_06911_gb300", "weights", f"warmstart_{dims}d.npy"))
    if dims == 1:
        w = W.riemann_1d_batch(n_batch=64, seed_index=810, lmin=128, lmax=512)
        make = lambda: Solver.riemann1d(w)
    elif case == "cylinder":
        w = W.cylinder_2d(nx=192, ny=96, diameter=16)
        make = lambda: Solver.grid2d(w)
    else:
        w = W.hot_box(2, 64, 0.5)
        make = lambda: Solver.grid2d(w)
    a, b = make(), make()
    L.lelbm_set_mlp(b.h, params)
    for s in (a, b):
        s.step(3)
        L.lelbm_reset_stats(s.h)
        s.step(2)
    mean = lambda st: float((np.arange(64) * np.array(st.newton_hist)).sum() / np.array(st.newton_hist).sum())
    ma, mb = mean(a.stats()), mean(b.stats())
    print(f"{dims}D {case}: mean Newton updates {ma:.3f} (Eq. IID13) -> {mb:.3f} (learned)")
    assert mb < ma - 0.2, (ma, mb)
    assert_close(b.get_moments(), a.get_moments(), 5e-12, "learned vs plain start")
    a.close()
    b.close()


def test_learned_start_gains_time_on_the_fp64_path():
    """What the 2D network trained along the 1024^2 four-quadrant run (weights/warmstart_2d_quadrants.npy)
    gains in time, not only in Newton updates: on the FP64 path, where every Newton update
    is an FP64 pass over the velocity set, the learned start (the network's kernel included)
    makes the step faster than Eq. (IID13), with the same results.  The 1024^2 four-quadrant
    problem, whose run the network was trained on (at other times), steps 3-6; kernel time
    by CUDA events."""
    import os

    here = os.path.dirname(os.path.abspath(__file__))
    params = np.load(os.path.join(here, "..", "paper_2508_06911_gb300", "weights", "warmstart_2d_quadrants.npy"))
    w = W.riemann_2d(n=1024, seed_index=2)
    res = {}
    for start in ("maxwell", "learned"):
        s = Solver.grid2d(w)
        if start == "learned":
            L.lelbm_set_mlp(s.h, params)
        s.step(2)
        s.synchronize()
        L.lelbm_reset_stats(s.h)
        L.lelbm_set_timing(s.h, True)
        s.step(4)
        st = s.stats()
        h = np.array(st.newton_hist)
        res[start] = (st.cell_kernel_ms, float((np.arange(64) * h).sum() / h.sum()), s.get_moments())
        s.close()
    (tm, um, Mm), (tl, ul, Ml) = res["maxwell"], res["learned"]
    print(f"FP64 path, 1024^2 four-quadrant: {um:.2f} -> {ul:.2f} Newton updates per solve, "
          f"{tm:.1f} -> {tl:.1f} ms for 4 steps (learned start)")
    assert ul < um - 0.3
    assert tl < 0.9 * tm
    assert_close(Ml, Mm, 5e-12, "learned vs plain start")
