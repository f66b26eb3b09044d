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
