"""Training driver of the learned EPR warm start (the kernels are in csrc/lelbm_mlp.cu).

Pairs (features -> converged multipliers minus the Maxwellian start of Eq. IID13) are
recorded by the plain solver during ordinary time steps (lelbm_step_record); the network is
initialised and trained by the library's own BF16/FP32 kernels (lelbm_mlp_init,
lelbm_mlp_train).  PyTorch only provides device buffers here.

  python -m paper_2508_06911_gb300.warmstart --dims 1 --out warm1d.npy
  python -m paper_2508_06911_gb300.warmstart --dims 2 --data quadrants --out warm2d_quadrants.npy
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lelbm as L


def record_pairs(solver, steps: int = 1, max_pairs: int | None = None):
    """(X, Y) float32 CUDA tensors of the pairs recorded over `steps` time steps."""
    import torch

    nin, nout, _, _ = L.lelbm_mlp_size(solver.dims)
    xs, ys = [], []
    total = 0
    for _ in range(steps):
        x = torch.full((solver.n_cells, nin), float("nan"), dtype=torch.float32, device="cuda")
        y = torch.full((solver.n_cells, nout), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        L.lelbm_step_record(solver.h, x.data_ptr(), y.data_ptr())
        solver.synchronize()
        ok = torch.isfinite(x).all(1) & torch.isfinite(y).all(1)
        xs.append(x[ok])
        ys.append(y[ok])
        total += int(ok.sum())
        if max_pairs is not None and total >= max_pairs:
            break
    X = torch.cat(xs).contiguous()
    Y = torch.cat(ys).contiguous()
    if max_pairs is not None:
        X, Y = X[:max_pairs].contiguous(), Y[:max_pairs].contiguous()
    return X, Y


def train(dims: int, X, Y, epochs: int = 4, batch: int = 4096, lr: float = 2e-3, seed: int = 0, stages=None):
    """Initialise (normalisation from the data) and train; returns (params float32, epoch losses).
    stages: [(epochs, lr), ...] trained one after the other (Adam restarted each time);
    default one stage of `epochs` at `lr`."""
    import numpy as np
    import torch

    n = X.shape[0]
    p0 = L.lelbm_mlp_init(dims, seed, X.data_ptr(), Y.data_ptr(), n)
    P = torch.from_numpy(p0).cuda()
    torch.cuda.synchronize()
    losses = []
    for k, (ep, rate) in enumerate(stages or [(epochs, lr)]):
        losses.append(L.lelbm_mlp_train(dims, P.data_ptr(), X.data_ptr(), Y.data_ptr(), n, ep, batch, rate,
                                        seed + k))
    return P.cpu().numpy(), np.concatenate(losses)


def record_pairs_2d(max_pairs: int):
    """2D pairs from states that cover what the solver meets: smooth random fields (a
    continuum of temperature, velocity and lattice offset, with the non-equilibrium
    their gradients produce) and developed four-quadrant flows (shocks, contacts).
    Seed indices 60-63 and 70-71 are not used by the benchmark or the tests."""
    import torch

    from . import workloads as W
    from .solver import Solver

    Xs, Ys = [], []
    sources = [(W.random_smooth_2d(1024, 1024, seed_index=60 + k, RT_lo=0.2, RT_hi=rt, umag=um), 1)
               for k, (rt, um) in enumerate([(2.0, 1.0), (4.0, 2.0), (8.0, 1.5), (1.0, 3.0)])]
    sources += [(W.riemann_2d(n=1024, seed_index=70 + k), 60) for k in range(2)]
    for w, skip in sources:
        s = Solver.grid2d(w)
        s.step(skip)
        X, Y = record_pairs(s, steps=2)
        Xs.append(X)
        Ys.append(Y)
        s.close()
    X, Y = torch.cat(Xs), torch.cat(Ys)
    g = torch.Generator(device=X.device).manual_seed(2)
    keep = torch.randperm(X.shape[0], device=X.device, generator=g)[:max_pairs]
    return X[keep].contiguous(), Y[keep].contiguous()


def record_pairs_quadrants(max_pairs: int, times=(0, 3, 10, 30, 100, 300, 1000, 1999), n: int = 1024,
                           extra_smooth: int = 2):
    """2D pairs along the 1024^2 four-quadrant run (the generator of the 4096^2 benchmark
    workload, seed index 2), the flow the learned start is meant for: the state is
    advanced by the mixed path and, at each time in `times`, copied into an FP64 handle that
    records one step (the mixed path's converged multipliers equal the FP64 path's to its
    1e-12 tolerance).  `extra_smooth` smooth random fields (seed indices 60-63: temperatures
    up to RT 2, 4, 8, 1 and velocity scales 1, 2, 1.5, 3) add states between those of the
    run.  At most max_pairs pairs, drawn at random."""
    import torch

    from . import workloads as W
    from .solver import Solver

    w = W.riemann_2d(n=n, seed_index=2)
    run = Solver.grid2d(w, precision=L.LELBM_MIXED)
    rec = Solver.grid2d(w)
    Xs, Ys = [], []
    t = 0
    for t_rec in times:
        run.step(t_rec - t)
        t = t_rec
        rec.set_moments(run.get_moments())
        X, Y = record_pairs(rec, steps=1)
        Xs.append(X)
        Ys.append(Y)
    run.close()
    rec.close()
    for k, (rt, um) in enumerate([(2.0, 1.0), (4.0, 2.0), (8.0, 1.5), (1.0, 3.0)][:extra_smooth]):
        s = Solver.grid2d(W.random_smooth_2d(n, n, seed_index=60 + k, RT_lo=0.2, RT_hi=rt, umag=um))
        s.step(1)
        X, Y = record_pairs(s, steps=1)
        Xs.append(X)
        Ys.append(Y)
        s.close()
    X, Y = torch.cat(Xs), torch.cat(Ys)
    g = torch.Generator(device=X.device).manual_seed(2)
    keep = torch.randperm(X.shape[0], device=X.device, generator=g)[:max_pairs]
    return X[keep].contiguous(), Y[keep].contiguous()


def main():
    import torch

    from . import build, workloads as W
    from .solver import Solver

    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, default=1)
    ap.add_argument("--pairs", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=None, help="default: 4 (1D), 24 (2D)")
    ap.add_argument("--out", required=True)
    ap.add_argument("--data", default="quadrants", choices=["quadrants", "diverse"],
                    help="2D pairs: along the 1024^2 four-quadrant run (default) or from diverse fields")
    ap.add_argument("--lr-stages", type=int, default=3, choices=[1, 3],
                    help="2D: 1 = one stage at lr 2e-3; 3 = three stages at 2e-3, 5e-4, 1.25e-4")
    a = ap.parse_args()
    build.build()
    torch.cuda.init()
    t0 = time.time()
    if a.dims == 1:  # pairs from the 4096-instance batch (seed index 11: not the benchmark's)
        s = Solver.riemann1d(W.riemann_1d_batch(n_batch=4096, seed_index=11))
        X, Y = record_pairs(s, steps=4, max_pairs=a.pairs)
    elif a.data == "quadrants":
        X, Y = record_pairs_quadrants(a.pairs)
    else:
        X, Y = record_pairs_2d(a.pairs)
    t1 = time.time()
    epochs = a.epochs if a.epochs is not None else (4 if a.dims == 1 else 24)
    stages = None
    if a.dims == 2 and a.lr_stages == 3:
        stages = [(epochs // 3, 2e-3), (epochs // 3, 5e-4), (epochs - 2 * (epochs // 3), 1.25e-4)]
    params, losses = train(a.dims, X, Y, epochs=epochs, stages=stages)
    t2 = time.time()
    np.save(a.out, params)
    print(json.dumps({"dims": a.dims, "pairs": int(X.shape[0]), "record_s": round(t1 - t0, 2),
                      "train_s": round(t2 - t1, 2), "epoch_loss": [float(v) for v in losses]}))


if __name__ == "__main__":
    main()
