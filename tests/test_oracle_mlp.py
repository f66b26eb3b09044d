"""Pins of the FP64 reference MLP (oracle/mlp.py): back-propagation against central finite
differences, and the layout against the sizes the library reports."""
import numpy as np
import pytest

from oracle import mlp as OM


@pytest.mark.parametrize("dims", [1, 2])
def test_backprop_matches_finite_differences(dims):
    rng = np.random.default_rng(3)
    _, nw, ntot = OM.layout(dims)
    nin, nout = OM.DIMS[dims]
    p = np.concatenate([0.3 * rng.standard_normal(nw), rng.standard_normal(nin), 0.5 + rng.random(nin),
                        rng.standard_normal(nout), 0.5 + rng.random(nout)])
    assert len(p) == ntot
    X = rng.standard_normal((13, nin))
    Y = rng.standard_normal((13, nout))
    loss, g = OM.loss_grad(dims, p, X, Y)
    for i in rng.choice(nw, 40, replace=False):
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (OM.loss_grad(dims, pp, X, Y)[0] - OM.loss_grad(dims, pm, X, Y)[0]) / (2 * h)
        # central differences: O(h^2) truncation plus eps * loss / h rounding
        assert abs(g[i] - fd) <= 1e-4 * abs(fd) + 1e-9 * loss
    # the loss is the mean squared error of the standardised forward pass
    q = OM.unpack(dims, p)
    yhat = (OM.forward(dims, p, X) - q["ym"]) / q["ys"]
    assert loss == pytest.approx(np.mean((yhat - (Y - q["ym"]) / q["ys"]) ** 2), rel=1e-12)


def test_layout_matches_library_sizes():
    from paper_2508_06911_gb300 import build, lelbm as L

    build.build()
    for dims in (1, 2):
        nin, nout, ntot, nw = L.lelbm_mlp_size(dims)
        o, nw2, ntot2 = OM.layout(dims)
        assert (nin, nout) == OM.DIMS[dims] and nw == nw2 and ntot == ntot2
