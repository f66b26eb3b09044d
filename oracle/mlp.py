"""Plain FP64 reference of the warm-start MLP (test infrastructure only).

Layout of the parameter vector (as in include/lelbm.h): W1[H][NIN] b1[H] W2[H][H] b2[H]
W3[NOUT][H] b3[NOUT], then xm[NIN] xs[NIN] ym[NOUT] ys[NOUT] (input/output standardisation).
Network: SiLU(W1 xs + b1) -> SiLU(W2 h1 + b2) -> W3 h2 + b3; loss = mean over samples and
outputs of (y - (Y - ym)/ys)^2.  Gradients by explicit back-propagation; pinned against
central finite differences in the tests.  Parity unpinned against anything but calculus.
"""
from __future__ import annotations

import numpy as np

H = 64
DIMS = {1: (8, 7), 2: (15, 16)}


def layout(dims: int):
    nin, nout = DIMS[dims]
    o = {}
    off = 0
    for name, size in [("W1", H * nin), ("b1", H), ("W2", H * H), ("b2", H), ("W3", nout * H), ("b3", nout)]:
        o[name] = (off, size)
        off += size
    nw = off
    for name, size in [("xm", nin), ("xs", nin), ("ym", nout), ("ys", nout)]:
        o[name] = (off, size)
        off += size
    return o, nw, off


def unpack(dims: int, p: np.ndarray):
    nin, nout = DIMS[dims]
    o, _, _ = layout(dims)
    g = lambda n: p[o[n][0]: o[n][0] + o[n][1]].astype(np.float64)
    return dict(W1=g("W1").reshape(H, nin), b1=g("b1"), W2=g("W2").reshape(H, H), b2=g("b2"),
                W3=g("W3").reshape(nout, H), b3=g("b3"), xm=g("xm"), xs=g("xs"), ym=g("ym"), ys=g("ys"))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(dims: int, p: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Raw targets predicted for raw features X[n, NIN]."""
    q = unpack(dims, p)
    xs = (X - q["xm"]) / q["xs"]
    h1 = silu(xs @ q["W1"].T + q["b1"])
    h2 = silu(h1 @ q["W2"].T + q["b2"])
    y = h2 @ q["W3"].T + q["b3"]
    return y * q["ys"] + q["ym"]


def loss_grad(dims: int, p: np.ndarray, X: np.ndarray, Y: np.ndarray):
    """(loss, gradient over the trained parameters) on standardised targets."""
    q = unpack(dims, p)
    n, nout = Y.shape
    xs = (X - q["xm"]) / q["xs"]
    z1 = xs @ q["W1"].T + q["b1"]
    h1 = silu(z1)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = silu(z2)
    y = h2 @ q["W3"].T + q["b3"]
    t = (Y - q["ym"]) / q["ys"]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / (n * nout)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ q["W3"]) * silu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ q["W2"]) * silu_grad(z1)
    gW1 = dz1.T @ xs
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
