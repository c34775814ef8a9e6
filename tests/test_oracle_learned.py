"""Pins for the oracle's learned-preconditioner pieces (no counterpart in the paper, so
parity is pinned to mathematics): the MLP forward on weight sets whose network is a
known function, the backward against central finite differences of the forward, and the
per-row statistics formulation of the loss against the loss evaluated directly on
explicit (r, e) pairs with an explicit sparse P."""
import numpy as np
import scipy.sparse as sp

import oracle as O
import workloads as W

SIZES = [(64, 7), (64,), (64, 64), (64,), (7, 64), (7,)]


def split(p):
    out, o = [], 0
    for s in SIZES:
        k = int(np.prod(s)); out.append(p[o:o + k].reshape(s)); o += k
    return out


def test_mlp_backward_matches_finite_differences(oracle_lib):
    rng = np.random.default_rng(0)
    p = rng.standard_normal(5127) * 0.3
    feat = rng.standard_normal((40, 7))
    gout = rng.standard_normal((40, 7))
    f = lambda q: float(np.sum(O.mlp_forward(feat, *split(q)) * gout))
    g = np.concatenate([x.ravel() for x in O.mlp_backward(feat, *split(p), gout)])
    idx = rng.choice(5127, 60, replace=False)
    for i in idx:
        h = 1e-6
        e = np.zeros_like(p); e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def _net(W1, b1, W2, b2, W3, b3):
    return [np.asarray(t, dtype=np.float64) for t in (W1, b1, W2, b2, W3, b3)]


def test_mlp_forward_closed_forms(oracle_lib):
    """Two weight sets whose network is a known function, on dyadic inputs (every
    operation exact in FP64):
    * shift and unshift: a1 = relu(f + 8) = f + 8, a2 = relu(a1 + 1) = f + 9, out = a2 - 9,
      the identity for |f| < 8 (every bias on the path matters);
    * absolute value: a1 = [relu(f), relu(-f)], a2 = relu(relu(f) + relu(-f)), out = |f|
      (the first ReLU matters: without it a2 would be relu(f - f) = 0)."""
    rng = np.random.default_rng(3)
    f = rng.integers(-64, 65, size=(50, 7)) / 16.0
    I7 = np.eye(7)
    W1 = np.zeros((64, 7)); W1[:7] = I7
    b1 = np.zeros(64); b1[:7] = 8.0
    W2 = np.eye(64); b2 = np.zeros(64); b2[:7] = 1.0
    W3 = np.zeros((7, 64)); W3[:, :7] = I7
    b3 = np.full(7, -9.0)
    assert np.array_equal(O.mlp_forward(f, *_net(W1, b1, W2, b2, W3, b3)), f)
    W1 = np.zeros((64, 7)); W1[:7] = I7; W1[7:14] = -I7
    W2 = np.zeros((64, 64)); W2[np.arange(7), np.arange(7)] = 1.0; W2[np.arange(7), np.arange(7) + 7] = 1.0
    W3 = np.zeros((7, 64)); W3[:, :7] = I7
    out = O.mlp_forward(f, *_net(W1, np.zeros(64), W2, np.zeros(64), W3, np.zeros(7)))
    assert np.array_equal(out, np.abs(f))


def _pattern_problem():
    A = W.diffusion3d_cc(6)[0]
    slot = O.spai_slots(A, 6, 36)
    diag = A.to_scipy().diagonal()
    return A, slot, diag


def test_statistics_loss_equals_direct_loss(oracle_lib):
    A, slot, diag = _pattern_problem()
    rng = np.random.default_rng(1)
    out = rng.standard_normal((A.n, 7))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    pvals = out[rows, slot] / diag[rows]
    P = sp.csr_matrix((pvals, A.col, A.rowptr), shape=(A.n, A.n))
    G = c = d = None
    direct = 0.0
    npairs = 5
    for _ in range(npairs):
        e = rng.standard_normal(A.n)
        r = A.to_scipy() @ e
        direct += np.sum((P @ r - e) ** 2) / (e @ e)
        G, c, d = O.spai_accumulate(A, slot, r, e, G, c, d)
    loss, gout = O.spai_loss(A, slot, out, diag, G, c, d, npairs, want_grad=True)
    assert abs(loss - direct / npairs) <= 1e-12 * max(1.0, direct)
    # gradient of the statistics loss by central differences
    for i, k in [(0, 3), (17, 2), (100, 6), (A.n - 1, 3)]:
        h = 1e-6
        o2 = out.copy(); o2[i, k] += h
        o1 = out.copy(); o1[i, k] -= h
        fd = (O.spai_loss(A, slot, o2, diag, G, c, d, npairs) - O.spai_loss(A, slot, o1, diag, G, c, d, npairs)) / (2 * h)
        assert abs(fd - gout[i, k]) <= 1e-6 * max(1.0, abs(fd))


def test_slots_follow_the_stencil(oracle_lib):
    A, slot, _ = _pattern_problem()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    off = np.array([-36, -6, -1, 0, 1, 6, 36])
    assert np.array_equal(A.col - rows, off[slot])
