"""Parity at the full sizes of the workloads bench.py times, in the configurations it times
them in: what the oracle computes there in seconds (the first Hessenberg columns, sampled
systems of a batch, sampled rows of a learned operator) and properties that hold at any
size (true residuals recomputed by the oracle's SpMV).  The headline conv-diff 128^3
workload is in test_gpu_solver.py (test_full_size_headline_workload)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import col_relerr, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fmt", ["f64", "bf16", "e4m3"])
def test_random27_full_size(fmt):
    """Random nonsymmetric n = 2^20, 27 nonzeros per row, delta = 0.1, GMRES(100) with the
    f64 / bf16 / e4m3 basis: the first 10 raw Hessenberg columns against the oracle; the
    full solve against the oracle's full solve (iterations within 2 %, x within 1e-6);
    the 1e-10 true residual, recomputed by the oracle's SpMV."""
    torch, cb = need_gpu()
    A = W.random27(1 << 20, 0.1)
    xs = W.exact_solution(A.n, 3)
    b = W.rhs_from_solution(A, xs)
    k, tol = 10, 1e-10
    r1 = O.gmres(A, b, m=k, fmt=O.FORMATS[fmt], tol=0.0, maxit=k, want_H1=True)
    ro = O.gmres(A, b, m=100, fmt=O.FORMATS[fmt], tol=tol, maxit=20000)
    assert ro["status"] == O.OK
    bd = to_dev(torch, b)
    with cb.Solver.from_csr(A, restart=100, fmt=fmt) as s:
        Hg = s.arnoldi(bd, torch.zeros(A.n, dtype=torch.float64, device="cuda"), k)
        err = col_relerr(Hg, r1["H1"], k)
        assert np.all(err <= 1e-10), err
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st = s.solve(bd, x, tol=tol, maxit=20000)
    assert st["status"] == 0, st
    xh = x.cpu().numpy()
    r = b - O.spmv(A, xh)
    assert np.linalg.norm(r) <= tol * np.linalg.norm(b) * (1 + 1e-9)
    assert abs(st["iters"] - ro["iters"]) <= max(1, 0.02 * ro["iters"]), (st["iters"], ro["iters"])
    assert np.linalg.norm(xh - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_batch512_full_size(fmt):
    """The 512-system batch (sizes log-uniform in [1024, 65536], Jacobi, restart 30,
    tol 1e-8) in one persistent launch: every system's true residual, and six sampled
    systems (the two smallest, the two largest, two in between) against the oracle's
    solves (iterations within 2 %, x within 1e-6)."""
    torch, cb = need_gpu()
    mats = W.stencil_batch()
    assert len(mats) == 512
    xs = [W.exact_solution(A.n, 4, salt=i) for i, A in enumerate(mats)]
    bs = [W.rhs_from_solution(A, x) for A, x in zip(mats, xs)]
    tol = 1e-8
    with cb.BatchedSolver(mats, restart=30, fmt=fmt, precond="jacobi", use_graph=True) as bt:
        b = torch.from_numpy(np.concatenate(bs)).cuda()
        x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
        out = bt.solve(b, x, tol=tol)
    assert out["status"] == 0
    xh = x.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([A.n for A in mats])])
    for i, (A, bi) in enumerate(zip(mats, bs)):
        assert out["statuses"][i] == 0, i
        xi = xh[offs[i]:offs[i + 1]]
        assert np.linalg.norm(bi - O.spmv(A, xi)) <= tol * np.linalg.norm(bi) * (1 + 1e-9), i
    order = np.argsort([A.n for A in mats])
    for i in (order[0], order[1], order[256], order[400], order[-2], order[-1]):
        A, bi = mats[i], bs[i]
        ro = O.gmres(A, bi, m=30, fmt=O.FORMATS[fmt], precond=O.PC_JACOBI, tol=tol, maxit=100000)
        assert ro["status"] == O.OK
        assert abs(out["iters"][i] - ro["iters"]) <= max(1, 0.02 * ro["iters"]), (i, out["iters"][i], ro["iters"])
        xi = xh[offs[i]:offs[i + 1]]
        assert np.linalg.norm(xi - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"]), i


def test_learned96_full_size():
    """Diffusion 96^3 (n = 884,736) with a lognormal(0, 1) field: pairs from FP64 GMRES and
    400 training steps as bench.py runs them; the learned operator at 2,000 sampled rows
    against the oracle's FP64 network on the same BF16-rounded weights (within 2e-2 of
    the outputs' scale: the network computes with BF16 activations); the SPAI-
    preconditioned f32-basis solve reaches the 1e-10 true residual in fewer steps than no
    preconditioner."""
    torch, cb = need_gpu()
    N = 96
    A = W.diffusion3d_cc(N)[0]
    xs = W.exact_solution(A.n, 5)
    b = W.rhs_from_solution(A, xs)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20201206)
    spai = cb.LearnedSpai(A, N, N * N)
    with cb.Solver.from_csr(A, restart=10, fmt="f64", arith="fp64") as s64:
        cb.collect_pairs(spai, s64, nrhs=667, iterates=3, gen=gen)
    l0, l1 = spai.train(steps=400, lr=3e-3)
    assert l1 < l0
    pv = spai.values().cpu().numpy()
    # sampled rows: the network on their stencil features, FP64 on the BF16-rounded weights
    p = spai.params()
    pb = torch.from_numpy(np.asarray(p, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
    sizes = [(64, 7), (64,), (64, 64), (64,), (7, 64), (7,)]
    parts, o = [], 0
    for sz in sizes:
        kk = int(np.prod(sz))
        parts.append(pb[o:o + kk].reshape(sz))
        o += kk
    slot = O.spai_slots(A, N, N * N)
    diag = A.to_scipy().diagonal()
    rng = np.random.default_rng(7)
    rows = rng.choice(A.n, 2000, replace=False)
    feat = np.zeros((rows.size, 7))
    for t, i in enumerate(rows):
        for q in range(A.rowptr[i], A.rowptr[i + 1]):
            feat[t, slot[q]] = A.val[q] / diag[i]
    ref = O.mlp_forward(feat, *parts)
    for t, i in enumerate(rows):
        for q in range(A.rowptr[i], A.rowptr[i + 1]):
            got = pv[q] * diag[i]
            assert abs(got - ref[t, slot[q]]) <= 2e-2 * max(1.0, np.max(np.abs(ref))), (i, q)
    bd = to_dev(torch, b)
    its = {}
    for pc in ("none", "spai"):
        with cb.Solver.from_csr(A, restart=100, fmt="f32", precond=pc) as s:
            if pc == "spai":
                s.set_spai(spai.values())
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            st = s.solve(bd, x, tol=1e-10, maxit=20000)
        assert st["status"] == 0, (pc, st)
        r = b - O.spmv(A, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
        its[pc] = st["iters"]
    assert its["spai"] < its["none"], its
    spai.close()


def test_multirhs_full_size():
    """The multi-RHS product at the size bench.py times (n = 2^21, 100 f16 columns, k = 8),
    on the tensor cores and on the CUDA cores: 40 sampled entries of H against the
    oracle's dot, and the two paths against each other everywhere."""
    torch, cb = need_gpu()
    n, ncols, k = 1 << 21, 100, 8
    rng = np.random.default_rng(20201207)
    v = (rng.standard_normal((ncols, n)) / np.sqrt(n)).astype(np.float16)
    dec = v.astype(np.float64)
    Wv = rng.standard_normal((k, n))
    V16 = torch.from_numpy(v.view(np.uint8)).cuda()
    Wd = torch.from_numpy(Wv).cuda()
    Ht = cb.basis_dot_multi("f16", n, V16, n, np.ones(ncols), Wd, path="tensor").cpu().numpy()
    Hc = cb.basis_dot_multi("f16", n, V16, n, np.ones(ncols), Wd, path="cuda").cpu().numpy()
    scale = np.linalg.norm(dec, axis=1)[:, None] * np.linalg.norm(Wv, axis=1)[None, :]
    assert np.all(np.abs(Ht - Hc) <= 2e-13 * scale)
    for t in range(40):
        c, r = int(rng.integers(ncols)), int(rng.integers(k))
        ref = O.dot(dec[c], Wv[r])
        assert abs(Ht[c, r] - ref) <= 1e-13 * scale[c, r], (c, r)
