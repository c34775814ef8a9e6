"""Learned SPAI preconditioner on the GPU: the BF16/FP32 forward and backward kernels
against the FP64 oracle (same BF16-rounded weights), the pair statistics and loss
against the oracle's, and what training buys in GMRES iterations (vs. no
preconditioner and vs. Jacobi), with the fallback chain judged by the true residual."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import need_gpu, to_dev

pytestmark = pytest.mark.gpu
SIZES = [(64, 7), (64,), (64, 64), (64,), (7, 64), (7,)]


def split(p):
    out, o = [], 0
    for s in SIZES:
        k = int(np.prod(s)); out.append(p[o:o + k].reshape(s)); o += k
    return out


def bf16_round(p):
    import torch
    return torch.from_numpy(np.asarray(p, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_mlp_kernels_match_oracle():
    torch, cb = need_gpu()
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(5127) * 0.25).astype(np.float32)
    rows = 3001
    feat = rng.standard_normal((rows, 7)).astype(np.float32)
    gout = rng.standard_normal((rows, 7)).astype(np.float32)
    pb = bf16_round(p)
    ref = O.mlp_forward(feat.astype(np.float64), *split(pb))
    out = cb.mlp_forward(torch.from_numpy(feat).cuda(), p).cpu().numpy()
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(ref))
    gref = np.concatenate([x.ravel() for x in O.mlp_backward(feat.astype(np.float64), *split(pb),
                                                             gout.astype(np.float64))])
    g = cb.mlp_backward(torch.from_numpy(feat).cuda(), p, torch.from_numpy(gout).cuda())
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel <= 2e-2 and rel <= 1e-4, rel


def _problem(N=16):
    A = W.diffusion3d_cc(N)[0]
    xs = W.exact_solution(A.n, 5)
    return A, xs, W.rhs_from_solution(A, xs)


def test_pair_statistics_and_loss_match_oracle():
    torch, cb = need_gpu()
    A, _, _ = _problem(12)
    N = 12
    sp = cb.LearnedSpai(A, N, N * N)
    slot = O.spai_slots(A, N, N * N)
    diag = A.to_scipy().diagonal()
    rng = np.random.default_rng(5)
    G = c = d = None
    for k in range(4):
        xs = rng.uniform(-1, 1, A.n)
        xk = xs + rng.standard_normal(A.n) * 10.0 ** -k
        sp.add_pair(to_dev(torch, xs), to_dev(torch, xk))
        e = xs - xk
        G, c, d = O.spai_accumulate(A, slot, O.spmv(A, e), e, G, c, d)
    out0 = O.mlp_forward(np.zeros((1, 7)), *split(bf16_round(sp.params())))   # any row: check init
    assert abs(out0[0, 3] - 1.0) < 0.1
    feat = np.zeros((A.n, 7))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    feat[rows, slot] = A.val / diag[rows]
    out = O.mlp_forward(feat, *split(bf16_round(sp.params())))
    ref = O.spai_loss(A, slot, out, diag, G, c, d, 4)
    got = sp.loss()
    assert abs(got - ref) <= 1e-4 * abs(ref), (got, ref)
    pv = sp.values().cpu().numpy()
    ref_out = out[rows, slot]
    # FP32 network outputs: compare on the scale of the outputs
    assert np.max(np.abs(pv * diag[rows] - ref_out)) <= 1e-5 * np.max(np.abs(ref_out))
    sp.close()


def test_training_reduces_iterations_and_fallback(tmp_path):
    torch, cb = need_gpu()
    N = 24
    A, xs, b = _problem(N)
    gen = torch.Generator(device="cuda"); gen.manual_seed(20201206)
    spai = cb.LearnedSpai(A, N, N * N)
    with cb.Solver.from_csr(A, restart=10, fmt="f64", arith="fp64") as s64:
        cb.collect_pairs(spai, s64, nrhs=60, iterates=3, gen=gen)
    l0, l1 = spai.train(steps=300, lr=3e-3)
    assert l1 < 0.9 * l0, (l0, l1)
    pv = spai.values()
    bd = to_dev(torch, b)
    its = {}
    for pc in ("none", "jacobi", "spai"):
        with cb.Solver.from_csr(A, restart=100, fmt="f32", precond=pc) as s:
            if pc == "spai":
                s.set_spai(pv)
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            st = s.solve(bd, x, tol=1e-10, maxit=20000)
            assert st["status"] == 0, (pc, st)
            its[pc] = st["iters"]
            r = b - O.spmv(A, x.cpu().numpy())
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
    print("iterations", its, "loss", l0, "->", l1)
    assert its["spai"] < its["none"]
    # the oracle agrees on the learned operator's iteration count
    ro = O.gmres(A, b, m=100, fmt=O.F32, precond=O.PC_SPAI, pvals=pv.cpu().numpy(), tol=1e-10, maxit=20000)
    assert abs(ro["iters"] - its["spai"]) <= max(1, 0.02 * ro["iters"])
    # checkpoint round trip
    path = str(tmp_path / "spai.bin")
    spai.save(path)
    w = spai.params()
    spai.set_params(np.zeros_like(w))
    spai.load(path)
    assert np.array_equal(spai.params(), w)
    # fallback chain: a broken learned P (all zero) stagnates, Jacobi takes over
    bad = torch.zeros_like(pv)
    with cb.Solver.from_csr(A, restart=30, fmt="f32", precond="spai", stop_on_stagnation=True) as s_bad, \
            cb.Solver.from_csr(A, restart=30, fmt="f32", precond="jacobi", stop_on_stagnation=True) as s_jac, \
            cb.Solver.from_csr(A, restart=30, fmt="f32", precond="none") as s_none:
        s_bad.set_spai(bad)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st, used = cb.solve_fallback([s_bad, s_jac, s_none], bd, x, tol=1e-10, maxit=20000)
    assert st["status"] == 0 and used == 1
    r = b - O.spmv(A, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
    spai.close()
