"""Learned SPAI preconditioner on the GPU: the tensor-core forward and backward kernels
(BF16 operands, FP32 accumulation) against the FP64 oracle on the same BF16-rounded
weights, and against a numpy restatement that rounds the same operands to BF16; the pair
statistics and loss against the oracle's; and what training buys in GMRES iterations
(vs. no preconditioner and vs. Jacobi), with the fallback chain decided by the true
residual.

Bars: against the FP64 oracle, the network's outputs and the loss within 2e-2
(normwise) and the weight gradients within 2e-2 relative -- what BF16 operands allow
(each BF16 rounding is 2^-9 relative).  The kernel feeds layers 1 and 2 and the output
gradient as hi + lo BF16 pairs, so that its ReLU decisions match FP64 ones except on
pre-activations within ~2^-16 of zero; with single BF16 features a few in a thousand
units flip and the gradient moves by several per cent.  Against the BF16 restatement,
where only the FP32 sums and rare rounding flips differ, 2e-3."""
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


def bf16_pair(x):
    """x (rounded to FP32) as the sum of a BF16 value and the BF16 rounding of the rest."""
    x32 = np.asarray(x, np.float32).astype(np.float64)
    hi = bf16_round(x32)
    return hi, hi + bf16_round(x32 - hi)


def bf16_net(feat, pb, gout):
    """The network with the tensor-core kernel's roundings, every sum in FP64: features,
    H1 and the output gradient as BF16 hi + lo pairs where they feed a layer, single BF16
    values elsewhere (H2, dZ2, dZ1, and the operands of the weight-gradient products).
    Returns out and the gradient."""
    W1, b1, W2, b2, W3, b3 = split(pb)
    F1, F = bf16_pair(feat)
    Z1 = F @ W1.T + b1
    H1a, H1 = bf16_pair(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = bf16_round(np.maximum(Z2, 0.0))
    out = H2 @ W3.T + b3
    G1, G = bf16_pair(gout)
    D2 = bf16_round((G @ W3) * (Z2 > 0))
    D1 = bf16_round((D2 @ W2) * (Z1 > 0))
    grads = [D1.T @ F1, D1.sum(0), D2.T @ H1a, D2.sum(0), G1.T @ H2, np.asarray(gout, np.float32).sum(0)]
    return out, np.concatenate([x.ravel() for x in grads])


@pytest.mark.parametrize("rows", [3001, 128, 77])
def test_mlp_kernels_match_oracle(rows):
    """Forward and backward on the tensor cores (several 128-row tiles and a ragged one;
    a single tile; fewer rows than a tile) against the FP64 oracle and the BF16
    restatement."""
    torch, cb = need_gpu()
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(5127) * 0.25).astype(np.float32)
    feat = rng.standard_normal((rows, 7)).astype(np.float32)
    gout = rng.standard_normal((rows, 7)).astype(np.float32)
    pb = bf16_round(p)
    ref = O.mlp_forward(feat.astype(np.float64), *split(pb))
    emu, gemu = bf16_net(feat.astype(np.float64), pb, gout.astype(np.float64))
    out = cb.mlp_forward(torch.from_numpy(feat).cuda(), p).cpu().numpy()
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    print(f"forward: vs FP64 oracle {err:.2e}, vs BF16 restatement "
          f"{np.linalg.norm(out - emu) / np.linalg.norm(emu):.2e}")
    assert err <= 2e-2, err
    assert np.linalg.norm(out - emu) <= 2e-3 * np.linalg.norm(emu)
    gref = np.concatenate([x.ravel() for x in O.mlp_backward(feat.astype(np.float64), *split(pb),
                                                             gout.astype(np.float64))])
    g = cb.mlp_backward(torch.from_numpy(feat).cuda(), p, torch.from_numpy(gout).cuda())
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    rel_emu = np.linalg.norm(g - gemu) / np.linalg.norm(gemu)
    print(f"backward: vs FP64 oracle {rel:.2e}, vs BF16 restatement {rel_emu:.2e}")
    assert rel <= 2e-2, rel
    assert rel_emu <= 2e-3, rel_emu
    # every parameter block is checked, not only the norm of the whole gradient
    for (a, b_) in zip(split(g), split(gref)):
        assert np.linalg.norm(a - b_) <= 2e-2 * np.linalg.norm(b_) + 1e-12


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
    assert abs(got - ref) <= 2e-2 * abs(ref), (got, ref)
    pv = sp.values().cpu().numpy()
    ref_out = out[rows, slot]
    # BF16 activations: compare on the scale of the outputs
    assert np.max(np.abs(pv * diag[rows] - ref_out)) <= 2e-2 * np.max(np.abs(ref_out))
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
