"""Batched persistent solve (one launch, many uneven systems) against the oracle, system
by system: the same GMRES(m) with Jacobi, restart 30, tol 1e-8 (weighted-Laplacian
stencils with lognormal edge conductances, 2D and 3D, log-uniform sizes)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import need_gpu, scaled_matrix

pytestmark = pytest.mark.gpu


def _batch(nsys, nmin, nmax, seed=4):
    mats = W.stencil_batch(nsys=nsys, nmin=nmin, nmax=nmax, config_id=seed)
    xs = [W.exact_solution(A.n, 4, salt=i) for i, A in enumerate(mats)]
    bs = [W.rhs_from_solution(A, x) for A, x in zip(mats, xs)]
    return mats, bs


def _check_against_oracle(mats, bs, x, out, fmt, tol, m=30, precond=O.PC_JACOBI):
    f = O.FORMATS[fmt]
    off = 0
    for i, (A, b) in enumerate(zip(mats, bs)):
        xi = x[off:off + A.n]
        off += A.n
        ro = O.gmres(A, b, m=m, fmt=f, precond=precond, tol=tol, maxit=100000)
        assert ro["status"] == O.OK
        assert out["statuses"][i] == 0, (i, out["statuses"][i])
        res = np.linalg.norm(b - O.spmv(A, xi)) / np.linalg.norm(b)
        assert res <= tol * (1 + 1e-9), (i, res)
        assert abs(out["iters"][i] - ro["iters"]) <= max(1, 0.02 * ro["iters"]), (i, out["iters"][i], ro["iters"])
        assert np.linalg.norm(xi - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"]), i


@pytest.mark.parametrize("fmt", ["f64", "f32", "f16"])
@pytest.mark.parametrize("schedule", [(1, 1 << 30), (4, 1500), (8, 3000)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_matches_oracle(fmt, schedule, use_graph):
    torch, cb = need_gpu()
    mats, bs = _batch(24, 200, 6000)
    with cb.BatchedSolver(mats, restart=30, fmt=fmt, precond="jacobi", use_graph=use_graph) as bt:
        bt.schedule(*schedule)
        b = torch.from_numpy(np.concatenate(bs)).cuda()
        for rep in range(2):          # a second solve reuses the basis and the graph
            x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
            out = bt.solve(b, x, tol=1e-8)
            assert out["status"] == 0
        _check_against_oracle(mats, bs, x.cpu().numpy(), out, fmt, 1e-8)


@pytest.mark.parametrize("lanes", [2, 4, 8])
@pytest.mark.parametrize("fmt", ["f64", "f32", "f16"])
def test_batched_spmv_lanes_match_oracle(fmt, lanes):
    """The SpMV schedules the tuner chooses from (2, 4 or 8 lanes per row, the lanes
    splitting a row's nonzeros) give the oracle's solutions, with clusters and single
    blocks."""
    torch, cb = need_gpu()
    mats, bs = _batch(24, 200, 6000)
    with cb.BatchedSolver(mats, restart=30, fmt=fmt, precond="jacobi", use_graph=True) as bt:
        bt.schedule(4, 1500)
        assert bt.spmv_lanes(lanes) == lanes
        b = torch.from_numpy(np.concatenate(bs)).cuda()
        x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
        out = bt.solve(b, x, tol=1e-8)
        assert out["status"] == 0
        _check_against_oracle(mats, bs, x.cpu().numpy(), out, fmt, 1e-8)
    # without a preconditioner the per-step SpMV takes A's own values (FP64 path for f64)
    with cb.BatchedSolver(mats[:6], restart=30, fmt=fmt, precond="none") as bt:
        bt.spmv_lanes(lanes)
        b = torch.from_numpy(np.concatenate(bs[:6])).cuda()
        x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
        out = bt.solve(b, x, tol=1e-8)
        assert out["status"] == 0
        _check_against_oracle(mats[:6], bs[:6], x.cpu().numpy(), out, fmt, 1e-8, precond=O.PC_NONE)


@pytest.mark.parametrize("case", ["one", "tiny", "huge", "wide"])
def test_batched_without_preconditioner(case):
    """No preconditioner, restart 64: the per-step SpMV takes A's own values, normalised by a
    power of two per system (tiny, huge) or kept in FP64 (wide dynamic range); each system
    against the oracle on the same matrix."""
    torch, cb = need_gpu()
    mats, _ = _batch(10, 200, 1200, seed=9)
    mats = [scaled_matrix(A, case) for A in mats]
    bs = [W.rhs_from_solution(A, W.exact_solution(A.n, 4, salt=i)) for i, A in enumerate(mats)]
    with cb.BatchedSolver(mats, restart=64, fmt="f32", precond="none") as bt:
        b = torch.from_numpy(np.concatenate(bs)).cuda()
        x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
        out = bt.solve(b, x, tol=1e-8)
        assert out["status"] == 0
    _check_against_oracle(mats, bs, x.cpu().numpy(), out, "f32", 1e-8, m=64, precond=O.PC_NONE)


def test_batched_zero_rhs_and_tuner(tmp_path):
    torch, cb = need_gpu()
    mats, bs = _batch(12, 300, 5000, seed=7)
    bs[3] = np.zeros(mats[3].n)
    cache = str(tmp_path / "tune.jsonl")
    with cb.BatchedSolver(mats, restart=30, fmt="f32", precond="jacobi") as bt:
        b = torch.from_numpy(np.concatenate(bs)).cuda()
        x = torch.zeros(bt.total, dtype=torch.float64, device="cuda")
        c1, s1 = bt.tune(b, x, tol=1e-8, cache_path=cache)
        l1 = bt.spmv_lanes()
        bt.spmv_lanes(8 if l1 != 8 else 1)
        c2, s2 = bt.tune(b, x, tol=1e-8, cache_path=cache)     # served from the cache
        assert (c1, s1) == (c2, s2) and c1 >= 1
        assert bt.spmv_lanes() == l1 and l1 in (1, 2, 4, 8)
        assert '"lanes": ' in open(cache).read()
        x.zero_()
        out = bt.solve(b, x, tol=1e-8)
    assert out["status"] == 0 and out["iters"][3] == 0
    off = int(sum(A.n for A in mats[:3]))
    assert float(x[off:off + mats[3].n].abs().max()) == 0.0
    _check_against_oracle([A for i, A in enumerate(mats) if i != 3], [b_ for i, b_ in enumerate(bs) if i != 3],
                          np.concatenate([x.cpu().numpy()[int(sum(A.n for A in mats[:i])):int(sum(A.n for A in mats[:i + 1]))]
                                          for i in range(len(mats)) if i != 3]),
                          {k: (np.delete(v, 3) if isinstance(v, np.ndarray) else v) for k, v in out.items()},
                          "f32", 1e-8)
