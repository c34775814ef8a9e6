"""Small, self-contained cases of the hot kernels, sized for one `ncu` capture each.

    python -m paper_2009_12101_gb300.profile_cases gemv [formats] [reps]
        one basis dot and one basis axpy per format on a 2^21 x 100 basis of random unit
        columns (formats: comma-separated, default f16,e4m3,i16,bf16)
    python -m paper_2009_12101_gb300.profile_cases spmv [group] [grid]
        six Arnoldi steps of the f32 solver on the upwind convection-diffusion grid^3
        (default 96) with the SpMV schedule `group` (k > 0: k lanes per CSR row; -1: the
        sliced-ELL copy; 0: timed at create; default -1)
    python -m paper_2009_12101_gb300.profile_cases mlp [grid]
        two fused training passes of the per-row network of the learned preconditioner
        on the lognormal cell-centred diffusion grid^3 (default 64)

Every case runs the library's own kernels through the C ABI on cuda:0 and prints "ok".
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def case_gemv(fmts=("f16", "e4m3", "i16", "bf16"), reps: int = 1) -> None:
    import torch

    import paper_2009_12101_gb300 as cb
    n = ld = 1 << 21
    ncols = 100
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    w = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    for f in fmts:
        v = torch.randn(ncols, n, device="cuda", generator=g) / (n ** 0.5)
        if f == "f16":
            V, scales = v.to(torch.float16), np.ones(ncols)
        elif f == "bf16":
            V, scales = (v * 64).to(torch.bfloat16), np.full(ncols, 1 / 64)
        elif f == "e4m3":
            V, scales = (v * 2 ** 12).clamp(-448, 448).to(torch.float8_e4m3fn), np.full(ncols, 2.0 ** -12)
        elif f == "i16":
            V, scales = (v * 2 ** 13).round().clamp(-32767, 32767).to(torch.int16), np.full(ncols, 2.0 ** -13)
        elif f == "f32":
            V, scales = v, np.ones(ncols)
        else:
            raise ValueError(f"no gemv case for format {f}")
        V = V.contiguous().view(torch.uint8)
        h = np.random.default_rng(0).standard_normal(ncols) * 1e-3
        for _ in range(reps):
            cb.basis_dot(f, "df32", n, V, ld, scales, w)
            cb.basis_axpy(f, "df32", n, V, ld, scales, h, w)
    torch.cuda.synchronize()


def case_spmv(group: int = -1, grid: int = 96) -> None:
    import torch

    import paper_2009_12101_gb300 as cb
    import workloads as W
    A = W.convdiff3d(grid)
    b = torch.from_numpy(W.rhs_from_solution(A, W.exact_solution(A.n, 2))).cuda()
    with cb.Solver.from_csr(A, restart=100, fmt="f32", spmv_group=group) as s:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        s.solve(b, x, tol=1e-10, maxit=6)
        print("spmv schedule (lanes per row; 0 = sliced ELL):", s.spmv_group())


def case_mlp(grid: int = 64) -> None:
    import torch

    import paper_2009_12101_gb300 as cb
    import workloads as W
    A = W.diffusion3d_cc(grid)[0]
    sp = cb.LearnedSpai(A, grid, grid * grid)
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    for _ in range(2):
        xs = torch.rand(A.n, dtype=torch.float64, device="cuda", generator=g) * 2 - 1
        xk = xs + 0.01 * torch.randn(A.n, dtype=torch.float64, device="cuda", generator=g)
        sp.add_pair(xs, xk)
    sp.train(steps=2, lr=1e-3)
    sp.close()


def main(argv) -> int:
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    cb.lib()
    which = argv[0] if argv else "gemv"
    if which == "gemv":
        case_gemv(tuple(argv[1].split(",")) if len(argv) > 1 else ("f16", "e4m3", "i16", "bf16"),
                  int(argv[2]) if len(argv) > 2 else 1)
    elif which == "spmv":
        case_spmv(int(argv[1]) if len(argv) > 1 else -1, int(argv[2]) if len(argv) > 2 else 96)
    elif which == "mlp":
        case_mlp(int(argv[1]) if len(argv) > 1 else 64)
    else:
        raise SystemExit(f"unknown case {which}")
    print("ok")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
