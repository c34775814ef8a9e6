"""Pins for the oracle's GMRES(m) (Fig. 1; Section 2; Section 5.2).

Every check compares the oracle with something it does not share code with: dense LU
solves, a dense least-squares minimiser over an explicitly built Krylov space, exact
termination on matrices with few distinct eigenvalues, closed-form eigenvalues of the
1D Poisson matrix, the Arnoldi relation, orthogonality, and monotonicity of the GMRES
residual.  A plausible mistake (dropped term, sign, index, transposed operand) breaks
at least one of them.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

ALL = ["f64", "f32", "f16", "bf16", "e4m3", "i32", "i16"]


def _rand_nonsym(n, seed, shift=3.0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n)
    return a


# --------------------------------------------------------------- dense LU (exact answer)
@pytest.mark.parametrize("fmt", ALL)
def test_matches_dense_lu(oracle_lib, fmt):
    for n, seed in ((5, 1), (17, 2), (40, 3)):
        a = _rand_nonsym(n, seed)
        A = W.from_dense(a)
        b = np.random.default_rng(seed + 10).standard_normal(n)
        ref = np.linalg.solve(a, b)
        r = O.gmres(A, b, m=max(n, 8), fmt=O.FORMATS[fmt], tol=1e-13, maxit=4000)
        assert r["status"] == O.OK, (fmt, n, r["status"], r["true_relres"])
        assert np.linalg.norm(r["x"] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_matches_dense_lu_jacobi(oracle_lib):
    a = _rand_nonsym(30, 4) + np.diag(np.linspace(1, 50, 30))
    A = W.from_dense(a)
    b = np.random.default_rng(5).standard_normal(30)
    r = O.gmres(A, b, m=10, precond=O.PC_JACOBI, tol=1e-13, maxit=2000)
    assert r["status"] == O.OK
    ref = np.linalg.solve(a, b)
    assert np.linalg.norm(r["x"] - ref) <= 1e-10 * np.linalg.norm(ref)


# ---------------------------------------- Krylov least squares: x_k = argmin over x0 + K_k
def _krylov_ls(a, minv, b, x0, k):
    r0 = b - a @ x0
    am = a @ minv
    K = np.empty((a.shape[0], k))
    v = r0.copy()
    for i in range(k):
        K[:, i] = v / np.linalg.norm(v)
        v = am @ K[:, i]
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(am @ Q, r0, rcond=None)
    x = x0 + minv @ (Q @ c)
    return x, np.linalg.norm(b - a @ x)


@pytest.mark.parametrize("precond", [O.PC_NONE, O.PC_JACOBI])
def test_iterates_are_krylov_minimisers(oracle_lib, precond):
    n = 30
    a = _rand_nonsym(n, 6, shift=2.0) + np.diag(np.linspace(0.5, 4, n))
    A = W.from_dense(a)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(n); x0 = rng.standard_normal(n) * 0.1
    minv = np.diag(1.0 / np.diag(a)) if precond == O.PC_JACOBI else np.eye(n)
    bn = np.linalg.norm(b)
    for k in range(1, 9):
        r = O.gmres(A, b, x0, m=20, precond=precond, tol=0.0, maxit=k, want_H1=True,
                    hist_cap=k)
        xk, resk = _krylov_ls(a, minv, b, x0, k)
        assert r["iters"] == k
        assert np.linalg.norm(r["x"] - xk) <= 1e-10 * np.linalg.norm(xk)
        # Givens recurrence residual equals the dense least-squares residual
        assert abs(r["hist"][k - 1] - resk / bn) <= 1e-12


def test_poisson2d_recurrence_matches_dense_krylov_ls(oracle_lib):
    A = W.poisson2d(16)
    a = A.dense()
    b = W.rhs_sin(A.n)
    r = O.gmres(A, b, m=50, tol=0.0, maxit=8, hist_cap=8)
    for k in range(1, 9):
        _, resk = _krylov_ls(a, np.eye(A.n), b, np.zeros(A.n), k)
        assert abs(r["hist"][k - 1] - resk / np.linalg.norm(b)) <= 1e-12


# ------------------------------------------------------------------- exact termination
def test_identity_converges_in_one_step(oracle_lib):
    A = W.from_dense(np.eye(12))
    b = np.arange(1.0, 13.0)
    r = O.gmres(A, b, m=5, tol=1e-14)
    assert r["status"] == O.OK and r["iters"] == 1
    assert np.allclose(r["x"], b, rtol=1e-15, atol=0)


@pytest.mark.parametrize("k", [2, 3, 5])
def test_k_distinct_eigenvalues_terminate_in_k_steps(oracle_lib, k):
    n = 25
    rng = np.random.default_rng(k)
    eig = np.arange(1, k + 1, dtype=float)[rng.integers(0, k, n)]
    eig[:k] = np.arange(1, k + 1)          # every eigenvalue present
    S = np.eye(n) + 0.3 * np.triu(rng.standard_normal((n, n)), 1)
    a = S @ np.diag(eig) @ np.linalg.inv(S)   # nonsymmetric, k distinct eigenvalues
    A = W.from_dense(a)
    b = rng.standard_normal(n)
    r = O.gmres(A, b, m=20, tol=1e-11, maxit=200, want_H1=True)
    assert r["status"] == O.OK
    assert r["k1"] <= k                      # first cycle ends by breakdown or convergence
    assert np.linalg.norm(r["x"] - np.linalg.solve(a, b)) <= 1e-9 * np.linalg.norm(r["x"])


# ------------------------------------------- 1D Poisson: closed-form eigenvalues (Lanczos)
def test_poisson1d_hessenberg_eigenvalues_closed_form(oracle_lib):
    n = 20
    a = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = W.from_dense(a)
    b = np.random.default_rng(11).standard_normal(n)
    r = O.gmres(A, b, m=n, tol=0.0, maxit=n, want_H1=True)
    k = r["k1"]
    assert k == n
    H = r["H1"][:k, :k]
    # symmetric A: the Hessenberg is tridiagonal and symmetric (Lanczos)
    assert np.max(np.abs(np.triu(H, 2))) <= 1e-12
    assert np.allclose(np.diag(H, 1), np.diag(H, -1), rtol=1e-10, atol=1e-12)
    lam = np.sort(np.linalg.eigvals(H).real)
    exact = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    assert np.max(np.abs(lam - exact)) <= 1e-10


# ------------------------------------------------------- Arnoldi relation, orthogonality
_DELTA = {"f64": (0.0, 0.0), "f32": (2.0 ** -24, 0.0), "f16": (2.0 ** -11, 2.0 ** -25),
          "bf16": (2.0 ** -8 + 2.0 ** -24, 0.0), "e4m3": (2.0 ** -4 + 2.0 ** -24, None),
          "i32": (0.0, None), "i16": (0.0, None)}


@pytest.mark.parametrize("fmt", ALL)
def test_arnoldi_relation(oracle_lib, fmt):
    A = W.convdiff3d(6)
    a = A.dense()
    b = W.rhs_sin(A.n)
    k = 25
    r = O.gmres(A, b, m=k, fmt=O.FORMATS[fmt], tol=0.0, maxit=k, want_H1=True, want_V1=True)
    V = r["V1"]; H = r["H1"][: k + 1, :k]
    assert V.shape[1] == k + 1
    E = a @ V[:, :k] - V @ H
    rel, absq = _DELTA[fmt]
    nA = np.linalg.norm(a, 2)
    for j in range(k):
        hn = H[j + 1, j]
        vj1 = V[:, j + 1]
        if absq is None:   # scaled formats: half the quantum of the stored vector
            if fmt in ("i32", "i16"):
                q = np.min(np.abs(vj1[vj1 != 0])) if np.any(vj1) else 0.0
                mx = 32767 if fmt == "i16" else 2147483647
                sigma = np.max(np.abs(vj1)) / mx
                bound_v = 0.5 * sigma * np.sqrt(A.n) * 1.0001
            else:
                s = 2.0 ** np.ceil(np.log2(np.max(np.abs(vj1)) / 448.0))
                bound_v = rel * 1.0 + 0.5 * 2.0 ** -9 * s * np.sqrt(A.n)
        else:
            bound_v = rel + absq * np.sqrt(A.n)
        assert np.linalg.norm(E[:, j]) <= hn * bound_v * 1.01 + 1e-13 * nA, (j, fmt)


def test_orthogonality_f64_cgs2(oracle_lib):
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    r = O.gmres(A, b, m=60, tol=0.0, maxit=60, want_V1=True)
    V = r["V1"]
    assert np.linalg.norm(np.eye(V.shape[1]) - V.T @ V, 2) <= 1e-13


@pytest.mark.parametrize("delta", [1e-8, 1e-10, 1e-12])
def test_orthogonality_cgs2_near_invariant_krylov_space(oracle_lib, delta):
    """A = I + delta E (E Gaussian): each new direction A v_j - V h is about delta of
    omega = ||A v_j||, so after the first CGS pass w still carries components along V of
    the order of the rounding of omega -- for small delta comparable to w itself.  The
    second pass removes them (CGS2, "twice is enough"), and v_{j+1} = w / h_{j+1,j} is a
    unit vector only if h_{j+1,j} is the norm after that pass (Fig. 1): the basis stays
    orthonormal to working precision."""
    n = 12
    rng = np.random.default_rng(11)
    M = np.eye(n) + delta * rng.standard_normal((n, n))
    A = W.from_dense(M)
    b = rng.standard_normal(n)
    r = O.gmres(A, b, m=6, tol=0.0, maxit=6, want_V1=True)
    V = r["V1"]
    assert V.shape[1] == 7
    assert np.linalg.norm(np.eye(7) - V.T @ V, 2) <= 1e-14


@pytest.mark.parametrize("fmt,bound", [("f32", 1e-6), ("i32", 1e-8), ("f16", 5e-3), ("i16", 5e-4)])
def test_orthogonality_compressed(oracle_lib, fmt, bound):
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    r = O.gmres(A, b, m=40, fmt=O.FORMATS[fmt], tol=0.0, maxit=40, want_V1=True)
    V = r["V1"]
    assert np.linalg.norm(np.eye(V.shape[1]) - V.T @ V, 2) <= bound


# -------------------------------------------------------------- residual behaviour
@pytest.mark.parametrize("fmt", ["f64", "f16", "i16"])
def test_recurrence_residual_monotone_within_cycle(oracle_lib, fmt):
    A = W.convdiff3d(10)
    b = W.rhs_sin(A.n)
    m = 15
    r = O.gmres(A, b, m=m, fmt=O.FORMATS[fmt], tol=1e-10, maxit=600, hist_cap=600, tres_cap=100)
    h = r["hist"]
    for c0 in range(0, len(h), m):
        seg = h[c0:c0 + m]
        assert np.all(np.diff(seg) <= 1e-15 * seg[0])


def test_explicit_equals_recurrence_residual_f64(oracle_lib):
    A = W.convdiff3d(10)
    b = W.rhs_sin(A.n)
    r = O.gmres(A, b, m=200, tol=1e-10, maxit=1000, hist_cap=1000)
    assert r["status"] == O.OK and r["cycles"] == 1
    assert abs(r["true_relres"] - r["hist"][-1]) <= 1e-13


def test_restarts_continue_from_explicit_residual(oracle_lib):
    A = W.poisson2d(32)
    xs = W.exact_solution(A.n, 1)
    b = W.rhs_from_solution(A, xs)
    r = O.gmres(A, b, m=10, tol=1e-8, maxit=5000, tres_cap=1000)
    assert r["status"] == O.OK and r["cycles"] > 3
    t = r["tres"]
    assert t[0] == pytest.approx(1.0) and t[-1] <= 1e-8
    assert np.all(np.diff(t) <= 1e-15)    # GMRES never increases the residual norm


# -------------------------------------------------------------- reorthogonalisation modes
def test_reorth_modes(oracle_lib):
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    ra = O.gmres(A, b, m=30, tol=1e-10, maxit=3000, reorth=O.REORTH_ALWAYS)
    rc = O.gmres(A, b, m=30, tol=1e-10, maxit=3000, reorth=O.REORTH_CONDITIONAL)
    rn = O.gmres(A, b, m=30, tol=1e-10, maxit=3000, reorth=O.REORTH_NEVER)
    for r in (ra, rc, rn):
        assert r["status"] == O.OK and r["true_relres"] <= 1e-10
    assert ra["reorths"] == ra["iters"]
    assert 0 <= rc["reorths"] <= rc["iters"]
    assert rn["reorths"] == 0


def test_conditional_reorth_limits(oracle_lib):
    """Fig. 1 re-orthogonalises when h_{j+1,j} < eta omega: with eta = 0 the test never
    holds (the conditional solve is the one that never re-orthogonalises, bit for bit),
    with eta beyond any ratio it always holds (the solve that always does)."""
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    kw = dict(m=30, tol=1e-10, maxit=3000)
    ra = O.gmres(A, b, reorth=O.REORTH_ALWAYS, **kw)
    rn = O.gmres(A, b, reorth=O.REORTH_NEVER, **kw)
    r0 = O.gmres(A, b, reorth=O.REORTH_CONDITIONAL, eta=0.0, **kw)
    rinf = O.gmres(A, b, reorth=O.REORTH_CONDITIONAL, eta=1e300, **kw)
    assert r0["reorths"] == 0 and r0["iters"] == rn["iters"] and np.array_equal(r0["x"], rn["x"])
    assert rinf["reorths"] == rinf["iters"] == ra["iters"] and np.array_equal(rinf["x"], ra["x"])


@pytest.mark.parametrize("k", [-60, 40])
def test_power_of_two_operator_scaling_is_exact(oracle_lib, k):
    """GMRES commutes with scaling A by 2^k: every product, norm and coefficient scales
    exactly in binary floating point, the Givens rotations and the tests of Fig. 1
    (h_{j+1,j} against eta omega, the breakdown test against omega) are ratios, so the
    solve of (2^k A) x = b returns 2^-k times the x of A x = b, bit for bit, after the same
    steps."""
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    As = W.CSR(A.n, A.rowptr, A.col, A.val * 2.0 ** k)
    for fmt in (O.F64, O.F32, O.I16):
        r = O.gmres(A, b, m=20, fmt=fmt, tol=1e-10, maxit=3000, hist_cap=3000)
        rs = O.gmres(As, b, m=20, fmt=fmt, tol=1e-10, maxit=3000, hist_cap=3000)
        assert r["status"] == rs["status"] == O.OK
        assert r["iters"] == rs["iters"] and r["cycles"] == rs["cycles"]
        assert np.array_equal(rs["x"] * 2.0 ** k, r["x"])
        assert np.array_equal(rs["hist"], r["hist"])


def test_literal_fig1_clause_truncates_cycles(oracle_lib):
    """Reading R2: the printed second clause of Fig. 1's breakdown test ends a cycle as soon as
    h_{j+1,j} < eta * omega; on this problem that happens within the first steps."""
    A = W.convdiff3d(8)
    b = W.rhs_sin(A.n)
    r_lit = O.gmres(A, b, m=30, tol=1e-10, maxit=30, reorth=O.REORTH_CONDITIONAL,
                    literal_fig1=True)
    r_brk = O.gmres(A, b, m=30, tol=1e-10, maxit=30, reorth=O.REORTH_CONDITIONAL)
    assert r_lit["k1"] < 30 <= r_brk["k1"] or r_lit["k1"] < r_brk["k1"]


# ------------------------------------------------------------------------- edge cases
def test_zero_rhs_gives_zero(oracle_lib):
    A = W.poisson2d(4)
    r = O.gmres(A, np.zeros(A.n), np.ones(A.n), m=5)
    assert r["status"] == O.OK and r["iters"] == 0 and np.all(r["x"] == 0)


def test_exact_initial_guess(oracle_lib):
    A = W.poisson2d(4)
    xs = np.arange(A.n, dtype=float)
    b = O.spmv(A, xs)
    r = O.gmres(A, b, xs, m=5)
    assert r["status"] == O.OK and r["iters"] == 0


def test_n_equals_one(oracle_lib):
    A = W.from_dense(np.array([[4.0]]))
    r = O.gmres(A, np.array([2.0]), m=3)
    assert r["status"] == O.OK and r["iters"] == 1 and r["x"][0] == 0.5


def test_maxit_limits_and_reports(oracle_lib):
    A = W.poisson2d(16)
    b = W.rhs_sin(A.n)
    r = O.gmres(A, b, m=10, tol=1e-12, maxit=7)
    assert r["status"] == O.NOT_CONVERGED and r["iters"] == 7
    r0 = O.gmres(A, b, m=10, tol=1e-12, maxit=0)
    assert r0["status"] == O.NOT_CONVERGED and r0["iters"] == 0


def test_nonfinite_input(oracle_lib):
    A = W.poisson2d(4)
    b = np.ones(A.n); b[3] = np.nan
    assert O.gmres(A, b, m=5)["status"] == O.ERR_NONFINITE


def test_jacobi_zero_diagonal_is_an_argument_error(oracle_lib):
    a = np.array([[0.0, 1.0], [1.0, 0.0]])
    A = W.from_dense(a)
    assert O.gmres(A, np.ones(2), m=2, precond=O.PC_JACOBI)["status"] == O.ERR_ARG


# --------------------------------------------------- Section 5.2 protocol (qualitative)
def test_paper_protocol_32bit_formats_match_f64(oracle_lib):
    """b_i = sin(i), x0 = 0, m = 100, tau = 1e-9 (Section 5.2).  Table 2 reports the
    32-bit formats close to the FP64 iteration count (mean ratio 1.02): qualitative
    only -- a 32-bit basis may need one extra restart to turn a converged recurrence
    residual into a converged true residual (Section 5.2), which is what happens here."""
    A = W.convdiff3d(12)
    b = W.rhs_sin(A.n)
    its = {}
    for fmt in ("f64", "f32", "i32"):
        r = O.gmres(A, b, m=100, fmt=O.FORMATS[fmt], precond=O.PC_JACOBI, tol=1e-9, maxit=5000)
        assert r["status"] == O.OK and r["true_relres"] <= 1e-9
        its[fmt] = r["iters"]
    assert its["f64"] <= its["f32"] <= 1.25 * its["f64"]
    assert its["f64"] <= its["i32"] <= 1.25 * its["f64"]


# ---------------------------------------------------------------- block-Jacobi (Section 5.5)
def _block_diag(n, seed):
    rng = np.random.default_rng(seed)
    D = np.zeros((n, n))
    for r0 in range(0, n, 4):
        k = min(4, n - r0)
        D[r0:r0 + k, r0:r0 + k] = rng.standard_normal((k, k)) + 3 * np.eye(k)
    return D


@pytest.mark.parametrize("n", [8, 22, 25])
def test_block_jacobi_exact_on_block_diagonal(n):
    """A block-diagonal A with 4x4 blocks (last block partial): M^{-1} = A^{-1}, so A M^{-1} = I
    and GMRES ends after one step with the exact solution."""
    D = _block_diag(n, n)
    A = W.from_dense(D)
    b = np.random.default_rng(1).standard_normal(n)
    r = O.gmres(A, b, m=10, fmt=O.F64, precond=O.PC_BJ4, tol=1e-12)
    assert r["status"] == O.OK and r["iters"] == 1
    assert np.allclose(r["x"], np.linalg.solve(D, b), rtol=1e-12, atol=1e-14)


def test_block_jacobi_equals_jacobi_when_blocks_are_diagonal():
    """If A has no couplings inside its 4-row blocks, block-Jacobi is scalar Jacobi."""
    rng = np.random.default_rng(3)
    n = 64
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.1)
    blk = np.arange(n) // 4
    M[blk[:, None] == blk[None, :]] = 0.0
    M += np.diag(4.0 + rng.random(n))
    A = W.from_dense(M)
    b = rng.standard_normal(n)
    rj = O.gmres(A, b, m=20, fmt=O.F64, precond=O.PC_JACOBI, tol=1e-11)
    rb = O.gmres(A, b, m=20, fmt=O.F64, precond=O.PC_BJ4, tol=1e-11)
    assert rj["status"] == rb["status"] == O.OK
    assert rj["iters"] == rb["iters"]
    assert np.allclose(rj["x"], rb["x"], rtol=1e-10)


def test_block_jacobi_singular_block_is_an_error():
    D = np.eye(8)
    D[4:8, 4:8] = 1.0
    A = W.from_dense(D)
    r = O.gmres(A, np.ones(8), m=5, fmt=O.F64, precond=O.PC_BJ4, tol=1e-10)
    assert r["status"] == O.ERR_ARG


def test_block_jacobi_reduces_iterations_on_poisson():
    """Block-Jacobi with 4-row blocks contains the x-direction couplings of a 2D Poisson
    grid, so it needs fewer iterations than point Jacobi (which on a constant diagonal
    is no preconditioning at all)."""
    A = W.poisson2d(16, 16)
    b = np.random.default_rng(4).standard_normal(A.n)
    rj = O.gmres(A, b, m=30, fmt=O.F64, precond=O.PC_JACOBI, tol=1e-10)
    rb = O.gmres(A, b, m=30, fmt=O.F64, precond=O.PC_BJ4, tol=1e-10)
    assert rj["status"] == rb["status"] == O.OK
    assert rb["iters"] < rj["iters"]


# -------------------------------------------------- adaptive basis format (reading R15)
def _cd16():
    A = W.convdiff3d(16)
    xs = W.exact_solution(A.n, 2)
    return A, W.rhs_from_solution(A, xs)


def test_adapt_never_moves_f64_and_huge_gap_is_static():
    A, b = _cd16()
    for fmt, gap in ((O.F64, 4.0), (O.E4M3, 1e300), (O.F16, 1e300)):
        r0 = O.gmres(A, b, m=30, fmt=fmt, tol=1e-10)
        r1 = O.gmres(A, b, m=30, fmt=fmt, tol=1e-10, adapt=True, adapt_gap=gap)
        assert r1["promotions"] == 0 and r1["fmt_final"] == fmt
        assert r1["iters"] == r0["iters"] and np.array_equal(r1["x"], r0["x"])


def test_adapt_zero_gap_climbs_the_whole_ladder():
    """gap 0 promotes at every restart: e4m3 -> bf16 -> f32 -> f64, then stays."""
    A, b = _cd16()
    r = O.gmres(A, b, m=8, fmt=O.E4M3, tol=1e-10, adapt=True, adapt_gap=0.0)
    assert r["status"] == O.OK and r["cycles"] >= 4
    assert r["promotions"] == 3 and r["fmt_final"] == O.F64
    r = O.gmres(A, b, m=8, fmt=O.I16, tol=1e-10, adapt=True, adapt_gap=0.0)
    assert r["promotions"] == 2 and r["fmt_final"] == O.F64


def test_adapt_rescues_an_8_bit_basis():
    """The e4m3 basis loses many iterations on conv-diff 16^3; the adaptive solve
    promotes it and needs far fewer, while reaching the same true residual."""
    A, b = _cd16()
    r0 = O.gmres(A, b, m=30, fmt=O.E4M3, tol=1e-10)
    r1 = O.gmres(A, b, m=30, fmt=O.E4M3, tol=1e-10, adapt=True)
    rf = O.gmres(A, b, m=30, fmt=O.F64, tol=1e-10)
    assert r0["status"] == r1["status"] == O.OK
    assert r1["promotions"] >= 1 and r1["iters"] < 0.8 * r0["iters"]
    assert r1["iters"] >= rf["iters"]
    assert r1["true_relres"] <= 1e-10


# ------------------------------------------------ modified Gram-Schmidt variant (Section 2)
def test_gram_schmidt_lauchli_closed_forms(oracle_lib):
    """Lauchli's matrix [1 1 1; d 0 0; 0 d 0; 0 0 d] with d = 1e-8, so that 1 + d^2 rounds
    to 1. Worked by hand in that arithmetic, q1 = (1, d, 0, 0) and q2 = (0, -1, 1, 0)/sqrt 2.
    CGS then gives q3 = (0, -1, 0, 1)/sqrt 2, so q2.q3 = 1/2. MGS gives
    q3 = (0, -1, -1, 2)/sqrt 6, so q2.q3 = 0. This is Bjorck's classic example. A pass
    that took MGS's coefficients from the unreduced w would reproduce CGS and fail."""
    d = 1e-8
    a = np.zeros((4, 3)); a[0, :] = 1.0; a[1, 0] = a[2, 1] = a[3, 2] = d
    q = {}
    for name, ortho in (("cgs", O.ORTHO_CGS), ("mgs", O.ORTHO_MGS)):
        Q = np.zeros((4, 3))
        for k in range(3):
            w = a[:, k].copy()
            if k:
                c, w = O.gram_schmidt_pass(Q[:, :k], w, ortho)
                assert c[0] == 1.0                          # q1 . a_k = 1 exactly
            Q[:, k] = w / np.linalg.norm(w)
        q[name] = Q
    assert np.allclose(q["cgs"][:, 1], np.array([0, -1, 1, 0]) / np.sqrt(2), rtol=0, atol=1e-15)
    assert np.allclose(q["cgs"][:, 2], np.array([0, -1, 0, 1]) / np.sqrt(2), rtol=0, atol=1e-15)
    assert abs(q["cgs"][:, 1] @ q["cgs"][:, 2] - 0.5) <= 1e-15
    assert np.allclose(q["mgs"][:, 2], np.array([0, -1, -1, 2]) / np.sqrt(6), rtol=0, atol=1e-15)
    assert abs(q["mgs"][:, 1] @ q["mgs"][:, 2]) <= 1e-15


def test_gram_schmidt_pass_one_column_and_orthonormal_columns(oracle_lib):
    """Against one column both variants are the same projection. Against orthonormal
    columns they give the same coefficients, V^T w, to rounding."""
    rng = np.random.default_rng(11)
    v = rng.standard_normal(50); v /= np.linalg.norm(v)
    w = rng.standard_normal(50)
    for ortho in (O.ORTHO_CGS, O.ORTHO_MGS):
        c, r = O.gram_schmidt_pass(v[:, None], w, ortho)
        assert abs(c[0] - v @ w) <= 1e-14 * np.linalg.norm(w)
        assert np.allclose(r, w - (v @ w) * v, rtol=0, atol=1e-14)
    Qm, _ = np.linalg.qr(rng.standard_normal((50, 7)))
    c1, r1 = O.gram_schmidt_pass(Qm, w, O.ORTHO_CGS)
    c2, r2 = O.gram_schmidt_pass(Qm, w, O.ORTHO_MGS)
    assert np.allclose(c1, Qm.T @ w, rtol=0, atol=1e-13)
    assert np.allclose(c2, Qm.T @ w, rtol=0, atol=1e-13)
    assert np.allclose(r1, r2, rtol=0, atol=1e-13)


@pytest.mark.parametrize("reorth", [O.REORTH_ALWAYS, O.REORTH_NEVER])
def test_mgs_iterates_are_krylov_minimisers(oracle_lib, reorth):
    """MGS builds the same Krylov space. Each iterate is still the dense least-squares
    minimiser over it, and the Givens recurrence gives that minimiser's residual."""
    n = 30
    a = _rand_nonsym(n, 6, shift=2.0) + np.diag(np.linspace(0.5, 4, n))
    A = W.from_dense(a)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(n); x0 = rng.standard_normal(n) * 0.1
    bn = np.linalg.norm(b)
    for k in range(1, 9):
        r = O.gmres(A, b, x0, m=20, tol=0.0, maxit=k, hist_cap=k, reorth=reorth, ortho=O.ORTHO_MGS)
        xk, resk = _krylov_ls(a, np.eye(n), b, x0, k)
        assert np.linalg.norm(r["x"] - xk) <= 1e-10 * np.linalg.norm(xk)
        assert abs(r["hist"][k - 1] - resk / bn) <= 1e-12


def test_mgs_arnoldi_relation_and_orthogonality(oracle_lib):
    """A V_k = V_{k+1} H_k and V^T V = I hold for the MGS basis (f64 codes, one
    re-orthogonalisation pass). Its Hessenberg matrix equals the CGS one to rounding."""
    A = W.convdiff3d(8)
    a = A.dense()
    b = W.rhs_sin(A.n)
    k = 40
    rm = O.gmres(A, b, m=k, tol=0.0, maxit=k, want_H1=True, want_V1=True, ortho=O.ORTHO_MGS)
    rc = O.gmres(A, b, m=k, tol=0.0, maxit=k, want_H1=True, ortho=O.ORTHO_CGS)
    V, H = rm["V1"], rm["H1"][: k + 1, :k]
    assert np.linalg.norm(a @ V[:, :k] - V @ H) <= 1e-13 * np.linalg.norm(a, 2) * np.sqrt(k)
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V, 2) <= 1e-13
    for j in range(k):
        hm, hc = rm["H1"][: j + 2, j], rc["H1"][: j + 2, j]
        assert np.linalg.norm(hm - hc) <= 1e-12 * np.linalg.norm(hc), j


def test_blocked_inner_product_reading_r19():
    """Inner products follow reading R19 exactly: index order within blocks of 4096 terms,
    then the block sums in block order (a pure-Python restatement gives the same bits);
    integer-valued data sums exactly."""
    rng = np.random.default_rng(19)
    n = 3 * 4096 + 1234 + 40000          # several blocks, a ragged last block, > the threading threshold
    a = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
    b = rng.standard_normal(n)
    ref = 0.0
    for k0 in range(0, n, 4096):
        s = 0.0
        for i in range(k0, min(n, k0 + 4096)):
            s += float(a[i]) * float(b[i])
        ref += s
    assert O.dot(a, b) == ref
    ai = rng.integers(-2 ** 20, 2 ** 20, n).astype(np.float64)
    bi = rng.integers(-2 ** 10, 2 ** 10, n).astype(np.float64)
    assert O.dot(ai, bi) == float(int(np.dot(ai.astype(np.int64), bi.astype(np.int64))))
    assert O.dot(a[:0], b[:0]) == 0.0


def test_oracle_results_do_not_depend_on_thread_count():
    """The oracle's parallel loops split only work whose result does not depend on the
    split (rows, elements, fixed inner-product blocks): 1, 3 and all threads give the same
    bits for x, the Hessenberg matrix and the iteration count."""
    import os
    A = W.convdiff3d(40)                 # n = 64,000: above the threading threshold
    xs = W.exact_solution(A.n, 2)
    b = W.rhs_from_solution(A, xs)
    runs = []
    try:
        for t in (1, 3, os.cpu_count() or 2):
            O.set_threads(t)
            runs.append(O.gmres(A, b, m=30, fmt=O.F16, tol=1e-10, maxit=70, want_H1=True))
    finally:
        O.set_threads(os.cpu_count() or 1)
    for r in runs[1:]:
        assert r["iters"] == runs[0]["iters"]
        assert np.array_equal(r["x"], runs[0]["x"])
        assert np.array_equal(r["H1"], runs[0]["H1"])
