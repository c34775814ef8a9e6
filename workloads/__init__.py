"""Seeded synthetic inputs for compressed-basis GMRES (shared by the oracle tests,
the CUDA-path tests and the benchmark).

This module only *builds inputs*: sparse matrices in CSR form, exact solutions and
right-hand sides.  It contains none of the solver's arithmetic (no Arnoldi step, no
orthogonalisation, no codec).  The right-hand side b = A x* is formed with a plain
scipy sparse product, which is input synthesis, not part of the method.

Matrices (all CSR, int32 row pointers / column indices, float64 values, columns
sorted within each row, rows in lexicographic x-fastest order):

* ``poisson2d(nx, ny)``      5-point -Laplace on an nx x ny interior grid, Dirichlet,
                              scaled by h^2 (diag 4, neighbours -1).
* ``convdiff3d(N, pe)``      7-point -Laplace + beta . grad u with beta = pe*(1, 0.5, 0.25),
                              first-order upwind (backward differences since beta > 0),
                              h = 1/(N+1), scaled by h^2: diag 6 + h*sum(beta),
                              west/south/down -1 - h*beta_d, east/north/up -1.
* ``random27(n, delta)``     nonsymmetric: band offsets -4..4 plus random distinct
                              columns outside the band, 27 entries per row, off-diagonal
                              N(0,1), diagonal (1+delta) * sum |off-diagonal|.
* ``stencil_batch(...)``     uneven batch of weighted-Laplacian 2D/3D grids with
                              lognormal edge conductances and Dirichlet boundary edges.
* ``diffusion3d_cc(N)``      cell-centred diffusion with a lognormal(0,1) cell field,
                              harmonic-mean face coefficients, Dirichlet boundary.

Seeds: numpy PCG64 with seed 20201201 + config id (configs 1..5 in the order
Poisson 64^2, conv-diff 128^3, random n=2^20, batch of 512, learned-preconditioner 96^3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

SEED_BASE = 20201201


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def _from_coo(n, rows, cols, vals) -> CSR:
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64))


def from_dense(a: np.ndarray) -> CSR:
    """CSR of a small dense matrix (explicit zeros dropped)."""
    m = sp.csr_matrix(np.asarray(a, dtype=np.float64))
    m.eliminate_zeros()
    m.sort_indices()
    return CSR(a.shape[0], m.indptr.astype(np.int32), m.indices.astype(np.int32),
               m.data.astype(np.float64))


def rng(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_id + 1000 * salt))


# ----------------------------------------------------------------------------- stencils
def poisson2d(nx: int, ny: int | None = None) -> CSR:
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 4.0)]
    for dy, dx in ((0, -1), (0, 1), (-1, 0), (1, 0)):
        src = idx[max(0, -dy):ny - max(0, dy), max(0, -dx):nx - max(0, dx)]
        dst = idx[max(0, -dy) + dy:ny - max(0, dy) + dy, max(0, -dx) + dx:nx - max(0, dx) + dx]
        rows.append(src.ravel()); cols.append(dst.ravel()); vals.append(np.full(src.size, -1.0))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def convdiff3d(N: int, pe: float = 10.0, beta=(1.0, 0.5, 0.25)) -> CSR:
    n = N ** 3
    h = 1.0 / (N + 1)
    bx, by, bz = (pe * b for b in beta)
    idx = np.arange(n).reshape(N, N, N)  # [z, y, x], x fastest
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 6.0 + h * (bx + by + bz))]
    # (axis, step, coefficient): backward neighbour gets the upwind term
    for axis, bcoef in ((2, bx), (1, by), (0, bz)):
        for step, coef in ((-1, -1.0 - h * bcoef), (1, -1.0)):
            sl_src = [slice(None)] * 3
            sl_dst = [slice(None)] * 3
            if step < 0:
                sl_src[axis] = slice(1, N); sl_dst[axis] = slice(0, N - 1)
            else:
                sl_src[axis] = slice(0, N - 1); sl_dst[axis] = slice(1, N)
            s = idx[tuple(sl_src)].ravel(); d = idx[tuple(sl_dst)].ravel()
            rows.append(s); cols.append(d); vals.append(np.full(s.size, coef))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def random27(n: int, delta: float, config_id: int = 3, per_row: int = 27, band: int = 4) -> CSR:
    g = rng(config_id, salt=int(round(delta * 1000)))
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(i - band, 0)
    hi = np.minimum(i + band, n - 1)
    nb = (hi - lo + 1)
    nextra = per_row - nb
    if n < per_row:
        raise ValueError("random27 needs n >= per_row")
    maxe = int(nextra.max())
    # draw candidates outside the band: uniform over [0, n - nb) then skip the band
    extra = np.full((n, maxe), -1, dtype=np.int64)
    need = np.ones((n, maxe), dtype=bool)
    need &= np.arange(maxe)[None, :] < nextra[:, None]
    for _ in range(100):
        rows_need = np.nonzero(need.any(axis=1))[0]
        if rows_need.size == 0:
            break
        r = rows_need
        u = g.integers(0, n - nb[r][:, None], size=(r.size, maxe))
        c = np.where(u >= lo[r][:, None], u + nb[r][:, None], u)
        cur = extra[r]
        cur = np.where(need[r], c, cur)
        # resolve duplicates within a row: keep first occurrence
        srt = np.sort(np.where(cur < 0, -1 - np.arange(maxe)[None, :], cur), axis=1)
        dup_rows = (np.diff(srt, axis=1) == 0).any(axis=1)
        extra[r] = cur
        need[r] = False
        if dup_rows.any():
            rr = r[dup_rows]
            for k in rr:  # rare: re-draw duplicate slots of these rows
                row = extra[k, :nextra[k]]
                _, first = np.unique(row, return_index=True)
                mask = np.ones(nextra[k], dtype=bool); mask[first] = False
                need[k, :nextra[k]] = mask
    assert not need.any()
    offs = np.arange(-band, band + 1)
    bc = i[:, None] + offs[None, :]
    bmask = (bc >= 0) & (bc < n)
    rows = np.concatenate([np.repeat(i, bmask.sum(axis=1)),
                           np.repeat(i, nextra)])
    cols = np.concatenate([bc[bmask], extra[np.arange(maxe)[None, :] < nextra[:, None]]])
    vals = g.standard_normal(rows.size)
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sort_indices()
    assert m.nnz == n * per_row, (m.nnz, n * per_row)
    # diagonal = (1 + delta) * sum |off-diagonal| of the row
    r_of = np.repeat(np.arange(n), np.diff(m.indptr))
    isdiag = m.indices == r_of
    offsum = np.bincount(r_of, weights=np.where(isdiag, 0.0, np.abs(m.data)), minlength=n)
    m.data[isdiag] = (1.0 + delta) * offsum
    return CSR(n, m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64))


def _weighted_laplacian(shape, g: np.random.Generator, sigma: float) -> CSR:
    """Graph Laplacian of a grid with lognormal(0, sigma) edge conductances, plus one
    Dirichlet boundary edge (also lognormal) for every missing grid neighbour."""
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    d = len(shape)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for axis in range(d):
        sl_a = [slice(None)] * d; sl_b = [slice(None)] * d
        sl_a[axis] = slice(0, shape[axis] - 1); sl_b[axis] = slice(1, shape[axis])
        a = idx[tuple(sl_a)].ravel(); b = idx[tuple(sl_b)].ravel()
        c = g.lognormal(0.0, sigma, size=a.size)
        rows += [a, b]; cols += [b, a]; vals += [-c, -c]
        np.add.at(diag, a, c); np.add.at(diag, b, c)
        # Dirichlet boundary edges on both faces of this axis
        for face in (0, shape[axis] - 1):
            sl = [slice(None)] * d; sl[axis] = face
            f = idx[tuple(sl)].ravel()
            np.add.at(diag, f, g.lognormal(0.0, sigma, size=f.size))
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def stencil_batch(nsys: int = 512, nmin: int = 1024, nmax: int = 65536, sigma: float = 0.5,
                  config_id: int = 4) -> list[CSR]:
    """Uneven batch: n_k log-uniform in [nmin, nmax], 2D (side round(sqrt n_k)) or 3D
    (side round(cbrt n_k)) by a coin flip, lognormal edge conductances."""
    g = rng(config_id)
    out = []
    for _ in range(nsys):
        nk = math.exp(g.uniform(math.log(nmin), math.log(nmax)))
        if g.random() < 0.5:
            s = max(2, int(round(math.sqrt(nk)))); shape = (s, s)
        else:
            s = max(2, int(round(nk ** (1.0 / 3.0)))); shape = (s, s, s)
        out.append(_weighted_laplacian(shape, g, sigma))
    return out


def diffusion3d_cc(N: int, sigma: float = 1.0, config_id: int = 5) -> tuple[CSR, np.ndarray]:
    """Cell-centred -div(kappa grad u) on N^3 cells, kappa ~ lognormal(0, sigma) per cell,
    face coefficient = harmonic mean of the two cells, boundary faces 2*kappa_c
    (Dirichlet at half a cell).  Returns (A, kappa)."""
    g = rng(config_id)
    n = N ** 3
    kap = g.lognormal(0.0, sigma, size=(N, N, N))
    idx = np.arange(n).reshape(N, N, N)
    diag = np.zeros((N, N, N))
    rows, cols, vals = [], [], []
    for axis in range(3):
        sl_a = [slice(None)] * 3; sl_b = [slice(None)] * 3
        sl_a[axis] = slice(0, N - 1); sl_b[axis] = slice(1, N)
        ka = kap[tuple(sl_a)]; kb = kap[tuple(sl_b)]
        face = 2.0 * ka * kb / (ka + kb)
        diag[tuple(sl_a)] += face; diag[tuple(sl_b)] += face
        a = idx[tuple(sl_a)].ravel(); b = idx[tuple(sl_b)].ravel()
        rows += [a, b]; cols += [b, a]; vals += [-face.ravel(), -face.ravel()]
        for f in (0, N - 1):
            sl = [slice(None)] * 3; sl[axis] = f
            diag[tuple(sl)] += 2.0 * kap[tuple(sl)]
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag.ravel())
    A = _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return A, kap


# ----------------------------------------------------------------------------- vectors
def exact_solution(n: int, config_id: int, salt: int = 7) -> np.ndarray:
    return rng(config_id, salt=salt).uniform(-1.0, 1.0, size=n)


def rhs_from_solution(A: CSR, xstar: np.ndarray) -> np.ndarray:
    return A.to_scipy() @ xstar


def rhs_sin(n: int) -> np.ndarray:
    """Right-hand side b_i = sin(i), i = 1..n (Section 5.2 accuracy protocol)."""
    return np.sin(np.arange(1, n + 1, dtype=np.float64))


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.Generator(np.random.PCG64(SEED_BASE + seed)).uniform(lo, hi, size=n)


# ----------------------------------------------------------------------------- configs
CONFIGS = {
    1: dict(name="poisson2d_64x64_f64_m100", restart=100, tol=1e-10),
    2: dict(name="convdiff3d_128_pe10_m100", restart=100, tol=1e-10),
    3: dict(name="random27_n1M", restart=100, tol=1e-10),
    4: dict(name="batch512_stencil_m30", restart=30, tol=1e-8),
    5: dict(name="learned_pc_diffusion96", restart=100, tol=1e-10),
}


def config_matrix(cid: int, scale: int | None = None):
    """Matrix of config `cid`; `scale` shrinks the grid for fast tests."""
    if cid == 1:
        return poisson2d(scale or 64)
    if cid == 2:
        return convdiff3d(scale or 128)
    if cid == 3:
        return random27(scale or (1 << 20), 0.1)
    if cid == 5:
        return diffusion3d_cc(scale or 96)[0]
    raise ValueError(cid)
