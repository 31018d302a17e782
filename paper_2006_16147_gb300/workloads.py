"""Seeded synthetic inputs shaped like the paper's model problems.

Holds input generation only: stencil assembly of the test matrices, smooth
vectors and right-hand sides. Nothing of the AMG method (weights, matching,
aggregation, Galerkin products, smoothing, Krylov iteration) lives here, so the
same arrays can be handed both to the CUDA library and to the CPU oracle.

Matrices follow the model problem of Section 4 (Eq. 8): -div(K grad u) = f on
the unit cube, homogeneous Dirichlet conditions, 7-point finite differences,
lexicographic ordering ``i + nx*(j + ny*k)`` with the Dirichlet nodes
eliminated. The stencil is left unscaled (diagonal 6, neighbours -1 for K = 1).
The anisotropic variant follows the supplementary anisotropic Poisson problem.

All arrays are numpy: CSR ``row_ptr`` (int32, n+1), ``col`` (int32, nnz,
ascending within each row) and ``val`` (float64, nnz).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Csr",
    "poisson3d",
    "poisson2d_aniso",
    "aniso3d",
    "varcoef3d",
    "csr_matvec",
    "rhs_ones",
    "rhs_uniform",
    "rhs_normal",
    "batch_edges",
    "block_diagonal",
    "random_spd",
    "random_spd_sparse",
    "with_hubs",
]


class Csr:
    """A square CSR matrix held as three numpy arrays."""

    __slots__ = ("n", "row_ptr", "col", "val", "name")

    def __init__(self, row_ptr, col, val, name=""):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = int(self.row_ptr.shape[0] - 1)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def _assemble_faces(cx, cy, cz, name):
    """Assemble the 7-point operator from face coefficients.

    ``cx`` has shape (nz, ny, nx+1): cx[k, j, i] couples nodes i-1 and i along x
    (i = 0 and i = nx are faces to eliminated Dirichlet nodes). ``cy`` is
    (nz, ny+1, nx) and ``cz`` is (nz+1, ny, nx) likewise. Row entries are
    emitted in ascending column order: -z, -y, -x, diagonal, +x, +y, +z.
    """
    nz, ny, nxp = cx.shape
    nx = nxp - 1
    n = nx * ny * nz
    diag = (cx[:, :, :-1] + cx[:, :, 1:]) + (cy[:, :-1, :] + cy[:, 1:, :]) + (cz[:-1] + cz[1:])
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = k.ravel(); j = j.ravel(); i = i.ravel()
    idx = np.arange(n, dtype=np.int64)
    slots = [
        (k > 0, -nx * ny, -cz[:-1].ravel()),
        (j > 0, -nx, -cy[:, :-1, :].ravel()),
        (i > 0, -1, -cx[:, :, :-1].ravel()),
        (np.ones(n, dtype=bool), 0, diag.ravel()),
        (i < nx - 1, 1, -cx[:, :, 1:].ravel()),
        (j < ny - 1, nx, -cy[:, 1:, :].ravel()),
        (k < nz - 1, nx * ny, -cz[1:].ravel()),
    ]
    counts = np.zeros(n, dtype=np.int64)
    for mask, _, _ in slots:
        counts += mask
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    if nnz > 2**31 - 1:
        raise ValueError("nnz exceeds int32")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = row_ptr[:-1].copy()
    for mask, off, v in slots:
        p = pos[mask]
        col[p] = (idx[mask] + off).astype(np.int32)
        val[p] = v[mask]
        pos[mask] += 1
    return Csr(row_ptr.astype(np.int32), col, val, name)


def poisson3d(nx: int, ny: int | None = None, nz: int | None = None) -> Csr:
    """7-point Laplacian on an nx*ny*nz interior grid (K = 1 in Eq. 8)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    cx = np.ones((nz, ny, nx + 1))
    cy = np.ones((nz, ny + 1, nx))
    cz = np.ones((nz + 1, ny, nx))
    return _assemble_faces(cx, cy, cz, f"poisson3d_{nx}x{ny}x{nz}")


def poisson2d_aniso(nx: int, ny: int | None = None, eps: float = 1e-2) -> Csr:
    """5-point discretisation of -u_xx - eps*u_yy on an nx*ny interior grid."""
    ny = nx if ny is None else ny
    cx = np.ones((1, ny, nx + 1))
    cy = np.full((1, ny + 1, nx), float(eps))
    cz = np.zeros((2, ny, nx))
    A = _assemble_faces(cx, cy, cz, f"aniso2d_{nx}x{ny}_eps{eps:g}")
    return A


def aniso3d(nx: int, ny: int | None = None, nz: int | None = None, k=(100.0, 100.0, 1.0)) -> Csr:
    """7-point discretisation of -(k1 u_xx + k2 u_yy + k3 u_zz) (the supplementary
    anisotropic Poisson problem; k = (100, 100, 1) as in its experiments,
    (1, 1, 100) for z-aligned anisotropy)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    cx = np.full((nz, ny, nx + 1), float(k[0]))
    cy = np.full((nz, ny + 1, nx), float(k[1]))
    cz = np.full((nz + 1, ny, nx), float(k[2]))
    return _assemble_faces(cx, cy, cz, f"aniso3d_{nx}x{ny}x{nz}_k{k[0]:g}-{k[1]:g}-{k[2]:g}")


def varcoef3d(nx: int, seed: int, sigma: float = 2.0) -> Csr:
    """Jump-coefficient diffusion: log-coefficient g ~ N(0, sigma^2) per node.

    g is drawn on the (nx+2)^3 grid that includes the Dirichlet nodes; each face
    carries the harmonic mean of exp(g) at its two nodes.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.normal(0.0, sigma, size=(nx + 2, nx + 2, nx + 2))
    kap = np.exp(g)

    def hm(a, b):
        return 2.0 * a * b / (a + b)

    inner = kap[1:-1, 1:-1, 1:-1]
    cx = hm(kap[1:-1, 1:-1, :-1], kap[1:-1, 1:-1, 1:])      # (nz, ny, nx+1)
    cy = hm(kap[1:-1, :-1, 1:-1], kap[1:-1, 1:, 1:-1])      # (nz, ny+1, nx)
    cz = hm(kap[:-1, 1:-1, 1:-1], kap[1:, 1:-1, 1:-1])      # (nz+1, ny, nx)
    del inner
    return _assemble_faces(cx, cy, cz, f"varcoef3d_{nx}_s{seed}")


def csr_matvec(A: Csr, x: np.ndarray) -> np.ndarray:
    """y = A x, used to manufacture right-hand sides b = A x*."""
    return A.scipy() @ np.asarray(x, dtype=np.float64)


def rhs_ones(A: Csr):
    """b = A * ones (exact solution ones), x0 = 0."""
    xs = np.ones(A.n)
    return csr_matvec(A, xs), xs


def rhs_uniform(A: Csr, seed: int):
    """x* ~ U[-1, 1] (PCG64 seed), b = A x*."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(-1.0, 1.0, size=A.n)
    return csr_matvec(A, xs), xs


def rhs_normal(n: int, seed: int, k: int | None = None) -> np.ndarray:
    """Entries N(0, 1); shape (n,) or row-major (n, k)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, 1.0, size=(n,) if k is None else (n, k))


def batch_edges(m: int, seed: int, lo: int = 16, hi: int = 64) -> list[int]:
    """Grid edge lengths of m independent Poisson systems, uniform in lo..hi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(e) for e in rng.integers(lo, hi + 1, size=m)]


def block_diagonal(mats: list) -> tuple:
    """Union of systems as one block-diagonal CSR; returns (Csr, row offsets)."""
    offs = np.zeros(len(mats) + 1, dtype=np.int64)
    for i, M in enumerate(mats):
        offs[i + 1] = offs[i] + M.n
    nnz = np.zeros(len(mats) + 1, dtype=np.int64)
    for i, M in enumerate(mats):
        nnz[i + 1] = nnz[i] + M.nnz
    rp = np.concatenate([M.row_ptr[:-1].astype(np.int64) + nnz[i] for i, M in enumerate(mats)] + [[nnz[-1]]])
    col = np.concatenate([M.col.astype(np.int64) + offs[i] for i, M in enumerate(mats)])
    val = np.concatenate([M.val for M in mats])
    return Csr(rp, col, val, "block_diagonal"), offs.astype(np.int32)


def random_spd(n: int, density: float, seed: int) -> Csr:
    """Small random sparse SPD matrix (structurally symmetric, diagonally dominant).

    Off-diagonal values are negative or positive at random; the diagonal is the
    absolute row sum plus a random positive margin, so the matrix is SPD.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = rng.random((n, n)) < density
    mask = np.triu(mask, 1)
    vals = rng.uniform(-1.0, 1.0, size=(n, n)) * mask
    d = vals + vals.T
    d[np.diag_indices(n)] = np.abs(d).sum(axis=1) + rng.uniform(0.1, 1.0, size=n)
    rows, cols = np.nonzero(d)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Csr(row_ptr.astype(np.int32), cols.astype(np.int32), d[rows, cols], f"random_spd_{n}_{seed}")


def random_spd_sparse(n: int, k: int, seed: int) -> Csr:
    """Random sparse SPD matrix without a dense mask: each row draws k random
    partners, the pattern is symmetrised, off-diagonal values are uniform in
    [-1, 1] (symmetric), the diagonal is the absolute row sum plus a margin in
    [0.1, 1]."""
    import scipy.sparse as sp
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = np.repeat(np.arange(n), k)
    cols = rng.integers(0, n, size=n * k)
    keep = rows != cols
    rows, cols = rows[keep], cols[keep]
    vals = rng.uniform(-1.0, 1.0, size=rows.shape[0])
    U = sp.coo_matrix((vals, (np.minimum(rows, cols), np.maximum(rows, cols))), shape=(n, n)).tocsr()
    U.sum_duplicates()
    S = (U + U.T).tocsr()
    d = np.asarray(abs(S).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, size=n)
    M = (S + sp.diags(d)).tocsr()
    M.sort_indices()
    return Csr(M.indptr, M.indices, M.data, f"random_spd_sparse_{n}_{k}_{seed}")


def with_hubs(A: Csr, sizes, seed: int) -> Csr:
    """A with hub unknowns appended: hub h couples to sizes[h] distinct random
    unknowns of A with values -U(0.1, 1) (symmetric). Every diagonal grows by
    the absolute values added to its row, so a diagonally dominant A stays
    SPD; a hub's diagonal is its absolute row sum times 1.5."""
    import scipy.sparse as sp
    rng = np.random.Generator(np.random.PCG64(seed))
    n, m = A.n, len(sizes)
    rows, cols, vals = [], [], []
    for h, k in enumerate(sizes):
        nb = np.sort(rng.choice(n, size=int(k), replace=False))
        rows.append(nb)
        cols.append(np.full(nb.shape[0], h))
        vals.append(-rng.uniform(0.1, 1.0, size=nb.shape[0]))
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, m)).tocsr()
    extra = np.asarray(abs(B).sum(axis=1)).ravel()
    hub_d = 1.5 * np.asarray(abs(B).sum(axis=0)).ravel()
    M = sp.bmat([[A.scipy() + sp.diags(extra), B], [B.T, sp.diags(hub_d)]]).tocsr()
    M.sort_indices()
    return Csr(M.indptr, M.indices, M.data, f"{A.name}_hubs{m}_{seed}")
