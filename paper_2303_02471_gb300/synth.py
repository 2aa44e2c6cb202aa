"""Seeded synthetic CSC inputs shaped like the workloads of arXiv 2303.02471.

This module only draws inputs. It holds none of the product's arithmetic, so
the CPU oracle (``oracle/``) and the CUDA path both take their inputs from
here and share nothing else.

CSC layout everywhere (Section 2.1 of the paper): ``colptr`` int64 of length
``ncols + 1`` with ``colptr[0] == 0`` and ``colptr[-1] == nnz``, ``rowidx``
int32 of length ``nnz``, ``values`` float64 (or float32) of length ``nnz``.

Generators (all numpy ``default_rng`` / PCG64):

* :func:`lap2d` -- 5-point Dirichlet Laplacian on a g x g grid (workload 1).
* :func:`random_z` -- n x n, per column Z ~ U{zmin..zmax} distinct rows placed
  uniformly, the paper's synthetic scheme of Section 5.2 (workloads 2 and 4).
* :func:`rmat` -- R-MAT power-law pattern with a per-column cap (workload 3).
* :func:`batch_pairs` -- 512 independent uneven pairs (workload 4).
* :func:`lap3d`, :func:`prolongation`, :func:`perturbation` -- Galerkin
  product inputs (workload 5).
* :func:`fuzz_pair` -- tiny seeded pairs with the degenerate shapes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSC:
    """A host CSC matrix (Section 2.1): values / row_indices / column_pointers."""

    nrows: int
    ncols: int
    colptr: np.ndarray  # int64 [ncols + 1]
    rowidx: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1]) if self.ncols >= 0 and len(self.colptr) else 0

    def astype(self, dtype) -> "CSC":
        return CSC(self.nrows, self.ncols, self.colptr, self.rowidx,
                   self.values.astype(dtype))

    def with_values(self, values: np.ndarray) -> "CSC":
        return CSC(self.nrows, self.ncols, self.colptr, self.rowidx, values)


def _from_sorted_cols(nrows: int, ncols: int, counts: np.ndarray,
                      rows: np.ndarray, values: np.ndarray) -> CSC:
    colptr = np.zeros(ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    return CSC(nrows, ncols, colptr, rows.astype(np.int32, copy=False),
               values)


def from_coo(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray,
             values: np.ndarray) -> CSC:
    """CSC from COO triplets with no duplicate (row, col); rows sorted per column."""
    order = np.lexsort((rows, cols))
    rows = np.asarray(rows)[order]
    cols = np.asarray(cols)[order]
    values = np.asarray(values)[order]
    counts = np.bincount(cols, minlength=ncols).astype(np.int64)
    return _from_sorted_cols(nrows, ncols, counts, rows, values)


# ---------------------------------------------------------------- workload 1
def lap2d(g: int, seed: int | None = 0, stencil_values: bool = False) -> CSC:
    """5-point Laplacian of a g x g Dirichlet grid; node (x, y) is row y*g + x.

    With ``stencil_values`` the entries are 4 (diagonal) and -1 (neighbours);
    otherwise they are U[-1, 1] drawn from ``seed`` in CSC storage order.
    """
    n = g * g
    idx = np.arange(n)
    x, y = idx % g, idx // g
    rows, cols, diag = [], [], []
    for dx, dy in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g)
        rows.append((idx + dx + dy * g)[ok])
        cols.append(idx[ok])
        diag.append(np.full(int(ok.sum()), dx == 0 and dy == 0))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    diag = np.concatenate(diag)
    base = from_coo(n, n, rows, cols, diag.astype(np.float64))
    if stencil_values:
        vals = np.where(base.values > 0, 4.0, -1.0)
    else:
        vals = np.random.default_rng(seed).uniform(-1.0, 1.0, base.nnz)
    return base.with_values(vals)


# ------------------------------------------------------- workloads 2 and 4
def _distinct_rows(rng: np.random.Generator, n_rows: int, z: np.ndarray,
                   zmax: int) -> np.ndarray:
    """Per column, z[j] distinct rows drawn uniformly from [0, n_rows).

    Draws a padded (ncols, zmax) table, sorts each column and redraws the
    duplicated entries until none is left; returns the table with padding
    set to ``n_rows`` (sorted last)."""
    ncols = z.shape[0]
    pad = np.arange(zmax)[None, :] >= z[:, None]
    tab = rng.integers(0, n_rows, size=(ncols, zmax), dtype=np.int64)
    tab[pad] = n_rows
    while True:
        tab.sort(axis=1)
        dup = np.zeros_like(pad)
        dup[:, 1:] = (tab[:, 1:] == tab[:, :-1]) & (tab[:, 1:] < n_rows)
        k = int(dup.sum())
        if k == 0:
            return tab
        tab[dup] = rng.integers(0, n_rows, size=k, dtype=np.int64)


def random_z(n: int, zmin: int, zmax: int, seed: int,
             dtype=np.float64) -> CSC:
    """n x n matrix, each column Z ~ U{zmin..zmax} distinct uniform rows, N(0,1)
    values (Section 5.2's synthetic scheme; constant Z when zmin == zmax).

    Draw order from ``default_rng(seed)``: Z per column, the rows (with
    redraws), then the values in CSC storage order."""
    rng = np.random.default_rng(seed)
    z = rng.integers(zmin, zmax + 1, size=n)
    tab = _distinct_rows(rng, n, z, zmax)
    rows = tab[tab < n]
    vals = rng.standard_normal(rows.shape[0]).astype(dtype)
    return _from_sorted_cols(n, n, z.astype(np.int64), rows, vals)


# ---------------------------------------------------------------- workload 3
def rmat(scale: int, edge_factor: int = 8, abcd=(0.57, 0.19, 0.19, 0.05),
         seed: int = 0, col_cap: int | None = 2000) -> CSC:
    """R-MAT pattern with 2^scale rows/columns, U[-1, 1] values.

    ``edge_factor * n`` edges are drawn one quadrant per level (a: row bit 0,
    col bit 0; b: 0/1; c: 1/0; d: 1/1), duplicates are dropped (self loops
    kept, no relabelling), and each column is cut to ``col_cap`` entries by a
    seeded random subset."""
    a, b, c, _ = abcd
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    r = np.zeros(m, dtype=np.int64)
    col = np.zeros(m, dtype=np.int64)
    for _ in range(scale):
        u = rng.random(m)
        rb = (u >= a + b).astype(np.int64)
        cb = (((u >= a) & (u < a + b)) | (u >= a + b + c)).astype(np.int64)
        r = 2 * r + rb
        col = 2 * col + cb
    key = np.unique(col * n + r)
    col, r = key // n, key % n
    counts = np.bincount(col, minlength=n).astype(np.int64)
    if col_cap is not None and counts.max() > col_cap:
        start = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=start[1:])
        keep = np.ones(r.shape[0], dtype=bool)
        for j in np.nonzero(counts > col_cap)[0]:
            drop = rng.permutation(int(counts[j]))[col_cap:]
            keep[start[j] + drop] = False
        r = r[keep]
        counts = np.minimum(counts, col_cap)
    vals = rng.uniform(-1.0, 1.0, r.shape[0])
    return _from_sorted_cols(n, n, counts, r, vals)


# ---------------------------------------------------------------- workload 4
def batch_pairs(count: int = 512, seed: int = 0, n_lo: int = 500,
                n_hi: int = 20000, z_lo: int = 2, z_hi: int = 40,
                n_scale: float = 1.0):
    """``count`` independent pairs (A_i, B_i), both n_i x n_i with exactly Z_i
    entries per column; n_i = round(exp(U[ln n_lo, ln n_hi])) * n_scale,
    Z_i ~ U{z_lo..z_hi}; the first half float64, the second half float32.

    ``n_scale`` < 1 shrinks every matrix (same Z mix) for small test cases."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)))
    ns = np.maximum(np.rint(ns * n_scale), z_hi).astype(np.int64)
    zs = rng.integers(z_lo, z_hi + 1, size=count)
    pairs = []
    for i in range(count):
        n, z = int(ns[i]), int(zs[i])
        dt = np.float64 if i < count // 2 else np.float32
        mats = []
        for _ in range(2):
            tab = _distinct_rows(rng, n, np.full(n, z), z)
            vals = rng.standard_normal(n * z).astype(dt)
            mats.append(_from_sorted_cols(n, n, np.full(n, z, np.int64),
                                          tab.reshape(-1), vals))
        pairs.append((mats[0], mats[1]))
    return pairs


# ---------------------------------------------------------------- workload 5
def lap3d(g: int) -> CSC:
    """7-point Laplacian (6 on the diagonal, -1 off) of a g^3 Dirichlet grid;
    node (x, y, z) is row x + g*y + g*g*z."""
    n = g ** 3
    idx = np.arange(n)
    x, y, z = idx % g, (idx // g) % g, idx // (g * g)
    rows, cols, vals = [], [], []
    for d, v in (((0, 0, 0), 6.0), ((-1, 0, 0), -1.0), ((1, 0, 0), -1.0),
                 ((0, -1, 0), -1.0), ((0, 1, 0), -1.0), ((0, 0, -1), -1.0),
                 ((0, 0, 1), -1.0)):
        dx, dy, dz = d
        ok = ((x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g)
              & (z + dz >= 0) & (z + dz < g))
        rows.append((idx + dx + dy * g + dz * g * g)[ok])
        cols.append(idx[ok])
        vals.append(np.full(int(ok.sum()), v))
    return from_coo(n, n, np.concatenate(rows), np.concatenate(cols),
                    np.concatenate(vals))


def prolongation(g: int, seed: int = 0) -> CSC:
    """Aggregation prolongation P of shape g^3 x (g/2)^3.

    Row (x, y, z) has an entry in column agg(x//2, y//2, z//2); with
    probability 1/2 it gets a second entry in the aggregate next to it along
    a random axis and sign (the sign is flipped at the grid edge, so the two
    columns always differ). Values U[0.5, 1] in CSC storage order."""
    assert g % 2 == 0
    h = g // 2
    n = g ** 3
    rng = np.random.default_rng(seed)
    coin = rng.random(n) < 0.5
    axis = rng.integers(0, 3, size=n)
    sign = np.where(rng.random(n) < 0.5, -1, 1)
    idx = np.arange(n)
    ac = np.stack([(idx % g) // 2, ((idx // g) % g) // 2, (idx // (g * g)) // 2])
    agg = ac[0] + h * ac[1] + h * h * ac[2]
    nb = ac.copy()
    sel = (axis[None, :] == np.arange(3)[:, None])
    moved = nb + sel * sign[None, :]
    out = (moved < 0) | (moved >= h)
    moved = np.where(out, nb - sel * sign[None, :], moved)
    agg2 = moved[0] + h * moved[1] + h * h * moved[2]
    rows = np.concatenate([idx, idx[coin]])
    cols = np.concatenate([agg, agg2[coin]])
    base = from_coo(n, h ** 3, rows, cols, np.zeros(rows.shape[0]))
    vals = rng.uniform(0.5, 1.0, base.nnz)
    return base.with_values(vals)


def perturbation(nnz: int, seed: int = 1) -> np.ndarray:
    """Factors 1 + 0.01 * U[-1, 1], one per stored entry of C in sorted CSC
    order; the loss target is T = C(P0) * factors on pattern(C)."""
    return 1.0 + 0.01 * np.random.default_rng(seed).uniform(-1.0, 1.0, nnz)


# ------------------------------------------------------------- fuzz cases
def random_pattern(rng: np.random.Generator, m: int, n: int, p: float,
                   dtype=np.float64, shuffle: bool = False,
                   zeros: bool = False, dense_col: bool = False) -> CSC:
    """m x n Bernoulli(p) pattern with N(0, 1) values.

    ``shuffle`` permutes rows inside every column (CSC needs no order),
    ``zeros`` stores some explicit zeros, ``dense_col`` fills one column."""
    mask = rng.random((m, n)) < p
    if dense_col and n > 0:
        mask[:, rng.integers(0, n)] = True
    cols, rows = np.nonzero(mask.T)
    vals = rng.standard_normal(rows.shape[0])
    if zeros and vals.size:
        vals[rng.random(vals.size) < 0.1] = 0.0
    counts = np.bincount(cols, minlength=n).astype(np.int64)
    A = _from_sorted_cols(m, n, counts, rows, vals.astype(dtype))
    if shuffle and n > 0:
        for j in range(n):
            lo, hi = A.colptr[j], A.colptr[j + 1]
            perm = lo + rng.permutation(int(hi - lo))
            A.rowidx[lo:hi] = A.rowidx[perm]
            A.values[lo:hi] = A.values[perm]
    return A


def fuzz_pair(seed: int, dtype=np.float64, max_dim: int = 64):
    """A tiny (A, B) pair with A m x k and B k x n, m, k, n in [0, max_dim].

    Seeds 0..5 are fixed degenerate shapes (0-sized dimensions, 1 x 1, all
    empty, fully dense); the rest draw sizes and densities at random."""
    rng = np.random.default_rng(1000 + seed)
    special = {0: (0, 5, 4, 0.5), 1: (5, 0, 4, 0.5), 2: (5, 4, 0, 0.5),
               3: (1, 1, 1, 1.0), 4: (9, 7, 6, 0.0), 5: (max_dim, 17, 23, 1.0)}
    if seed in special:
        m, k, n, p = special[seed]
    else:
        m, k, n = (int(v) for v in rng.integers(0, max_dim + 1, size=3))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.3, 0.6, 1.0]))
    A = random_pattern(rng, m, k, p, dtype, shuffle=bool(seed % 3 == 1),
                       zeros=bool(seed % 4 == 2), dense_col=bool(seed % 5 == 3))
    B = random_pattern(rng, k, n, p, dtype, shuffle=bool(seed % 3 == 2),
                       zeros=bool(seed % 4 == 3), dense_col=bool(seed % 5 == 4))
    return A, B


def random_vector(n: int, seed: int) -> np.ndarray:
    """N(0, 1) vector of length n."""
    return np.random.default_rng(seed).standard_normal(n)


def workload(k: int):
    """The inputs of workload k (1, 2, 3 or 5) as (A, B); workload 5 returns
    (A, P)."""
    if k == 1:
        A = lap2d(32, seed=0)
        return A, A
    if k == 2:
        return random_z(1 << 20, 1, 8, seed=0), random_z(1 << 20, 1, 8, seed=1)
    if k == 3:
        A = rmat(18, seed=0)
        return A, A
    if k == 5:
        return lap3d(40), prolongation(40, seed=0)
    raise ValueError(f"no single-pair workload {k}")
