"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
example of Fig. 1, dense brute force, the boolean product, identities, the
closed form of the squared 5-point Laplacian, (A B) x = A (B x), the work
identity of Op_j (Section 3.1), and for the backward dense brute force,
adjoint identities and finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2303_02471_gb300 import synth

from helpers import (from_dense, identity, read_golden, scipy_csc, to_dense,
                     to_pattern)

TAU64 = 1e-12


def test_fig1_worked_example():
    g = read_golden("fig1.txt")
    A, B = from_dense(g["A"]), from_dense(g["B"])
    C, _ = oracle.spgemm(A, B)
    assert np.array_equal(to_dense(C), g["C"])
    assert C.colptr[-1] == int(g["NNZ_C"][0, 0])
    assert np.array_equal(oracle.op_counts(A, B), g["OP"][0].astype(np.int64))
    # Column 1 is the sum of the two scaled A columns the figure draws.
    assert np.array_equal(g["COL1_TERMS"].sum(axis=0), g["C"][:, 1])
    for j in range(C.ncols):
        rows = C.rowidx[C.colptr[j]:C.colptr[j + 1]]
        assert np.all(np.diff(rows) > 0)


@pytest.mark.parametrize("seed", range(200))
def test_bruteforce_dense(seed):
    A, B = synth.fuzz_pair(seed)
    C, cabs = oracle.spgemm(A, B)
    Ad, Bd = to_dense(A), to_dense(B)
    ref = Ad @ Bd
    absref = np.abs(Ad) @ np.abs(Bd)
    pat = (to_pattern(A) @ to_pattern(B)) > 0
    assert C.colptr[0] == 0 and C.colptr[-1] == C.rowidx.shape[0]
    assert np.array_equal(to_pattern(C) > 0, pat)
    assert np.array_equal(np.diff(C.colptr), pat.sum(axis=0))
    for j in range(C.ncols):
        rows = C.rowidx[C.colptr[j]:C.colptr[j + 1]]
        assert np.all(np.diff(rows) > 0)
    r, c = np.nonzero(pat.T)[1], np.nonzero(pat.T)[0]
    got = to_dense(C)[r, c]
    err = np.abs(got - ref[r, c])
    assert np.all(err <= TAU64 * absref[r, c] + 0.0)
    # The error scale is the sum of |A_ik B_kj| over the formed products.
    cols = np.repeat(np.arange(C.ncols), np.diff(C.colptr))
    assert np.allclose(cabs, absref[C.rowidx, cols], rtol=1e-13, atol=0)


def test_identity_products_bit_exact():
    A = synth.random_z(300, 1, 9, seed=5)
    I = identity(300)
    C1, _ = oracle.spgemm(A, I)
    C2, _ = oracle.spgemm(I, A)
    for C in (C1, C2):
        assert np.array_equal(C.colptr, A.colptr)
        assert np.array_equal(C.rowidx, A.rowidx)
        assert np.array_equal(C.values, A.values)


def _squared_laplacian_closed_form(g):
    """L = 4I - Adj on a g x g Dirichlet grid: L^2 = 16 I - 8 Adj + Adj^2.

    Entry (p, q): 16 + deg(p) on the diagonal, -8 at the four axis
    neighbours, +2 at the four diagonal neighbours (two 2-step paths), +1 at
    axis distance two (one path)."""
    D = {}
    for y in range(g):
        for x in range(g):
            p = y * g + x
            deg = sum(1 for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1))
                      if 0 <= x + dx < g and 0 <= y + dy < g)
            D[(p, p)] = 16.0 + deg
            for dx, dy, v in ((1, 0, -8.0), (-1, 0, -8.0), (0, 1, -8.0), (0, -1, -8.0),
                              (1, 1, 2.0), (1, -1, 2.0), (-1, 1, 2.0), (-1, -1, 2.0),
                              (2, 0, 1.0), (-2, 0, 1.0), (0, 2, 1.0), (0, -2, 1.0)):
                if 0 <= x + dx < g and 0 <= y + dy < g:
                    D[(p, (y + dy) * g + x + dx)] = v
    return D


@pytest.mark.parametrize("g", [1, 2, 3, 5, 32])
def test_squared_laplacian_13_point(g):
    L = synth.lap2d(g, stencil_values=True)
    C, _ = oracle.spgemm(L, L)
    want = _squared_laplacian_closed_form(g)
    assert C.colptr[-1] == len(want)
    cols = np.repeat(np.arange(C.ncols), np.diff(C.colptr))
    got = {(int(r), int(c)): float(v) for r, c, v in zip(C.rowidx, cols, C.values)}
    assert got == want
    if g == 32:
        assert C.colptr[-1] == 12676


def test_workload1_pattern_is_13_point():
    A, B = synth.workload(1)
    C, _ = oracle.spgemm(A, B)
    want = _squared_laplacian_closed_form(32)
    cols = np.repeat(np.arange(C.ncols), np.diff(C.colptr))
    assert set(zip(C.rowidx.tolist(), cols.tolist())) == set(want)


@pytest.mark.parametrize("kind", ["random", "rmat"])
def test_product_times_vector(kind):
    if kind == "random":
        A = synth.random_z(4000, 1, 8, seed=3)
        B = synth.random_z(4000, 1, 8, seed=4)
    else:
        A = synth.rmat(11, seed=7, col_cap=200)
        B = A
    C, _ = oracle.spgemm(A, B)
    As, Bs, Cs = scipy_csc(A), scipy_csc(B), scipy_csc(C)
    for s in range(8):
        x = synth.random_vector(B.ncols, seed=100 + s)
        lhs = Cs @ x
        rhs = As @ (Bs @ x)
        bound = abs(As) @ (abs(Bs) @ np.abs(x))
        assert np.all(np.abs(lhs - rhs) <= 4 * TAU64 * bound + 1e-300)


def test_work_identity_and_constant_z():
    A = synth.rmat(12, seed=1, col_cap=300)
    B = synth.random_z(A.ncols, 0, 12, seed=2)
    op = oracle.op_counts(A, B)
    zA = np.diff(A.colptr)
    rowdeg_B = np.bincount(B.rowidx, minlength=B.nrows)
    assert op.sum() == int((rowdeg_B * zA).sum())
    for z in (2, 5, 10):
        M = synth.random_z(2560, z, z, seed=z)
        assert np.all(oracle.op_counts(M, M) == z * z)


def test_thread_count_does_not_change_bits():
    A = synth.rmat(12, seed=3, col_cap=400)
    C1, a1 = oracle.spgemm(A, A, nthreads=1)
    C4, a4 = oracle.spgemm(A, A, nthreads=4)
    assert np.array_equal(C1.colptr, C4.colptr)
    assert np.array_equal(C1.rowidx, C4.rowidx)
    assert np.array_equal(C1.values, C4.values)
    assert np.array_equal(a1, a4)


def test_unsorted_input_columns():
    rng = np.random.default_rng(9)
    A = synth.random_pattern(rng, 50, 40, 0.2)
    B = synth.random_pattern(rng, 40, 30, 0.2)
    As = synth.random_pattern(np.random.default_rng(9), 50, 40, 0.2, shuffle=True)
    C, _ = oracle.spgemm(A, B)
    Cs, _ = oracle.spgemm(As, B)
    assert np.array_equal(C.colptr, Cs.colptr)
    assert np.array_equal(C.rowidx, Cs.rowidx)
    assert np.allclose(C.values, Cs.values, rtol=1e-13, atol=1e-15)


def test_float32_inputs_are_widened():
    A, B = synth.fuzz_pair(17)
    C64, _ = oracle.spgemm(A, B)
    A32 = A.astype(np.float32)
    B32 = B.astype(np.float32)
    C32, _ = oracle.spgemm(A32, B32)
    ref = to_dense(A32) @ to_dense(B32)
    assert np.array_equal(C64.rowidx, C32.rowidx)
    cols = np.repeat(np.arange(C32.ncols), np.diff(C32.colptr))
    assert np.allclose(C32.values, ref[C32.rowidx, cols], rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ backward
@pytest.mark.parametrize("seed", range(40))
def test_backward_bruteforce_dense(seed):
    A, B = synth.fuzz_pair(seed)
    C, _ = oracle.spgemm(A, B)
    dC = np.random.default_rng(seed).standard_normal(C.rowidx.shape[0])
    dA, dB = oracle.backward(A, B, C, dC)
    dCd = to_dense(C.__class__(nrows=C.nrows, ncols=C.ncols, colptr=C.colptr,
                               rowidx=C.rowidx, values=dC))
    gA = dCd @ to_dense(B).T
    gB = to_dense(A).T @ dCd
    colsA = np.repeat(np.arange(A.ncols), np.diff(A.colptr))
    colsB = np.repeat(np.arange(B.ncols), np.diff(B.colptr))
    assert np.allclose(dA, gA[A.rowidx, colsA], rtol=1e-12, atol=1e-12)
    assert np.allclose(dB, gB[B.rowidx, colsB], rtol=1e-12, atol=1e-12)


def test_backward_adjoint_identity():
    A = synth.rmat(10, seed=4, col_cap=100)
    B = synth.random_z(A.ncols, 1, 6, seed=5)
    C, _ = oracle.spgemm(A, B)
    rng = np.random.default_rng(6)
    dC = rng.standard_normal(C.rowidx.shape[0])
    dA, dB = oracle.backward(A, B, C, dC)
    EA = A.with_values(rng.standard_normal(A.rowidx.shape[0]))
    EB = B.with_values(rng.standard_normal(B.rowidx.shape[0]))
    # C is bilinear: d/de <dC, (A + e E_A) B> = <dC, E_A B> = <dA, E_A>.
    CA, _ = oracle.spgemm(EA, B)
    CB, _ = oracle.spgemm(A, EB)
    assert np.array_equal(CA.rowidx, C.rowidx) and np.array_equal(CB.rowidx, C.rowidx)
    lhsA, rhsA = np.dot(dC, CA.values), np.dot(dA, EA.values)
    lhsB, rhsB = np.dot(dC, CB.values), np.dot(dB, EB.values)
    scale = np.abs(dC) @ np.abs(CA.values) + np.abs(dC) @ np.abs(CB.values)
    assert abs(lhsA - rhsA) <= 1e-12 * scale
    assert abs(lhsB - rhsB) <= 1e-12 * scale


def test_galerkin_finite_differences():
    A = synth.lap3d(8)
    P = synth.prolongation(8, seed=0)
    M0, _ = oracle.spgemm(A, P)
    Pt0, _ = oracle.transpose(P)
    C0, _ = oracle.spgemm(Pt0, M0)
    T = C0.values * synth.perturbation(C0.rowidx.shape[0], seed=1)
    rng = np.random.default_rng(3)
    Pv = P.values * (1 + 0.05 * rng.uniform(-1, 1, P.values.shape[0]))
    Pw = P.with_values(Pv)
    L, _, _, dP = oracle.galerkin(A, Pw, T_values=T)
    for idx in rng.choice(P.values.shape[0], 24, replace=False):
        h = 1e-6 * max(1.0, abs(Pv[idx]))
        vp, vm = Pv.copy(), Pv.copy()
        vp[idx] += h
        vm[idx] -= h
        Lp = oracle.galerkin(A, P.with_values(vp), T_values=T)[0]
        Lm = oracle.galerkin(A, P.with_values(vm), T_values=T)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dP[idx]) <= 1e-6 * max(1.0, abs(dP[idx])), (idx, fd, dP[idx])


@pytest.mark.parametrize("seed", range(8))
def test_transpose_matches_dense(seed):
    # transpose against the dense transpose; values follow their entries (perm)
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    M = synth.random_pattern(rng, m, n, float(rng.uniform(0.0, 0.5)))
    T, perm = oracle.transpose(M)
    assert (T.nrows, T.ncols) == (n, m)
    D = np.zeros((m, n))
    for j in range(n):
        for q in range(M.colptr[j], M.colptr[j + 1]):
            D[M.rowidx[q], j] = M.values[q]
    E = np.zeros((n, m))
    for j in range(m):
        rows = T.rowidx[T.colptr[j]:T.colptr[j + 1]]
        assert np.all(np.diff(rows) > 0)
        E[rows, j] = T.values[T.colptr[j]:T.colptr[j + 1]]
    assert np.array_equal(E, D.T)
    assert np.array_equal(T.values, M.values[perm])
