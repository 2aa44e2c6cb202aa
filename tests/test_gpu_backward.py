"""Backward (masked products), transpose and autograd of the CUDA path,
against the CPU oracle and FP64 finite differences."""
import os

import numpy as np
import pytest

import oracle
from paper_2303_02471_gb300 import synth

from gpu_helpers import upload

pytestmark = pytest.mark.gpu

INF = (1 << 63) - 1
NCPU = len(os.sched_getaffinity(0))
TAU = {np.dtype(np.float64): 1e-12, np.dtype(np.float32): 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check_backward(A, B, dtype=np.float64, seed=0, **cfg):
    """GPU dA, dB vs the oracle; tolerance tau * (sum of |terms|), the sums
    taken by the oracle on absolute values."""
    import torch
    from paper_2303_02471_gb300 import ops
    dA_, dB_ = upload(A, dtype), upload(B, dtype)
    C, plan = ops.spgemm(dA_, dB_, ops.Config(**cfg) if cfg else None)
    Ch = C.to_host()
    rng = np.random.default_rng(seed)
    dc = rng.standard_normal(C.nnz).astype(dtype)
    gA, gB = ops.spgemm_backward(plan, dA_, dB_, C, torch.as_tensor(dc, device="cuda"))
    plan.check()
    # the oracle widens float32 inputs and always accumulates in float64
    rA, rB = oracle.backward(A, B, Ch, dc)
    sA, sB = oracle.backward(A.with_values(np.abs(A.values)), B.with_values(np.abs(B.values)), Ch, np.abs(dc))
    tau = TAU[np.dtype(dtype)]
    for got, want, scale, name in ((gA, rA, sA, "dA"), (gB, rB, sB, "dB")):
        g = got.cpu().numpy().astype(np.float64)
        bad = np.abs(g - want) > tau * scale + (0 if dtype == np.float64 else 1e-30)
        assert not bad.any(), f"{name}: {int(bad.sum())} entries off, worst {np.max(np.abs(g - want) - tau * scale)}"
    return C, plan


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", range(30))
def test_backward_fuzz(seed, dtype):
    A, B = synth.fuzz_pair(seed, dtype=dtype)
    _check_backward(A, B, dtype, seed)


@pytest.mark.parametrize("t", [0, 40, None, INF])
def test_backward_rmat_every_bin(t):
    A = synth.rmat(13, seed=2, col_cap=600)
    B = synth.rmat(13, seed=3, col_cap=600)
    _check_backward(A, B, t=t, hash_cta_max=1024)


@pytest.mark.parametrize("promote,pct", [(1, 125), (2, 400)])
def test_backward_table_size_and_group_promotion(promote, pct):
    A = synth.rmat(13, seed=2, col_cap=600)
    B = synth.rmat(13, seed=3, col_cap=600)
    _check_backward(A, B, t=3000, hash_cta_max=1024, table_slots_pct=pct, group_promote=promote)


@pytest.mark.parametrize("t", [0, INF])
def test_backward_tall_products(t):
    # 2^20 rows, nearly all holding entries: the backward's row bitmaps and
    # tables live in the per-CTA global scratch
    from test_gpu_forward import _tall
    A = _tall(1 << 20, 3000, 900, 1100, seed=31)
    B = _tall(3000, 400, 1, 12, seed=32)
    _check_backward(A, B, t=t)


def test_backward_only_one_side():
    import torch
    from paper_2303_02471_gb300 import ops
    A = synth.random_z(3000, 1, 8, seed=1)
    B = synth.random_z(3000, 1, 8, seed=2)
    dA_, dB_ = upload(A), upload(B)
    C, plan = ops.spgemm(dA_, dB_)
    dc = torch.ones(C.nnz, dtype=torch.float64, device="cuda")
    gA, gB = ops.spgemm_backward(plan, dA_, dB_, C, dc, need_dA=False)
    assert gA is None and gB is not None
    Ch = C.to_host()
    rA, rB = oracle.backward(A, B, Ch, np.ones(C.nnz))
    _, sB = oracle.backward(_abs(A), _abs(B), Ch, np.ones(C.nnz))
    _within(gB.cpu().numpy(), rB, sB, 1e-12, "dB")


# ---------------------------------------------------------------- transpose
@pytest.mark.parametrize("case", ["fuzz", "rmat", "long_rows", "empty"])
def test_transpose_matches_oracle(case):
    from paper_2303_02471_gb300 import ops
    rng = np.random.default_rng(4)
    if case == "fuzz":
        M = synth.random_pattern(rng, 300, 200, 0.05, shuffle=True)
    elif case == "rmat":
        M = synth.rmat(12, seed=1, col_cap=300)
    elif case == "long_rows":  # rows of 600 and 20000 entries: shared and global sorts
        M = synth.random_pattern(rng, 3, 20000, 1.0)
        M2 = synth.random_pattern(rng, 5, 600, 1.0)
        T2, p2 = ops.csc_transpose(upload(M2))
        R2, q2 = oracle.transpose(M2)
        assert np.array_equal(T2.rowidx.cpu().numpy(), R2.rowidx)
        assert np.array_equal(p2.cpu().numpy(), q2)
    else:
        M = synth.random_pattern(rng, 7, 0, 0.5)
    T, perm = ops.csc_transpose(upload(M))
    R, q = oracle.transpose(M)
    Th = T.to_host()
    assert np.array_equal(Th.colptr, R.colptr)
    assert np.array_equal(Th.rowidx, R.rowidx)
    assert np.array_equal(Th.values, R.values)
    assert np.array_equal(perm.cpu().numpy(), q)


# ----------------------------------------------------------------- autograd
def _abs(M):
    return M.with_values(np.abs(np.asarray(M.values, dtype=np.float64))) if hasattr(M, "with_values") else \
        synth.CSC(M.nrows, M.ncols, M.colptr, M.rowidx, np.abs(np.asarray(M.values, dtype=np.float64)))


def _within(got, want, scale, tau, what):
    err = np.abs(np.asarray(got, dtype=np.float64) - want)
    bad = err > tau * scale
    assert not bad.any(), f"{what}: {int(bad.sum())} entries off, worst excess {np.max(err - tau * scale)}"


def test_autograd_matches_oracle():
    """Gradients through the autograd Function: per stored entry within
    tau * (sum of |terms|) of the oracle, the sums taken by the oracle on
    absolute values (dC = w exactly, so nothing propagates)."""
    import torch
    from paper_2303_02471_gb300 import autograd as ag
    A = synth.rmat(11, seed=5, col_cap=200)
    B = synth.random_z(A.ncols, 1, 7, seed=6)
    dA_, dB_ = upload(A), upload(B)
    a = dA_.values.clone().requires_grad_(True)
    b = dB_.values.clone().requires_grad_(True)
    C = ag.spgemm(dA_.with_values(a), dB_.with_values(b))
    w = torch.as_tensor(np.random.default_rng(7).standard_normal(C.nnz), device="cuda")
    (C.values * w).sum().backward()
    Ch = C.to_host()
    wh = w.cpu().numpy()
    rA, rB = oracle.backward(A, B, Ch, wh)
    sA, sB = oracle.backward(_abs(A), _abs(B), Ch, np.abs(wh))
    _within(a.grad.cpu().numpy(), rA, sA, 1e-12, "dA")
    _within(b.grad.cpu().numpy(), rB, sB, 1e-12, "dB")


def _galerkin_problem(g):
    A = synth.lap3d(g)
    P = synth.prolongation(g, seed=0)
    M0, _ = oracle.spgemm(A, P)
    Pt0, _ = oracle.transpose(P)
    C0, _ = oracle.spgemm(Pt0, M0)
    T = C0.values * synth.perturbation(C0.rowidx.shape[0], seed=1)
    rng = np.random.default_rng(3)
    Pv = P.values * (1 + 0.05 * rng.uniform(-1, 1, P.values.shape[0]))
    return A, P, T, Pv


def _with(M, values):
    return synth.CSC(M.nrows, M.ncols, np.asarray(M.colptr), np.asarray(M.rowidx), np.asarray(values, np.float64))


@pytest.mark.parametrize("g", [8, 40])
def test_galerkin_gradient_vs_oracle(g):
    """C = P^T (A P), loss ||C - T||^2 and dL/dP against the oracle, entry by entry.

    Every intermediate x of the GPU chain is held to |x - x_ref| <= tau * s_x
    (tau = 1e-12) with s_x the oracle's sum of |terms| carried through the
    chain (each step adds the error its inputs bring to its own rounding):
      M = A P            s_M  = sum |A||P|                       (a plain product)
      C = P^T M          s_C  = 2 sum |P^T| s_M                  (own rounding + M's error)
      G = 2 (C - T)      s_G  = |G| + 2 s_C
      dM = (P^T)^T G     s_dM = 2 sum |P^T| s_G                  (on pattern(M))
      dP^T = G M^T       s_dPt = 3 sum s_G s_M                   (on pattern(P^T))
      dP1 = A^T dM       s_dP1 = 2 sum |A| s_dM                  (on pattern(P))
      dP = dP1 + dP^T scattered back:   s_dP = s_dP1 + s_dPt[perm] + |dP|
    The second product is also compared on its own: the GPU's C against the
    oracle applied to the GPU's M, under the plain rule tau * sum |P^T||M|."""
    import torch
    from paper_2303_02471_gb300 import autograd as ag
    from paper_2303_02471_gb300 import ops
    tau = 1e-12
    A, P, T, Pv = _galerkin_problem(g)
    P1 = P.with_values(Pv)
    dA_ = upload(A)
    dP = upload(P1)
    # the two products and the transpose one by one
    M, _ = ops.spgemm(dA_, dP)
    Mref, sM = oracle.spgemm(A, P1, nthreads=NCPU)
    Mh = M.to_host()
    assert np.array_equal(Mh.colptr, Mref.colptr) and np.array_equal(Mh.rowidx, Mref.rowidx)
    _within(Mh.values, Mref.values, sM, tau, "M = A P")
    Pt, perm = ops.csc_transpose(dP)
    Ptref, pref = oracle.transpose(P1)
    assert np.array_equal(Pt.colptr.cpu().numpy(), Ptref.colptr)
    assert np.array_equal(Pt.rowidx.cpu().numpy(), Ptref.rowidx)
    assert np.array_equal(Pt.values.cpu().numpy(), Ptref.values)
    C2, _ = ops.spgemm(Pt, M)
    C2h = C2.to_host()
    Cg, absCg = oracle.spgemm(Ptref, Mh, nthreads=NCPU)
    assert np.array_equal(C2h.colptr, Cg.colptr) and np.array_equal(C2h.rowidx, Cg.rowidx)
    _within(C2h.values, Cg.values, absCg, tau, "C = P^T M (oracle on the GPU's M)")
    # the differentiable chain
    p = dP.values.clone().requires_grad_(True)
    C = ag.galerkin(dA_, dP.with_values(p))
    Tt = torch.as_tensor(T, device="cuda")
    loss = ((C.values - Tt) ** 2).sum()
    loss.backward()
    L, Cr, _, gP = oracle.galerkin(A, P1, T_values=T)
    Ch = C.to_host()
    assert np.array_equal(Ch.colptr, Cr.colptr) and np.array_equal(Ch.rowidx, Cr.rowidx)
    # error scales of the chain (oracle sums on absolute values)
    absPt = _with(Ptref, np.abs(Ptref.values))
    sC = 2 * oracle.spgemm(absPt, _with(Mref, sM), nthreads=NCPU)[0].values
    _within(Ch.values, Cr.values, sC, tau, "C = P^T (A P)")
    Gref = 2 * (Cr.values - T)
    sG = np.abs(Gref) + 2 * sC
    _, s_dM = oracle.backward(absPt, _with(Mref, sM), Cr, sG, want_dA=False)
    s_dM = 2 * s_dM
    s_dPt, _ = oracle.backward(absPt, _with(Mref, sM), Cr, sG, want_dB=False)
    s_dPt = 3 * s_dPt
    _, s_dP1 = oracle.backward(_abs(A), _with(P1, np.abs(Pv)), Mref, s_dM, want_dA=False)
    s_dP = 2 * s_dP1 + np.abs(gP)
    np.add.at(s_dP, pref, s_dPt)
    # the loss sums |C - T|^2 over pattern(C): its error is at most
    # sum 2 |C - T| tau s_C (first order) plus the rounding of n squares
    # and their sum, n u sum |C - T|^2
    R = np.abs(Cr.values - T)
    n = Cr.values.shape[0]
    assert abs(loss.item() - L) <= tau * np.sum(2 * R * sC) + 2 * n * np.finfo(np.float64).eps * np.sum(R * R)
    _within(p.grad.cpu().numpy(), gP, s_dP, tau, "dL/dP")


def test_galerkin_finite_differences_workload5():
    """FP64 central differences of L = ||P^T A P - T||^2 on 64 seeded entries
    of P at the full 40^3 size (L is a quartic polynomial in each entry)."""
    import torch
    from paper_2303_02471_gb300 import autograd as ag
    A, P, T, Pv = _galerkin_problem(40)
    dA_ = upload(A)
    dP = upload(P.with_values(Pv))
    Tt = torch.as_tensor(T, device="cuda")

    def loss_of(vals):
        C = ag.galerkin(dA_, dP.with_values(vals))
        return ((C.values - Tt) ** 2).sum()

    p = dP.values.clone().requires_grad_(True)
    loss_of(p).backward()
    grad = p.grad.cpu().numpy()
    rng = np.random.default_rng(11)
    idx = rng.choice(Pv.shape[0], 64, replace=False)
    with torch.no_grad():
        for i in idx:
            h = 1e-6 * max(1.0, abs(Pv[i]))
            vp = dP.values.clone()
            vm = dP.values.clone()
            vp[i] += h
            vm[i] -= h
            fd = (loss_of(vp).item() - loss_of(vm).item()) / (2 * h)
            assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), (int(i), fd, grad[i])
