"""Pins for the oracle's reverse sweep: central finite differences in FP64.

The forward is evaluated with the pivots of the unperturbed matrix held fixed
(they are piecewise constant), and the directional derivative
(f(A + hE) - f(A - hE)) / 2h is compared with <dA, E>.
"""
import numpy as np
import pytest

from oracle import rqlp_ref as O
from paper_1811_09334_gb300 import workloads as W


def _f(t, cQ, cL, cP):
    return float(np.sum(cQ * t["Q"]) + np.sum(cL * np.tril(t["L"])) + np.sum(cP * t["P"]))


def test_qr_vjp_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((12, 5))
    E = rng.standard_normal(X.shape)
    cQ, cR = rng.standard_normal((12, 5)), np.triu(rng.standard_normal((5, 5)))
    f = lambda Z: float(np.sum(cQ * O.householder_qr(Z)[0]) + np.sum(cR * O.householder_qr(Z)[1]))
    h = 1e-6
    fd = (f(X + h * E) - f(X - h * E)) / (2 * h)
    Q, R = O.householder_qr(X)
    dX = O.qr_vjp(Q, R, cQ, cR)
    assert abs(fd - np.sum(dX * E)) <= 1e-7 * max(1.0, abs(fd))


def test_wide_qr_vjp_matches_finite_differences():
    rng = np.random.default_rng(2)
    C = rng.standard_normal((5, 11))
    E = rng.standard_normal(C.shape)
    cQ, cR = rng.standard_normal((5, 5)), np.triu(rng.standard_normal((5, 11)))
    f = lambda Z: float(np.sum(cQ * O.wide_qr(Z)[0]) + np.sum(cR * O.wide_qr(Z)[1]))
    h = 1e-6
    fd = (f(C + h * E) - f(C - h * E)) / (2 * h)
    Q, R = O.wide_qr(C)
    assert abs(fd - np.sum(O.wide_qr_vjp(Q, R, cQ, cR) * E)) <= 1e-7 * max(1.0, abs(fd))


def test_fixed_pivot_trace_reproduces_rqlp():
    A, _ = W.low_rank_from_spectrum(50, 35, 0.8 ** np.arange(35), 3), None
    Om = W.omega(35, 9, 0)
    free = O.rqlp(A, 6, 3, Om, q=1, pivot2=True)
    t = O.rqlp_trace(A, 6, 3, Om, q=1, piv0=free["piv0"], piv1=free["piv1"])
    for key in ("Q", "L", "P"):
        assert np.allclose(t[key], free[key], atol=1e-12)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rqlp_vjp_matches_finite_differences(q):
    m, n, k, p = 60, 40, 6, 4
    A = W.gaussian(m, n, 5) * (2.0 ** (-np.arange(n) / 8.0))[None, :]
    Om = W.omega(n, k + p, q)
    rng = np.random.default_rng(10 + q)
    l = k + p
    cQ, cL, cP = rng.standard_normal((m, l)), rng.standard_normal((l, l)), rng.standard_normal((n, l))
    E = rng.standard_normal((m, n))
    base = O.rqlp_trace(A, k, p, Om, q)
    piv0, piv1 = base["piv0"], base["piv1"]
    h = 1e-6
    fp = _f(O.rqlp_trace(A + h * E, k, p, Om, q, piv0, piv1), cQ, cL, cP)
    fm = _f(O.rqlp_trace(A - h * E, k, p, Om, q, piv0, piv1), cQ, cL, cP)
    fd = (fp - fm) / (2 * h)
    dA = O.rqlp_vjp(A, k, p, Om, cQ, np.tril(cL), cP, q=q)
    assert abs(fd - np.sum(dA * E)) <= 1e-6 * max(1.0, abs(fd)), (fd, np.sum(dA * E))


def test_sum_of_lvalues_gradient_entrywise():
    # the loss sum_{j<k} L_jj, checked entry by entry on a few entries
    m, n, k, p = 30, 20, 4, 3
    A = W.gaussian(m, n, 8) * (2.0 ** (-np.arange(n) / 6.0))[None, :]
    Om = W.omega(n, k + p, 1)
    dL = np.diag([1.0] * k + [0.0] * p)
    dA = O.rqlp_vjp(A, k, p, Om, None, dL, None, q=1)
    base = O.rqlp_trace(A, k, p, Om, 1)
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(6):
        i, j = rng.integers(m), rng.integers(n)
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fp = np.trace(O.rqlp_trace(Ap, k, p, Om, 1, base["piv0"], base["piv1"])["L"][:k, :k])
        fm = np.trace(O.rqlp_trace(Am, k, p, Om, 1, base["piv0"], base["piv1"])["L"][:k, :k])
        assert abs((fp - fm) / (2 * h) - dA[i, j]) <= 1e-6 * max(1.0, abs(dA[i, j]))


def test_rqlp_vjp_at_given_pivots_matches_finite_differences():
    # pivots that the CPQRs would not choose (two pivots swapped in each QR):
    # the sweep is the derivative of the factorization at those pivots
    m, n, k, p = 50, 30, 5, 3
    A = W.gaussian(m, n, 12) * (2.0 ** (-np.arange(n) / 6.0))[None, :]
    Om = W.omega(n, k + p, 2)
    base = O.rqlp_trace(A, k, p, Om, 1)
    piv0 = base["piv0"].copy()
    piv0[[1, 4]] = piv0[[4, 1]]
    piv1 = base["piv1"].copy()
    piv1[[0, 2]] = piv1[[2, 0]]
    rng = np.random.default_rng(21)
    l = k + p
    cQ, cL, cP = rng.standard_normal((m, l)), rng.standard_normal((l, l)), rng.standard_normal((n, l))
    E = rng.standard_normal((m, n))
    h = 1e-6
    fp = _f(O.rqlp_trace(A + h * E, k, p, Om, 1, piv0, piv1), cQ, cL, cP)
    fm = _f(O.rqlp_trace(A - h * E, k, p, Om, 1, piv0, piv1), cQ, cL, cP)
    fd = (fp - fm) / (2 * h)
    dA = O.rqlp_vjp(A, k, p, Om, cQ, np.tril(cL), cP, q=1, piv0=piv0[:l], piv1=piv1)
    assert abs(fd - np.sum(dA * E)) <= 1e-6 * max(1.0, abs(fd)), (fd, np.sum(dA * E))
    # and it differs from the derivative at the chosen pivots
    dA0 = O.rqlp_vjp(A, k, p, Om, cQ, np.tril(cL), cP, q=1)
    assert np.linalg.norm(dA - dA0) > 1e-3 * np.linalg.norm(dA0)
