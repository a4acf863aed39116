"""Pins for the FP64 CPU oracle (no GPU).

Each test ties an oracle function to something other than itself: brute
force on tiny inputs, LAPACK routines reached through numpy / scipy (a
different implementation from the oracle's own Householder loops), closed
forms, and the identities and bounds of Sections 2-4 of the paper.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import rqlp_ref as R
from paper_1811_09334_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _decaying(m, n, seed, decay=0.7):
    """Full-rank m x n matrix with distinct, geometrically decaying singular values."""
    sigma = decay ** np.arange(min(m, n))
    return W.low_rank_from_spectrum(m, n, sigma, seed), sigma


# ------------------------------------------------------------ products
def test_products_match_brute_force():
    A = _rand((5, 4), 1)
    Om = _rand((4, 3), 2)
    V = _rand((5, 3), 3)
    Y = [[sum(A[i][t] * Om[t][j] for t in range(4)) for j in range(3)] for i in range(5)]
    Z = [[sum(A[t][i] * V[t][j] for t in range(5)) for j in range(3)] for i in range(4)]
    B = [[sum(V[t][i] * A[t][j] for t in range(5)) for j in range(4)] for i in range(3)]
    assert np.allclose(R.sketch(A, Om), Y, rtol=0, atol=1e-14)
    assert np.allclose(R.adjoint_product(A, V), Z, rtol=0, atol=1e-14)
    assert np.allclose(R.project(V, A), B, rtol=0, atol=1e-14)


# ------------------------------------------------------------- Householder QR
@pytest.mark.parametrize("shape", [(30, 7), (9, 9), (200, 40), (1, 1), (5, 1)])
def test_householder_qr_matches_lapack(shape):
    X = _rand(shape, 11)
    Q, Rr = R.householder_qr(X)
    Ql, Rl = np.linalg.qr(X)  # LAPACK dgeqrf/dorgqr
    s = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    Ql, Rl = Ql * s, Rl * s[:, None]
    assert np.allclose(Q, Ql, atol=1e-12)
    assert np.allclose(Rr, Rl, atol=1e-12 * np.abs(Rl).max())
    assert np.all(np.diag(Rr) >= 0)
    assert np.allclose(np.tril(Rr, -1), 0)
    assert np.allclose(Q.T @ Q, np.eye(shape[1]), atol=1e-13)
    assert np.allclose(Q @ Rr, X, atol=1e-13 * np.abs(X).max() * shape[0])


def test_householder_qr_closed_form_and_zero_column():
    # X = diag(-3, 2) stacked on zeros: R = diag(3, 2), Q = [[-1, 0], [0, 1], 0...]
    X = np.zeros((4, 2))
    X[0, 0], X[1, 1] = -3.0, 2.0
    Q, Rr = R.householder_qr(X)
    assert np.allclose(Rr, np.diag([3.0, 2.0]))
    assert np.allclose(Q[:, 0], [-1, 0, 0, 0]) and np.allclose(Q[:, 1], [0, 1, 0, 0])
    # a zero column gives a zero diagonal entry and still X = Q R
    X = _rand((10, 4), 3)
    X[:, 2] = 0.0
    Q, Rr = R.householder_qr(X)
    assert Rr[2, 2] == 0.0
    assert np.allclose(Q @ Rr, X, atol=1e-13)


# ------------------------------------------------------------------ CPQR
@pytest.mark.parametrize("shape,seed", [((8, 40), 1), ((40, 8), 2), ((25, 25), 3), ((12, 300), 4)])
def test_cpqr_matches_lapack_pivots(shape, seed):
    X = _rand(shape, seed) * (0.8 ** np.arange(shape[1]))[None, :]
    Q, Rr, piv = R.cpqr(X)
    Ql, Rl, pl = sla.qr(X, pivoting=True, mode="economic")  # LAPACK dgeqp3
    t = min(shape)
    assert list(piv[:t]) == list(pl[:t])
    assert np.allclose(np.abs(np.diag(Rr)), np.abs(np.diag(Rl)), rtol=1e-11)
    d = np.diag(Rr)
    assert np.all(d >= 0) and np.all(np.diff(d) <= 1e-12 * d[0])  # R-values non-increasing
    assert np.allclose(Q @ Rr, X[:, piv], atol=1e-12)
    assert np.allclose(Q.T @ Q, np.eye(t), atol=1e-13)
    assert sorted(piv.tolist()) == list(range(shape[1]))


def test_cpqr_closed_form_and_ties():
    # orthogonal columns of norms 1, 3, 2 -> pivots 1, 2, 0 and R = diag(3, 2, 1)
    X = np.zeros((3, 3))
    X[0, 0], X[1, 1], X[2, 2] = 1.0, -3.0, 2.0
    Q, Rr, piv = R.cpqr(X)
    assert list(piv) == [1, 2, 0]
    assert np.allclose(Rr, np.diag([3.0, 2.0, 1.0]))
    # equal norms: lowest original index first; unchosen columns keep their order
    X = np.array([[0.0, 1.0, 0.0, 1.0, 0.5],
                  [1.0, 0.0, 0.0, 0.0, 0.0]])
    Q, Rr, piv = R.cpqr(X)
    assert list(piv) == [0, 1, 2, 3, 4]


# ------------------------------------------------------------ whole method
def _scipy_pivoted_qlp(A, l):
    """Deterministic truncated pivoted QLP (Section 1, eq. 1.2) through LAPACK."""
    Q, Rr, P = sla.qr(A, pivoting=True, mode="economic")
    Q2, R2, P2 = sla.qr(Rr[:l, :].T, pivoting=True, mode="economic")
    return np.abs(np.diag(R2)), P, P2


def test_full_sketch_equals_deterministic_qlp():
    # l = n: V spans range(A), B^T B = A^T A, so RQLP is Stewart's pivoted QLP of A.
    A, _ = _decaying(60, 40, 5, decay=0.8)
    Om = _rand((40, 40), 6)
    out = R.rqlp(A, 30, 10, Om, pivot2=True)
    lv, p0, p1 = _scipy_pivoted_qlp(A, 40)
    assert list(out["piv0"][:40]) == list(p0[:40])
    assert list(out["piv1"]) == list(p1)
    assert np.allclose(out["Lvalues"], lv, rtol=1e-10)


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("variant", [("rqlp", 1), ("erqlp", 1), ("erqlp", 2), ("erqlp", 3), ("erqlp", 4)])
def test_factorization_identities(q, variant):
    A, sigma = _decaying(70, 50, 7, decay=0.85)
    k, p = 8, 4
    Om = W.omega(50, k + p, trial=q)
    out = R.rqlp(A, k, p, Om, q=q, d=variant[1], pivot2=(variant[0] == "rqlp"))
    Q, L, P, V, B = out["Q"], out["L"], out["P"], out["V"], out["B"]
    l = k + p
    # Q, P column-orthonormal (eq. 1.1); V orthonormal
    assert np.allclose(Q.T @ Q, np.eye(l), atol=1e-13)
    assert np.allclose(P.T @ P, np.eye(l), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(l), atol=1e-13)
    # triangular middle factor with non-negative diagonal
    tri = np.triu(L, 1) if out["lower"] else np.tril(L, -1)
    assert np.abs(tri).max() == 0.0
    assert np.all(out["Lvalues"] >= 0)
    # Q L P^T = V V^T A (eq. 2.3) and the projector identity (eq. 2.1)
    QLP = Q @ L @ P.T
    assert np.allclose(QLP, V @ (V.T @ A), atol=1e-13)
    e2 = np.linalg.norm(A - QLP) ** 2
    assert abs(e2 - (np.linalg.norm(A) ** 2 - np.linalg.norm(B) ** 2)) <= 1e-12 * np.linalg.norm(A) ** 2
    # Lemma 3.1: sigma_j(L) = sigma_j(B) <= sigma_j(A)
    sL = np.linalg.svd(L, compute_uv=False)
    sB = np.linalg.svd(B, compute_uv=False)
    assert np.allclose(sL, sB, rtol=1e-12)
    assert np.all(sB <= sigma[:l] * (1 + 1e-12))
    # rank-deficiency floor: no rank-l factorization beats the SVD tail
    assert np.sqrt(e2) >= np.sqrt(np.sum(sigma[l:] ** 2)) * (1 - 1e-10)


def test_even_d_assembly_reading():
    # The paper's step 9 (L = R(d)^T) fails to reproduce B for even d; the
    # oracle's middle factor R(d) does.  Both share the diagonal.
    A, _ = _decaying(40, 30, 9)
    Om = _rand((30, 10), 10)
    out = R.rqlp(A, 6, 4, Om, d=2, pivot2=False)
    f = R.qlp_of_B(out["B"], d=2, pivot2=False)
    B = out["B"]
    assert np.allclose(f["QB"] @ f["T"] @ f["PB"].T, B, atol=1e-13)
    paper = f["QB"] @ f["T"].T @ f["PB"].T
    assert np.linalg.norm(paper - B) > 1e-3 * np.linalg.norm(B)


def test_exact_recovery_when_l_exceeds_rank():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((60, 5)) @ rng.standard_normal((5, 45))
    for pivot2, d in [(True, 1), (False, 2), (False, 3)]:
        out = R.rqlp(A, 6, 3, _rand((45, 9), 13), d=d, pivot2=pivot2)
        assert np.linalg.norm(A - out["Q"] @ out["L"] @ out["P"].T) <= 1e-12 * np.linalg.norm(A)
        assert np.all(out["Lvalues"][5:] <= 1e-12 * out["Lvalues"][0])


def test_power_iteration_spans_the_power_range():
    # well conditioned, so the plain product (A A^T)^q A Omega is accurate enough
    A, _ = _decaying(30, 20, 14, decay=0.9)
    Om = _rand((20, 6), 15)
    for q in (1, 2):
        V, _ = R.range_finder(A, Om, q)
        Yp = Om
        Yp = A @ Yp
        for _ in range(q):
            Yp = A @ (A.T @ Yp)
        Qp, _ = np.linalg.qr(Yp)
        assert np.allclose(V @ V.T, Qp @ Qp.T, atol=1e-10)


def test_corollary_2_1_expected_error_bound():
    # Corollary 2.1 (eq. 2.4): E||A - Q L P^T||_F <= (1 + k/(p-1))^(1/2) (sum_{j>k} sigma_j^2)^(1/2)
    m, n, k, p = 80, 60, 10, 5
    sigma = 1.0 / np.arange(1, n + 1) ** 1.0
    A = W.low_rank_from_spectrum(m, n, sigma, 21)
    errs = []
    for t in range(200):
        Om = W.omega(n, k + p, trial=1000 + t)
        out = R.rqlp(A, k, p, Om, pivot2=True)
        errs.append(np.linalg.norm(A - out["Q"] @ out["L"] @ out["P"].T))
    tail_k = np.sqrt(np.sum(sigma[k:] ** 2))
    tail_l = np.sqrt(np.sum(sigma[k + p:] ** 2))
    bound = np.sqrt(1 + k / (p - 1)) * tail_k
    mean = float(np.mean(errs))
    assert mean <= bound
    assert min(errs) >= tail_l * (1 - 1e-12)  # Eckart-Young floor
    assert mean >= 0.5 * tail_k  # the sketch is not better than it can be


def test_inner_qr_iterations_improve_lvalues():
    # Lemma 3.3 / Theorem 3.2: more inner QRs give more accurate L-values on
    # average, measured with the Section 5 error err = max_j |sigma_j - L_jj|.
    n, k, p = 200, 20, 5
    for sigma in (W.pds_spectrum(n, 5, 2.0), W.eds_spectrum(n, 5, 0.1)):
        A = W.low_rank_from_spectrum(n, n, sigma, 22)
        mean_err = {}
        for d in (1, 2, 4):
            e = [R.lvalue_err(sigma, R.rqlp(A, k, p, W.omega(n, k + p, trial=t), d=d,
                                            pivot2=False)["Lvalues"], k) for t in range(8)]
            mean_err[d] = np.mean(e)
        assert mean_err[2] < mean_err[1] and mean_err[4] < mean_err[2]


def test_brqlp_matches_unblocked_projector():
    # Section 4: for a fixed Omega the blocked and unblocked range finders give
    # the same projector, and A - Q L P^T = A - V B (eq. 4.5).
    A, _ = _decaying(80, 50, 23, decay=0.8)
    k, p, b = 10, 2, 4
    Om = _rand((50, k + p), 24)
    blk = R.brqlp(A, k, p, b, Om)
    unb = R.rqlp(A, k, p, Om)
    Vb, Vu = blk["V"], unb["V"]
    assert np.allclose(Vb @ Vb.T, Vu @ Vu.T, atol=1e-10)
    QLP = blk["Q"] @ blk["L"] @ blk["P"].T
    assert np.allclose(QLP, Vb @ blk["B"], atol=1e-12)
    assert np.allclose(Vb.T @ Vb, np.eye(k + p), atol=1e-12)
    for j in range((k + p) // b):
        Pj = blk["P"][:, j * b:(j + 1) * b]
        assert np.allclose(Pj.T @ Pj, np.eye(b), atol=1e-12)
        Lj = blk["L"][j * b:(j + 1) * b, j * b:(j + 1) * b]
        assert np.abs(np.triu(Lj, 1)).max() == 0.0
    # the block-diagonal L holds no entries outside its blocks
    mask = np.kron(np.eye((k + p) // b), np.ones((b, b)))
    assert np.abs(blk["L"] * (1 - mask)).max() == 0.0


def test_brqlp_tol_meets_the_tolerance_with_the_fewest_blocks():
    # the stopping rule evaluated directly, without eq. 2.1: the returned
    # basis meets ||A - V V^T A||_F <= tol ||A||_F and one block fewer does not
    A, _ = _decaying(90, 60, 31, decay=0.85)
    b, l_max = 4, 40
    Om = _rand((60, l_max), 32)
    na = np.linalg.norm(A)
    for tol in (0.3, 0.1, 0.03, 1e-2):
        out = R.brqlp_tol(A, b, l_max, tol, Om)
        l = out["l"]
        V = out["V"]
        assert V.shape[1] == l and l % b == 0 and b <= l <= l_max
        assert np.linalg.norm(A - V @ (V.T @ A)) <= tol * na * (1 + 1e-12)
        if l > b:
            Vs = V[:, :l - b]
            assert np.linalg.norm(A - Vs @ (Vs.T @ A)) > tol * na
        # eq. 2.1 itself: ||A - V V^T A||_F^2 = ||A||_F^2 - ||B||_F^2
        assert np.isclose(np.linalg.norm(A - V @ (V.T @ A)) ** 2,
                          na ** 2 - np.linalg.norm(out["B"]) ** 2, rtol=1e-9, atol=1e-12 * na ** 2)


def test_brqlp_tol_zero_tolerance_is_the_full_brqlp():
    A, _ = _decaying(70, 50, 33)
    b, l_max = 5, 20
    Om = _rand((50, l_max), 34)
    full = R.brqlp(A, l_max, 0, b, Om)
    out = R.brqlp_tol(A, b, l_max, 0.0, Om)
    assert out["l"] == l_max
    for key in ("Q", "L", "P", "V", "B"):
        assert np.array_equal(out[key], full[key]), key


def test_brqlp_tol_finds_an_exact_rank():
    # rank 12 = 3 blocks of 4: three blocks capture A to rounding, two cannot
    m, n, r, b = 60, 45, 12, 4
    A = _rand((m, r), 35) @ _rand((r, n), 36)
    Om = _rand((n, 24), 37)
    out = R.brqlp_tol(A, b, 24, 1e-10, Om)
    assert out["l"] == r
    assert np.linalg.norm(A - out["Q"] @ out["L"] @ out["P"].T) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("kind", ["pds", "eds"])
def test_lvalues_track_singular_values_better_than_rvalues(kind):
    # Section 5, Figures 1-2: the L-values |L_jj| follow sigma_j closely while
    # the R-values |R0_jj| of the first pivoted QR (the CPQR of B) fall well
    # below them; measured here 6-9 % against ~74 % mean relative error
    pr = W.w6(kind, 1000)
    k = 120
    s = pr.sigma[:k]
    for pivot2, d in ((True, 1), (False, 2)):
        out = R.rqlp(pr.A, k, 5, W.omega(1000, k + 5, 0), q=0, d=d, pivot2=pivot2)
        er = np.abs(s - np.abs(np.diag(out["R0"]))[:k]) / s
        el = np.abs(s - np.abs(out["Lvalues"])[:k]) / s
        assert el.mean() < 0.2 * er.mean()
        assert np.mean(el <= er) >= 0.9


@pytest.mark.slow
def test_paper_tables_1_2_order_of_magnitude():
    """Section 5, Tables 1-2 (n = 2000): RQLP matches deterministic QLP and inner QRs help.

    Omega is unseeded in the paper, so only the printed orders of magnitude
    and the paper's qualitative observations (1) are checked.
    """
    with open(os.path.join(HERE, "golden", "paper_tables.json")) as f:
        g = json.load(f)
    for row in g["rows"]:
        if row["n"] != 2000:
            continue
        pr = W.w6(row["kind"], row["n"], t=g["t"], s=row["s"])
        Om = W.omega(row["n"], g["k"] + g["p"], trial=0)
        err = {}
        for key, piv, d in [("RQLP", True, 1), ("ERQLP_d2", False, 2), ("ERQLP_d4", False, 4)]:
            out = R.rqlp(pr.A, g["k"], g["p"], Om, d=d, pivot2=piv)
            err[key] = R.lvalue_err(pr.sigma, out["Lvalues"], g["k"])
        lv, _, _ = _scipy_pivoted_qlp(pr.A, g["k"] + g["p"])
        err["QLP"] = R.lvalue_err(pr.sigma, lv, g["k"])
        # observation (1): QLP and RQLP have almost the same error; ERQLP is better
        assert abs(err["RQLP"] - err["QLP"]) <= 0.1 * err["QLP"]
        assert err["ERQLP_d2"] <= err["RQLP"] and err["ERQLP_d4"] < err["RQLP"]
        # printed orders of magnitude (RQLP / QLP columns)
        for key in ("RQLP", "QLP"):
            ratio = err[key] / row[key]
            assert 0.2 <= ratio <= 5.0, (row["kind"], key, err[key], row[key])


# ---------------------------------------------------------- fixed pivots, R-values
def test_complete_perm_closed_form():
    assert list(R.complete_perm([4, 1], 6)) == [4, 1, 0, 2, 3, 5]
    assert list(R.complete_perm([], 3)) == [0, 1, 2]
    for bad in ([1, 1], [6], [-1]):
        with pytest.raises(ValueError):
            R.complete_perm(bad, 6)


@pytest.mark.parametrize("pivot2,d", [(True, 1), (False, 2), (False, 3)])
def test_fixed_pivots_equal_the_chosen_ones(pivot2, d):
    # given the pivots the CPQRs chose, the unpivoted QRs of the permuted
    # matrices are the same factorization (the QR with non-negative diagonal
    # is unique)
    A, _ = _decaying(120, 90, 41, decay=0.85)
    Om = _rand((90, 20), 42)
    ref = R.rqlp(A, 15, 5, Om, q=1, d=d, pivot2=pivot2)
    fix = R.rqlp(A, 15, 5, Om, q=1, d=d, pivot2=pivot2, piv0=ref["piv0"][:20],
                 piv1=ref["piv1"] if pivot2 else None)
    for key in ("Q", "L", "P", "Lvalues"):
        assert np.allclose(fix[key], ref[key], rtol=0, atol=1e-13), key
    assert np.array_equal(fix["piv0"], ref["piv0"])


def test_fixed_pivots_in_another_order_match_lapack_qr():
    # any given column order: R0[:, :l] is LAPACK's QR (sign-fixed) of the
    # chosen columns, and B = Q_B T P_B^T still holds with orthonormal factors
    B = _rand((12, 40), 43) * (0.9 ** np.arange(40))[None, :]
    piv0 = [7, 3, 30, 0, 11, 25, 2, 39, 14, 5, 21, 33]
    piv1 = [3, 0, 11, 1, 2, 10, 4, 9, 5, 8, 6, 7]
    f = R.qlp_of_B(B, pivot2=True, piv0=piv0, piv1=piv1)
    assert list(f["piv0"][:12]) == piv0 and list(f["piv1"]) == piv1
    Ql, Rl = np.linalg.qr(B[:, piv0])
    s = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    assert np.allclose(f["R0"][:, :12], Rl * s[:, None], atol=1e-13)
    assert np.allclose(f["QB"] @ f["T"] @ f["PB"].T, B, atol=1e-13)
    assert np.allclose(f["PB"].T @ f["PB"], np.eye(12), atol=1e-13)
    assert np.allclose(np.triu(f["T"], 1), 0.0)


def test_rvalues_are_lapack_pivoted_qr_diagonal():
    A, _ = _decaying(150, 100, 44, decay=0.8)
    Om = _rand((100, 25), 45)
    out = R.rqlp(A, 20, 5, Om, q=0, d=2, pivot2=False)
    _, Rl, pl = sla.qr(out["B"], pivoting=True, mode="economic")  # LAPACK dgeqp3
    assert np.array_equal(pl[:25], out["piv0"][:25])
    assert np.allclose(out["Rvalues"], np.abs(np.diag(Rl)), rtol=1e-12)
    # truncation to k keeps the leading k columns
    t = R.truncate(out, 20)
    assert t["Q"].shape == (150, 20) and t["L"].shape == (20, 20) and t["P"].shape == (100, 20)
    assert np.array_equal(t["Lvalues"], out["Lvalues"][:20])


# ---------------------------------------------------------- deterministic QLP
@pytest.mark.parametrize("t", [12, 25, 40])
def test_truncated_qlp_matches_lapack_pivoted_qlp(t):
    # the truncated QLP (Section 1, eq. 1.2): pivots and R-rows of the first t
    # steps are LAPACK dgeqp3's, and with the pivoted second QR the L-values
    # are those of LAPACK's two-step pivoted QLP truncated at t
    A, _ = _decaying(60, 40, 21, decay=0.8)
    out = R.qlp_truncated(A, t, pivot2=True)
    lv, p0, p1 = _scipy_pivoted_qlp(A, t)
    assert list(out["piv0"][:t]) == list(p0[:t])
    assert list(out["piv1"]) == list(p1)
    assert np.allclose(out["Lvalues"], lv, rtol=1e-10)
    # Q L P^T = Q0 Q0^T A: the residual identity of eq. 2.1 for the projector
    Q, L, P = out["Q"], out["L"], out["P"]
    E = A - Q @ L @ P.T
    assert abs(np.linalg.norm(E) ** 2 - (np.linalg.norm(A) ** 2 - np.linalg.norm(Q.T @ A) ** 2)) \
        <= 1e-12 * np.linalg.norm(A) ** 2
    assert np.allclose(Q.T @ Q, np.eye(t), atol=1e-13)
    assert np.allclose(P.T @ P, np.eye(t), atol=1e-13)
    assert np.allclose(np.triu(L, 1), 0.0)
    # unpivoted second QR: the same projector, L-values of an unpivoted QR of R0^T
    un = R.qlp_truncated(A, t, pivot2=False)
    assert np.allclose(un["Q"] @ un["L"] @ un["P"].T, Q @ L @ P.T, atol=1e-12)
    if t == 40:  # t = n: the full pivoted QLP reproduces A
        assert np.abs(E).max() <= 1e-13
