"""Plain FP64 CPU oracle of the randomized QLP factorization.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import or run this module.  The CUDA library
shares no code with it: every step here is written out plainly in numpy
(float64), in the order and notation of the paper (Wu & Xiang, "Randomized
QLP algorithm and error analysis", arXiv 1811.09334).  A numpy matrix
product serves as the one library primitive; every QR and column-pivoted QR
below is a textbook Householder loop written here.

Conventions fixed where the paper is silent (each one is a stated reading):

* Every QR / CPQR returns an R factor with non-negative diagonal
  (row i of R and column i of Q are negated together when needed), which
  makes the thin QR of a full-rank matrix unique.
* Column pivoting compares exact trailing column norms, recomputed from the
  current entries at every step (no downdating); on an exact tie the column
  with the lowest original index wins.  After the min(rows, cols) pivot
  steps the columns that were never chosen keep their original order.
* Power steps (Y = (A A^T)^q A Omega) are not in the paper; they follow the
  Halko-style subspace iteration with a QR after every product.
* ERQLP (Algorithm 2.2) is assembled so that B = Q_B T P_B^T holds for
  every d >= 1: with B Pi = Q0 R0 and [R(i-1)]^T = Q(i) R(i),
  Q_B = Q0 Q2 Q4 ..., P_B = Pi Q1 Q3 ..., and the middle factor T is
  R(d)^T (lower triangular) for odd d and R(d) (upper) for even d.  The
  paper's step 9 writes L = R(d)^T for even d, which does not reproduce B;
  both readings have the same diagonal, so the L-values are unaffected.

Pinned by tests/test_oracle.py (brute force, library routines, the
identities of Sections 2-4 and the statistics of Corollary 2.1).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- products
def sketch(A: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """Y = A Omega (Algorithm 2.1, step 2)."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(Omega, dtype=np.float64)


def project(V: np.ndarray, A: np.ndarray) -> np.ndarray:
    """B = V^T A (Algorithm 2.1, step 4)."""
    return np.asarray(V, dtype=np.float64).T @ np.asarray(A, dtype=np.float64)


def adjoint_product(A: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Z = A^T V, the second half of a power step."""
    return np.asarray(A, dtype=np.float64).T @ np.asarray(V, dtype=np.float64)


# ------------------------------------------------------------- Householder
def _reflector(x: np.ndarray):
    """Householder reflector H = I - tau v v^T with v[0] = 1 and H x = beta e1.

    Textbook choice beta = -sign(x0) ||x|| (no cancellation).  Returns
    (v, tau, beta); a zero vector gives tau = 0 and H = I.
    """
    alpha = float(np.sqrt(np.dot(x, x)))
    if alpha == 0.0:
        v = np.zeros_like(x)
        v[0] = 1.0
        return v, 0.0, 0.0
    x0 = float(x[0])
    beta = -alpha if x0 >= 0.0 else alpha
    v = x.copy()
    v[0] = x0 - beta
    tau = (beta - x0) / beta
    v = v / v[0]
    return v, tau, beta


def householder_qr(X: np.ndarray):
    """Thin Householder QR X = Q R (rows >= cols), diag(R) >= 0.

    Returns Q (rows x cols) with orthonormal columns and R (cols x cols)
    upper triangular.
    """
    W = np.array(X, dtype=np.float64, copy=True)
    rows, cols = W.shape
    if rows < cols:
        raise ValueError("householder_qr needs rows >= cols")
    refl = []
    for j in range(cols):
        v, tau, beta = _reflector(W[j:, j])
        if tau != 0.0:
            W[j:, j:] -= tau * np.outer(v, v @ W[j:, j:])
        W[j, j] = beta
        W[j + 1:, j] = 0.0
        refl.append((v, tau))
    R = np.triu(W[:cols, :])
    Q = np.zeros((rows, cols))
    Q[:cols, :cols] = np.eye(cols)
    for j in reversed(range(cols)):
        v, tau = refl[j]
        if tau != 0.0:
            Q[j:, :] -= tau * np.outer(v, v @ Q[j:, :])
    sgn = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * sgn[None, :], R * sgn[:, None]


def orth(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(X): the Q factor of householder_qr."""
    return householder_qr(X)[0]


def cpqr(X: np.ndarray, steps: int = None):
    """Householder QR with column pivoting, X Pi = Q R (Section 1, CPQR).

    At step s the column of largest exact trailing norm ||X(s:, j)|| among
    the columns not yet chosen is moved to position s (ties: lowest original
    index), then a Householder reflector zeroes it below row s.  Runs
    min(rows, cols) steps.

    Returns (Q, R, piv): Q is rows x t with orthonormal columns
    (t = min(rows, cols)), R is t x cols upper trapezoidal with diag >= 0 and
    piv[i] is the original index of the column at position i
    (X[:, piv] = Q R).  With `steps`, only the first t = min(steps, rows,
    cols) pivot steps run (a truncated CPQR: R is the first t rows of R).
    """
    W = np.array(X, dtype=np.float64, copy=True)
    rows, cols = W.shape
    t = min(rows, cols) if steps is None else min(rows, cols, int(steps))
    remaining = list(range(cols))
    order = []
    refl = []
    for s in range(t):
        rem = np.array(remaining)
        norms = np.sqrt(np.sum(W[s:, rem] ** 2, axis=0))
        jstar = int(rem[int(np.argmax(norms))])  # first maximum = lowest index
        order.append(jstar)
        remaining.remove(jstar)
        v, tau, beta = _reflector(W[s:, jstar])
        rest = np.array(remaining, dtype=np.int64)
        if tau != 0.0 and rest.size:
            W[s:, rest] -= tau * np.outer(v, v @ W[s:, rest])
        W[s, jstar] = beta
        W[s + 1:, jstar] = 0.0
        refl.append((v, tau))
    piv = np.array(order + remaining, dtype=np.int64)
    R = W[:t, piv].copy()
    R[np.tril_indices(t, -1, cols)] = 0.0
    Q = np.zeros((rows, t))
    Q[:t, :t] = np.eye(t)
    for s in reversed(range(t)):
        v, tau = refl[s]
        if tau != 0.0:
            Q[s:, :] -= tau * np.outer(v, v @ Q[s:, :])
    sgn = np.where(np.diag(R[:, :t]) < 0.0, -1.0, 1.0)
    return Q * sgn[None, :], R * sgn[:, None], piv


def qlp_truncated(A: np.ndarray, t: int, pivot2: bool = False):
    """Stewart's pivoted QLP truncated at t steps (Section 1, eq. 1.2): the
    first t steps of the CPQR of A, A Pi0 ~= Q0 R0 (R0 = the first t rows of
    R), then the QR of R0^T = Q1 R1, pivoted (cpqr) when pivot2.  Returns Q
    (m x t), L = R1^T, P = Pi0 Q1 (n x t), Lvalues, piv0, piv1 with
    A ~= Q L P^T (exact for t = min(m, n))."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Q0, R0, piv0 = cpqr(A, steps=t)
    X = R0.T
    if pivot2:
        Q1, R1, piv1 = cpqr(X)
        Q = Q0[:, piv1]
    else:
        Q1, R1 = householder_qr(X)
        piv1 = np.arange(R1.shape[0], dtype=np.int64)
        Q = Q0
    P = np.zeros((n, Q1.shape[1]))
    P[piv0, :] = Q1
    L = R1.T
    return dict(Q=Q, L=L, P=P, Lvalues=np.diag(L).copy(), piv0=piv0, piv1=piv1)


# ----------------------------------------------------------- range finder
def range_finder(A: np.ndarray, Omega: np.ndarray, q: int = 0):
    """V with orthonormal columns spanning range((A A^T)^q A Omega).

    q = 0 is the randomized range finder of Section 2 (Algorithm 2.1 steps
    2-3).  For q > 0 every product is followed by a QR:
    V = orth(Y); Z = A^T V; W = orth(Z); Y = A W, repeated q times.
    Returns (V, Y) with Y the last sample matrix.
    """
    A = np.asarray(A, dtype=np.float64)
    Y = sketch(A, Omega)
    for _ in range(q):
        V = orth(Y)
        Z = adjoint_product(A, V)
        Wq = orth(Z)
        Y = sketch(A, Wq)
    return orth(Y), Y


# ---------------------------------------------------------- QLP of small B
def complete_perm(first, n: int) -> np.ndarray:
    """A permutation of range(n) that starts with the given distinct indices,
    the others following in their original order (the convention for the
    columns a column-pivoted QR never chooses)."""
    first = [int(i) for i in first]
    if len(set(first)) != len(first) or any(i < 0 or i >= n for i in first):
        raise ValueError("given pivots must be distinct indices in range")
    chosen = set(first)
    return np.array(first + [j for j in range(n) if j not in chosen], dtype=np.int64)


def qlp_of_B(B: np.ndarray, d: int = 1, pivot2: bool = True, piv0=None, piv1=None):
    """Pivoted QLP of the small l x n matrix B: B = Q_B T P_B^T.

    pivot2 = True: Algorithm 2.1 steps 5-7 (two CPQRs); T = L = R1^T.
    pivot2 = False: Algorithm 2.2 steps 5-9 with d >= 1 unpivoted inner QRs
    [R(i-1)]^T = Q(i) R(i); assembled as described in the module header.
    With piv0 (its first l entries) and, for pivot2, piv1 given, the two
    pivoted QRs become unpivoted QRs of the permuted matrices B Pi0 and
    R0^T Pi1 (the factorization at fixed pivots).

    Returns a dict with QB (l x l), T (l x l), PB (n x l), piv0 (n,),
    piv1 (l,) (identity when pivot2 is False), lower (bool), R0 (l x n).
    """
    B = np.asarray(B, dtype=np.float64)
    l, n = B.shape
    if piv0 is None:
        Q0, R0, piv0 = cpqr(B)
    else:
        piv0 = complete_perm(np.asarray(piv0)[:l], n)
        Q0, R0 = wide_qr(B[:, piv0])
    X = R0.T  # n x l, rows in pivoted order
    if pivot2 and piv1 is not None:
        piv1 = complete_perm(np.asarray(piv1)[:l], l)
        Q1, R1 = householder_qr(X[:, piv1])
        T = R1.T
        QB = Q0[:, piv1]
        M = Q1
        lower = True
    elif pivot2:
        Q1, R1, piv1 = cpqr(X)
        T = R1.T
        QB = Q0[:, piv1]
        M = Q1
        lower = True
    else:
        if d < 1:
            raise ValueError("ERQLP needs d >= 1")
        Qs = [Q0]
        R = R0
        for _ in range(d):
            Qi, Ri = householder_qr(R.T)
            Qs.append(Qi)
            R = Ri
        QB = Qs[0]
        for i in range(2, d + 1, 2):
            QB = QB @ Qs[i]
        M = Qs[1]
        for i in range(3, d + 1, 2):
            M = M @ Qs[i]
        T = R.T if d % 2 == 1 else R
        piv1 = np.arange(l, dtype=np.int64)
        lower = (d % 2 == 1)
    PB = np.zeros((n, l))
    PB[piv0, :] = M
    return dict(QB=QB, T=T, PB=PB, piv0=piv0, piv1=piv1, lower=lower, R0=R0)


# ------------------------------------------------------------ RQLP / ERQLP
def rqlp(A: np.ndarray, k: int, p: int, Omega: np.ndarray, q: int = 0, d: int = 1,
         pivot2: bool = True, piv0=None, piv1=None):
    """Randomized QLP (Algorithm 2.1) / enhanced RQLP (Algorithm 2.2).

    A (m x n), target rank k, oversampling p, l = k + p, Omega (n x l) given
    by the caller, q power steps, d inner QRs (used when pivot2 is False);
    optional given pivots as in qlp_of_B.  Returns a dict with Q (m x l),
    L (l x l; lower unless even-d ERQLP), P (n x l), Lvalues (l,), Rvalues
    (l,), piv0, piv1, V, B, lower.  A ~= Q L P^T.  The R-values diag R0 are
    the diagonal of the CPQR of B that Section 5 compares with the L-values.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    Omega = np.asarray(Omega, dtype=np.float64)
    if Omega.shape != (n, l):
        raise ValueError("Omega must be n x (k + p)")
    if not (1 <= l <= min(m, n)):
        raise ValueError("need 1 <= k + p <= min(m, n)")
    V, Y = range_finder(A, Omega, q)
    B = project(V, A)
    f = qlp_of_B(B, d=d, pivot2=pivot2, piv0=piv0, piv1=piv1)
    Q = V @ f["QB"]
    L = f["T"]
    return dict(Q=Q, L=L, P=f["PB"], Lvalues=np.diag(L).copy(), piv0=f["piv0"],
                piv1=f["piv1"], V=V, B=B, lower=f["lower"], R0=f["R0"], Y=Y,
                Rvalues=np.diag(f["R0"][:, :l]).copy())


def truncate(res: dict, k: int) -> dict:
    """The rank-k truncation of a factorization (the abstract's rank-k L):
    Q[:, :k], L[:k, :k], P[:, :k] and the first k L-values."""
    return dict(Q=res["Q"][:, :k], L=res["L"][:k, :k], P=res["P"][:, :k],
                Lvalues=res["Lvalues"][:k])


# ------------------------------------------------------------------ BRQLP
def _brqlp_blocks(A: np.ndarray, b: int, Omega: np.ndarray, nblocks: int, pivot2: bool, d: int,
                  tol: float = None):
    """The block loop of Algorithm 4.1: per block j, Y_j = A Omega_j;
    V_j = qr(Y_j); V_j = qr(V_j - sum_{i<j} V_i V_i^T V_j); B_j = V_j^T A(j-1);
    A(j) = A(j-1) - V_j B_j; [Q_B(j), L_j, P_B(j)] = qlp(B_j).  With tol, the
    loop stops after the first block at which ||A||_F^2 - ||B||_F^2 <=
    tol^2 ||A||_F^2, B the stacked B_j (the residual ||A - V V^T A||_F^2 of
    eq. 2.1, V = [V_j] orthonormal)."""
    A = np.asarray(A, dtype=np.float64)
    Aj = A.copy()
    a2 = float(np.sum(A * A))
    b2 = 0.0
    Vs, Bs, Qs, Ls, Ps = [], [], [], [], []
    for j in range(nblocks):
        Om = np.asarray(Omega, dtype=np.float64)[:, j * b:(j + 1) * b]
        Yj = sketch(A, Om)
        Vj = orth(Yj)
        if Vs:
            Vprev = np.concatenate(Vs, axis=1)
            Vj = orth(Vj - Vprev @ (Vprev.T @ Vj))
        Bj = project(Vj, Aj)
        Aj = Aj - Vj @ Bj
        f = qlp_of_B(Bj, d=d, pivot2=pivot2)
        Vs.append(Vj)
        Bs.append(Bj)
        Qs.append(Vj @ f["QB"])
        Ls.append(f["T"])
        Ps.append(f["PB"])
        b2 += float(np.sum(Bj * Bj))
        if tol is not None and a2 - b2 <= tol * tol * a2:
            break
    h = len(Vs)
    l = h * b
    L = np.zeros((l, l))
    for j in range(h):
        L[j * b:(j + 1) * b, j * b:(j + 1) * b] = Ls[j]
    return dict(Q=np.concatenate(Qs, axis=1), L=L, P=np.concatenate(Ps, axis=1),
                Lvalues=np.diag(L).copy(), V=np.concatenate(Vs, axis=1),
                B=np.concatenate(Bs, axis=0), Lblocks=Ls, l=l)


def brqlp(A: np.ndarray, k: int, p: int, b: int, Omega: np.ndarray, pivot2: bool = True,
          d: int = 1):
    """Block randomized QLP, Algorithm 4.1, taken literally.

    l = k + p = h b.  Per block j: Y_j = A Omega_j; V_j = qr(Y_j);
    V_j = qr(V_j - sum_{i<j} V_i V_i^T V_j); B_j = V_j^T A(j-1);
    A(j) = A(j-1) - V_j B_j; [Q_B(j), L_j, P_B(j)] = qlp(B_j);
    Q_j = V_j Q_B(j), P_j = P_B(j).  Output Q = [Q_j], L = blkdiag(L_j),
    P = [P_j]; also V = [V_j] and B = [B_j] (stacked).
    """
    l = k + p
    if l % b != 0:
        raise ValueError("block size must divide k + p")
    return _brqlp_blocks(A, b, Omega, l // b, pivot2, d)


def brqlp_tol(A: np.ndarray, b: int, l_max: int, tol: float, Omega: np.ndarray,
              pivot2: bool = True, d: int = 1):
    """Fixed-accuracy BRQLP: the blocks of Algorithm 4.1 are added until the
    relative residual ||A - V V^T A||_F / ||A||_F is at most tol (evaluated
    through eq. 2.1 as ||A||_F^2 - ||B||_F^2), or until l_max = h b columns
    (the blocked scheme's use named at the end of the paper).  Omega is
    n x l_max; returns brqlp's dict for the l = j b columns used, with "l"."""
    if l_max % b != 0:
        raise ValueError("block size must divide l_max")
    if tol < 0:
        raise ValueError("tol must be >= 0")
    return _brqlp_blocks(A, b, Omega, l_max // b, pivot2, d, tol=tol)


def lvalue_err(sigma: np.ndarray, Lvalues: np.ndarray, k: int) -> float:
    """err = max_{j<=k} |sigma_j(A) - |L_jj|| (Section 5 error measure)."""
    return float(np.max(np.abs(np.asarray(sigma)[:k] - np.abs(np.asarray(Lvalues)[:k]))))


# ------------------------------------------------------------------ adjoint
# Reverse-mode derivative of RQLP (Algorithm 2.1) with the column pivots
# held fixed (the pivots are piecewise constant in A).  Not in the paper.
def qr_vjp(Q, R, dQ, dR):
    """Cotangent of X for the thin QR X = Q R (rows >= cols, R invertible).

    dX = (dQ + Q copyltu(M)) R^{-T},  M = R dR^T - dQ^T Q,
    copyltu(M) = tril(M) + tril(M, -1)^T.
    """
    M = R @ dR.T - dQ.T @ Q
    S = np.tril(M) + np.tril(M, -1).T
    T = dQ + Q @ S
    return sla_solve_triangular(R, T.T, lower=False, trans="N").T  # T R^{-T}


def sla_solve_triangular(R, B, lower, trans):
    import scipy.linalg as sla
    return sla.solve_triangular(R, B, lower=lower, trans=trans)


def wide_qr(C):
    """Unpivoted QR C = Q R of an l x n matrix (l <= n), diag(R) >= 0."""
    l = C.shape[0]
    Q, U = householder_qr(C[:, :l])
    return Q, np.concatenate([U, Q.T @ C[:, l:]], axis=1)


def wide_qr_vjp(Q, R, dQ, dR):
    """Cotangent of C for C = Q R, C l x n (l <= n), R = [U | V].

    C2 = Q V gives V = Q^T C2: dC2 = Q dV and dQ picks up C2 dV^T; the
    square part C1 = Q U then follows qr_vjp.
    """
    l = Q.shape[0]
    U, Vr = R[:, :l], R[:, l:]
    dU, dV = dR[:, :l], dR[:, l:]
    C2 = Q @ Vr
    dC1 = qr_vjp(Q, U, dQ + C2 @ dV.T, dU)
    return np.concatenate([dC1, Q @ dV], axis=1)


def rqlp_trace(A, k, p, Omega, q=0, piv0=None, piv1=None):
    """RQLP forward (Algorithm 2.1) keeping every intermediate.

    With piv0 / piv1 given, the two column-pivoted QRs use these pivots
    instead of choosing them (B Pi0 = Q0 R0 and R0^T Pi1 = Q1 R1 as
    unpivoted QRs of the permuted matrices).
    """
    A = np.asarray(A, dtype=np.float64)
    Om = np.asarray(Omega, dtype=np.float64)
    t = {"Ys": [A @ Om], "Vs": [], "RYs": [], "Zs": [], "Ws": [], "RZs": []}
    for _ in range(q):
        V, RY = householder_qr(t["Ys"][-1])
        Z = A.T @ V
        Wq, RZ = householder_qr(Z)
        t["Vs"].append(V); t["RYs"].append(RY); t["Zs"].append(Z); t["Ws"].append(Wq)
        t["RZs"].append(RZ)
        t["Ys"].append(A @ Wq)
    V, RY = householder_qr(t["Ys"][-1])
    t["V"], t["RY"] = V, RY
    B = V.T @ A
    if piv0 is None or piv1 is None:
        Q0, R0, piv0 = cpqr(B)
        Q1, R1, piv1 = cpqr(R0.T)
    else:
        piv0 = np.asarray(piv0)
        piv1 = np.asarray(piv1)
        Q0, R0 = wide_qr(B[:, piv0])
        Q1, R1 = householder_qr(R0.T[:, piv1])
    n, l = A.shape[1], V.shape[1]
    P = np.zeros((n, l))
    P[piv0, :] = Q1
    QB = Q0[:, piv1]
    t.update(B=B, Q0=Q0, R0=R0, Q1=Q1, R1=R1, piv0=piv0, piv1=piv1, QB=QB,
             Q=V @ QB, L=R1.T, P=P)
    return t


def rqlp_vjp(A, k, p, Omega, dQ, dL, dP, q=0, piv0=None, piv1=None):
    """dA = J^T (dQ, dL, dP) for RQLP (Algorithm 2.1) with fixed pivots.

    The sweep runs the forward of rqlp_trace backwards, product by product
    and QR by QR (qr_vjp, wide_qr_vjp), recomputing the forward first (at the
    given pivots, when piv0 and piv1 are given; piv0 may hold only its first
    l entries, completed as in complete_perm).
    """
    A = np.asarray(A, dtype=np.float64)
    Om = np.asarray(Omega, dtype=np.float64)
    if piv0 is not None:
        piv0 = complete_perm(np.asarray(piv0)[:k + p], A.shape[1])
    t = rqlp_trace(A, k, p, Om, q, piv0, piv1)
    l = t["V"].shape[1]
    n = A.shape[1]
    dQ = np.zeros_like(t["Q"]) if dQ is None else dQ
    dL = np.zeros((l, l)) if dL is None else dL
    dP = np.zeros_like(t["P"]) if dP is None else dP
    piv0, piv1 = t["piv0"], t["piv1"]
    # step 7: Q = V Q0[:, piv1], L = R1^T, P[piv0] = Q1
    dV = dQ @ t["QB"].T
    dQ0 = np.zeros((l, l))
    dQ0[:, piv1] = t["V"].T @ dQ
    dQ1 = dP[piv0, :]
    dR1 = np.triu(dL.T)
    # step 6: R0^T[:, piv1] = Q1 R1
    dXp = qr_vjp(t["Q1"], t["R1"], dQ1, dR1)
    dX = np.zeros((n, l))
    dX[:, piv1] = dXp
    dR0 = np.triu(dX.T)
    # step 5: B[:, piv0] = Q0 R0
    dC = wide_qr_vjp(t["Q0"], t["R0"], dQ0, dR0)
    dB = np.zeros((l, n))
    dB[:, piv0] = dC
    # step 4: B = V^T A
    dV = dV + A @ dB.T
    dA = t["V"] @ dB
    # step 3: V = qr(Y_q), R discarded
    dY = qr_vjp(t["V"], t["RY"], dV, np.zeros((l, l)))
    # step 2, backwards: Y_i = A W_i, W_i = qr(Z_i), Z_i = A^T V_i, V_i = qr(Y_{i-1})
    for i in reversed(range(q)):
        dA += dY @ t["Ws"][i].T
        dW = A.T @ dY
        dZ = qr_vjp(t["Ws"][i], t["RZs"][i], dW, np.zeros((l, l)))
        dA += t["Vs"][i] @ dZ.T
        dVi = A @ dZ
        dY = qr_vjp(t["Vs"][i], t["RYs"][i], dVi, np.zeros((l, l)))
    # step 1: Y_0 = A Omega
    dA += dY @ Om.T
    return dA
