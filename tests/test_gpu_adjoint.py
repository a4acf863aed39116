"""GPU adjoint of RQLP (pivots fixed) against the oracle's FP64 reverse sweep
and against central finite differences of the oracle forward.

Tolerances: the FP64 sweep against the oracle's sweep to 1e-8 normwise
(both recompute the forward; the conditioning of the QR adjoints, about
kappa(R)^2 <= 1e6 here, scales eps); through torch.autograd the gradient
comes back in A's dtype, FP32 for the differentiable workload, so 1e-6
there; finite differences with h = 1e-3 in FP64 (the oracle forward with
the pivots fixed) to 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import rqlp_ref as O
from paper_1811_09334_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_09334_gb300 import rqlp
    rqlp.lib()
    return rqlp


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("m,n,k,p,q", [(300, 200, 10, 5, 1), (257, 130, 7, 3, 0), (400, 300, 20, 8, 2)])
def test_vjp_matches_oracle_sweep(R, m, n, k, p, q):
    A = W.gaussian(m, n, 3) * (2.0 ** (-np.arange(n) / 32.0))[None, :]
    Om = W.omega(n, k + p, q)
    rng = np.random.default_rng(m)
    l = k + p
    cQ, cL, cP = rng.standard_normal((m, l)), rng.standard_normal((l, l)), rng.standard_normal((n, l))
    dA = R.vjp(_t(A), k, p, _t(Om), _t(cQ), _t(cL), _t(cP), q=q).cpu().numpy()
    ref = O.rqlp_vjp(A, k, p, Om, cQ, cL, cP, q=q)
    assert np.linalg.norm(dA - ref) <= 1e-8 * np.linalg.norm(ref)


def _c4(small):
    if small:
        pr = W.c4(m=1024, n=512, k=32, p=8)
    else:
        pr = W.c4()
    return pr


@pytest.mark.parametrize("small", [True, False])
def test_c4_losses_autograd_vs_oracle_and_fd(R, small):
    """The differentiable workload: A = N(0,1) diag(2^(-j/256)) in FP32, q = 1,
    losses sum_{j<k} L_jj and ||A - Q_k L11 P_k^T||_F^2."""
    pr = _c4(small)
    k, p = pr.k, pr.p
    A32 = pr.A
    A64 = A32.astype(np.float64)
    Om = W.omega(pr.n, k + p, 0)
    Ag = _t(A32).requires_grad_(True)
    Omg = _t(Om)
    Q, L, P = R.rqlp_autograd(Ag, k, p, Omg, q=1)
    f1 = torch.diagonal(L)[:k].sum()
    g1, = torch.autograd.grad(f1, Ag)
    Ag2 = _t(A32).requires_grad_(True)
    Q, L, P = R.rqlp_autograd(Ag2, k, p, Omg, q=1)
    E = Ag2.double() - Q[:, :k] @ L[:k, :k] @ P[:, :k].T
    f2 = (E * E).sum()
    g2, = torch.autograd.grad(f2, Ag2)
    # oracle reverse sweep (FP64)
    base = O.rqlp_trace(A64, k, p, Om, 1)
    dL1 = np.diag([1.0] * k + [0.0] * p)
    ref1 = O.rqlp_vjp(A64, k, p, Om, None, dL1, None, q=1)
    Ek = A64 - base["Q"][:, :k] @ base["L"][:k, :k] @ base["P"][:, :k].T
    l = k + p
    dQ = np.zeros((pr.m, l)); dLm = np.zeros((l, l)); dP = np.zeros((pr.n, l))
    dQ[:, :k] = -2 * Ek @ base["P"][:, :k] @ base["L"][:k, :k].T
    dLm[:k, :k] = -2 * base["Q"][:, :k].T @ Ek @ base["P"][:, :k]
    dP[:, :k] = -2 * Ek.T @ base["Q"][:, :k] @ base["L"][:k, :k]
    ref2 = 2 * Ek + O.rqlp_vjp(A64, k, p, Om, dQ, dLm, dP, q=1)
    g1n, g2n = g1.double().cpu().numpy(), g2.double().cpu().numpy()
    # autograd returns the gradient in A's dtype (FP32): FP32 rounding level
    assert np.linalg.norm(g1n - ref1) <= 1e-6 * np.linalg.norm(ref1)
    assert np.linalg.norm(g2n - ref2) <= 1e-6 * np.linalg.norm(ref2)
    # central differences (h = 1e-3, FP64 forward with the pivots fixed)
    h = 1e-3
    piv0, piv1 = base["piv0"], base["piv1"]

    def losses(Ap):
        t = O.rqlp_trace(Ap, k, p, Om, 1, piv0, piv1)
        Ep = Ap - t["Q"][:, :k] @ t["L"][:k, :k] @ t["P"][:, :k].T
        return np.trace(t["L"][:k, :k]), float(np.sum(Ep * Ep))

    rng = np.random.default_rng(4)
    D = rng.standard_normal(A64.shape)
    fp, fm = losses(A64 + h * D), losses(A64 - h * D)
    for j, g in enumerate((g1n, g2n)):
        fd = (fp[j] - fm[j]) / (2 * h)
        assert abs(fd - np.sum(g * D)) <= 1e-4 * abs(fd), (j, fd, np.sum(g * D))
    # 200 random entries at every size: the oracle forwards run in a pool of
    # worker processes (spawned, single-threaded BLAS each)
    import fd_pool
    entries = [(int(rng.integers(pr.m)), int(rng.integers(pr.n))) for _ in range(200)]
    fds = fd_pool.fd_entries(A64, Om, k, p, 1, piv0, piv1, h, entries)
    worst = 0.0
    for (i, c), pair in zip(entries, fds):
        for j, g in enumerate((g1n, g2n)):
            fd = pair[j]
            scale = max(abs(fd), 1e-3 * np.abs(g).max())
            worst = max(worst, abs(fd - g[i, c]) / scale)
    assert worst <= 1e-4, worst
