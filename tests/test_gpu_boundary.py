"""The boundary options of rqlp() on the GPU (through the C ABI): fixed
pivots, the rank-k truncation, the R-values, and the adjoint at the forward
call's pivots, against the FP64 oracle.

Tolerances are those of the FP64 parity tests (L and L-values 1e-10
relative, Q and P 1e-9); a factorization at the pivots it chose itself, the
truncation and a backward sweep given the pivots it would have chosen are
the same computation as the free call, so they are compared bit for bit.
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


def _relmax(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


KEYS = ("Q", "L", "P", "Lvalues")


@pytest.mark.parametrize("pivot2,d", [(True, 1), (False, 2), (False, 3)])
def test_fixed_pivots_equal_to_the_chosen_ones_reproduce_the_call(R, pivot2, d):
    pr = W.c1(m=1500, n=900, k=25, p=7)
    Om = _t(W.omega(pr.n, pr.l, 3))
    A = _t(pr.A)
    free = R.rqlp(A, pr.k, pr.p, Om, q=1, d=d, pivot2=pivot2)
    p0 = free["piv0"][:pr.l].clone()
    p1 = free["piv1"].clone() if pivot2 else None
    fix = R.rqlp(A, pr.k, pr.p, Om, q=1, d=d, pivot2=pivot2, piv0=p0, piv1=p1)
    for key in KEYS:
        assert torch.equal(fix[key], free[key]), key
    assert torch.equal(fix["Rvalues"], free["Rvalues"])


@pytest.mark.parametrize("pivot2,d", [(True, 1), (False, 2)])
def test_fixed_pivots_in_another_order_match_the_oracle(R, pivot2, d):
    # the oracle's pivots with two pairs swapped: not what the CPQRs choose
    pr = W.c1(m=1200, n=700, k=20, p=6)
    Om = W.omega(pr.n, pr.l, 4)
    l = pr.l
    free = O.rqlp(pr.A, pr.k, pr.p, Om, q=1, d=d, pivot2=pivot2)
    p0 = free["piv0"][:l].copy()
    p0[[2, 5]] = p0[[5, 2]]
    p0[-1] = free["piv0"][l + 3]  # a column outside the chosen set
    p1 = None
    if pivot2:
        p1 = free["piv1"].copy()
        p1[[0, 1]] = p1[[1, 0]]
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, q=1, d=d, pivot2=pivot2, piv0=p0, piv1=p1)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=1, d=d, pivot2=pivot2,
                 piv0=_t(p0.astype(np.int32)), piv1=None if p1 is None else _t(p1.astype(np.int32)))
    assert _relmax(out["L"], ref["L"]) <= 1e-10
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])) <= 1e-10
    assert _relmax(out["Q"], ref["Q"]) <= 1e-9
    assert _relmax(out["P"], ref["P"]) <= 1e-9
    rv = out["Rvalues"].cpu().numpy()
    assert np.max(np.abs(rv - ref["Rvalues"]) / ref["Rvalues"]) <= 1e-10
    # the given pivots were not overwritten
    assert np.array_equal(out["piv0"].cpu().numpy()[:l], p0)


@pytest.mark.parametrize("bad", ["repeat", "range"])
def test_invalid_given_pivots_are_a_device_status(R, bad):
    pr = W.c1(m=600, n=300, k=10, p=5)
    Om = _t(W.omega(pr.n, pr.l, 0))
    A = _t(pr.A)
    p0 = np.arange(pr.l, dtype=np.int32)
    if bad == "repeat":
        p0[7] = p0[3]
    else:
        p0[7] = pr.n + 11
    with pytest.raises(R.RqlpError) as e:
        R.rqlp(A, pr.k, pr.p, Om, d=2, pivot2=False, piv0=_t(p0))
    assert e.value.code == -1
    # the context and the next call are unharmed
    assert R.rqlp(A, pr.k, pr.p, Om, d=2, pivot2=False)["status"] == 0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("block_b", [0, 6])
def test_truncation_is_the_leading_k_columns(R, prec, block_b):
    pr = W.c1(m=1000, n=600, k=18, p=6)
    Om = _t(W.omega(pr.n, pr.l, 5))
    A = _t(pr.A)
    kw = dict(q=0 if block_b else 1, d=2, pivot2=bool(block_b), prec=prec, block_b=block_b)
    full = R.rqlp(A, pr.k, pr.p, Om, **kw)
    tr = R.rqlp(A, pr.k, pr.p, Om, truncate_k=True, **kw)
    k = pr.k
    assert tuple(tr["Q"].shape) == (pr.m, k) and tuple(tr["L"].shape) == (k, k)
    assert torch.equal(tr["Q"], full["Q"][:, :k].contiguous())
    assert torch.equal(tr["L"], full["L"][:k, :k].contiguous())
    assert torch.equal(tr["P"], full["P"][:, :k].contiguous())
    assert torch.equal(tr["Lvalues"], full["Lvalues"][:k])
    assert torch.equal(tr["Rvalues"], full["Rvalues"][:k])
    if prec == "fp64" and not block_b:
        ref = O.truncate(O.rqlp(pr.A, pr.k, pr.p, W.omega(pr.n, pr.l, 5), q=1, d=2,
                                pivot2=False), k)
        assert _relmax(tr["L"], ref["L"]) <= 1e-10
        assert _relmax(tr["Q"], ref["Q"]) <= 1e-9


@pytest.mark.parametrize("pivot2,d", [(True, 1), (False, 2), (False, 4)])
def test_rvalues_match_the_oracle(R, pivot2, d):
    pr = W.w6("pds", 1000)
    Om = W.omega(pr.n, pr.l, 0)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), d=d, pivot2=pivot2)
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, d=d, pivot2=pivot2)
    rv = out["Rvalues"].cpu().numpy()
    assert np.max(np.abs(rv - ref["Rvalues"]) / ref["Rvalues"]) <= 1e-10
    # Section 5: the L-values track sigma_j far more closely than the R-values
    s = pr.sigma[:pr.k]
    el = np.abs(s - out["Lvalues"].cpu().numpy()[:pr.k]) / s
    er = np.abs(s - rv[:pr.k]) / s
    assert el.mean() < 0.2 * er.mean()


def test_brqlp_rvalues_per_block(R):
    pr = W.c1()
    Om = W.omega(pr.n, pr.l, 5)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), pivot2=True, block_b=10)
    ref = O.brqlp(pr.A, pr.k, pr.p, 10, Om, pivot2=True)
    rv = out["Rvalues"].cpu().numpy()
    for j in range(3):
        _, Rj, _ = O.cpqr(ref["B"][10 * j:10 * (j + 1)])
        want = np.diag(Rj)
        got = rv[10 * j:10 * (j + 1)]
        # block B_j = V_j^T A against the oracle's literal deflation (reading A8)
        assert np.max(np.abs(got - want)) <= 1e-10 * np.abs(rv).max()


def test_backward_at_the_forward_pivots(R):
    pr = W.c4(m=1024, n=512, k=32, p=8)
    A64 = pr.A.astype(np.float64)
    Om = W.omega(pr.n, pr.l, 0)
    A, Omd = _t(A64), _t(Om)
    l = pr.l
    rng = np.random.default_rng(9)
    cQ, cL, cP = rng.standard_normal((pr.m, l)), rng.standard_normal((l, l)), rng.standard_normal((pr.n, l))
    fwd = R.rqlp(A, pr.k, pr.p, Omd, q=1, pivot2=True)
    free = R.vjp(A, pr.k, pr.p, Omd, _t(cQ), _t(cL), _t(cP), q=1)
    given = R.vjp(A, pr.k, pr.p, Omd, _t(cQ), _t(cL), _t(cP), q=1, piv0=fwd["piv0"][:l],
                  piv1=fwd["piv1"])
    assert torch.equal(free, given)
    # other pivots: the derivative of the factorization at those pivots
    p0 = fwd["piv0"][:l].cpu().numpy().copy()
    p0[[1, 3]] = p0[[3, 1]]
    p1 = fwd["piv1"].cpu().numpy().copy()
    p1[[0, 2]] = p1[[2, 0]]
    swapped = R.vjp(A, pr.k, pr.p, Omd, _t(cQ), _t(cL), _t(cP), q=1, piv0=_t(p0), piv1=_t(p1))
    ref = O.rqlp_vjp(A64, pr.k, pr.p, Om, cQ, cL, cP, q=1, piv0=p0, piv1=p1)
    sw = swapped.cpu().numpy()
    assert np.linalg.norm(sw - ref) <= 1e-8 * np.linalg.norm(ref)


def test_autograd_of_a_bf16x3_forward_uses_its_pivots(R):
    # the backward recomputes the forward at the pivots the BF16x3 forward
    # returned; against the oracle's FP64 sweep at those pivots the gradient
    # carries the BF16x3 products' error (about 1e-5 relative, amplified by
    # the QR adjoints' conditioning)
    pr = W.c4(m=1024, n=512, k=32, p=8)
    A32 = pr.A
    Om = W.omega(pr.n, pr.l, 0)
    Ag = _t(A32).requires_grad_(True)
    Q, L, P = R.rqlp_autograd(Ag, pr.k, pr.p, _t(Om), q=1, prec="bf16x3")
    f = torch.diagonal(L)[:pr.k].sum()
    g, = torch.autograd.grad(f, Ag)
    fwd = R.rqlp(_t(A32), pr.k, pr.p, _t(Om), q=1, pivot2=True, prec="bf16x3")
    p0 = fwd["piv0"].cpu().numpy()[:pr.l]
    p1 = fwd["piv1"].cpu().numpy()
    dL = np.diag([1.0] * pr.k + [0.0] * pr.p)
    ref = O.rqlp_vjp(A32.astype(np.float64), pr.k, pr.p, Om, None, dL, None, q=1, piv0=p0, piv1=p1)
    gn = g.double().cpu().numpy()
    assert np.linalg.norm(gn - ref) <= 1e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["bf16x3", "fp64tc"])
def test_factorizations_in_flight_on_several_streams_are_the_single_stream_one(R, prec):
    # three problems at once on three streams (each its own workspace, the
    # count passed as in_flight: the pivoted QR of B then runs on half of the
    # SMs, the FP64 Cholesky on 8-CTA clusters): every output equals the
    # single-stream factorization bit for bit
    pr = W.c1(m=3000, n=2500, k=40, p=10)
    A = _t(pr.A)
    Om = _t(W.omega(pr.n, pr.l, 6))
    kw = dict(q=1, d=2, pivot2=False, prec=prec)
    ref = R.rqlp(A, pr.k, pr.p, Om, **kw)
    streams = [torch.cuda.Stream() for _ in range(3)]
    outs = []
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    for rep in range(2):
        for s in streams:
            outs.append(R.rqlp(A, pr.k, pr.p, Om, stream=s, check=False, in_flight=3, **kw))
    torch.cuda.synchronize()
    for o in outs:
        # the same status too (this spectrum makes the shifted pass run: a warning)
        assert R.read_status(o["ws"]) == ref["status"] >= 0
        for key in ("Q", "L", "P", "Lvalues", "piv0", "piv1"):
            assert torch.equal(o[key], ref[key]), key
