"""Mixed-precision (tcgen05 tensor-core) products and factorizations.

Tolerances, derived from the arithmetic: BF16 keeps 8 significant bits
(unit roundoff u = 2^-8); the BF16x3 split represents A and W to about u^2
and drops only the Al Wl term (about u^2 |A| |W|), and the FP32 accumulation
over K <= 16384 adds about 1e-6; so the normwise relative error of a BF16x3
product is held to 1e-4 and that of a plain BF16 product to 2e-2.  TF32
keeps 11 (u = 2^-11): the TF32x3 pairs represent A and W to about u^2 =
2^-22, and the tensor cores' FP32 accumulation then dominates, about one
2^-24 per MMA of 8 values along K: with one accumulator a product at
K = 8192 (4096 per K split, 512 MMAs) measured 2.9e-5 normwise; the TF32
forms rotate four accumulators (128 MMAs each), measured 7.2e-6 (BF16x3:
1.5e-5).  So a TF32x3 product is held to 2e-5 and a plain TF32 product to
4e-3.  For whole factorizations the L-values are compared with the FP64
oracle on the same Omega at 1e-3 relative for sigma_j / sigma_1 >= 1e-3.
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


def _normrel(a, b):
    a = a.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m,n,l", [(256, 192, 16), (1000, 700, 30), (2048, 1536, 110),
                                   (333, 257, 17), (130, 4100, 200), (8192, 8192, 110)])
@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("bf16", 2e-2), ("tf32x3", 2e-5),
                                      ("tf32", 4e-3)])
def test_mixed_products(R, m, n, l, prec, tol):
    rng = np.random.default_rng(m * 3 + n + l)
    A = rng.standard_normal((m, n))
    Om = rng.standard_normal((n, l))
    V = rng.standard_normal((m, l))
    Y = R.sketch(_t(A), _t(Om), prec=prec)
    Z = R.project(_t(A), _t(V), prec=prec)
    assert _normrel(Y, O.sketch(A, Om)) <= tol
    assert _normrel(Z, O.adjoint_product(A, V)) <= tol


def test_mixed_product_fp32_input(R):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((1500, 900)).astype(np.float32)
    Om = rng.standard_normal((900, 40))
    Y = R.sketch(_t(A), _t(Om), prec="bf16x3")
    assert _normrel(Y, O.sketch(A.astype(np.float64), Om)) <= 1e-4


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32x3", "tf32"])
@pytest.mark.parametrize("q,d,pivot2", [(1, 2, False), (0, 1, True), (2, 1, False)])
def test_mixed_factorization_lvalues(R, prec, q, d, pivot2):
    pr = W.c2(m=2048, n=1536, k=60, p=10, q=q, d=d)
    Om = W.omega(pr.n, pr.l, 0)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=q, d=d, pivot2=pivot2, prec=prec)
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, q=q, d=d, pivot2=pivot2)
    lv = out["Lvalues"].cpu().numpy()
    keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"].max()
    if prec in ("bf16x3", "tf32x3"):
        # pivots agree with the FP64 oracle, so L-values compare index by index
        assert np.array_equal(out["piv0"].cpu().numpy()[:pr.l], ref["piv0"][:pr.l])
        rel = np.abs(lv - ref["Lvalues"])[keep] / ref["Lvalues"][keep]
        assert rel.max() <= 1e-3, rel.max()
    else:
        # a 2^-8 (2^-11) perturbation may reorder near-equal pivots; compare
        # what does not depend on them: the singular values of L (= those of B)
        sg = np.linalg.svd(out["L"].cpu().numpy(), compute_uv=False)
        so = np.linalg.svd(ref["L"], compute_uv=False)
        keep = so >= 1e-3 * so[0]
        assert (np.abs(sg - so)[keep] / so[keep]).max() <= (2e-2 if prec == "bf16" else 5e-3)
    Q = out["Q"].cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(pr.l)).max() <= 1e-12


@pytest.mark.parametrize("m,n,l", [(256, 192, 16), (2048, 1536, 110), (333, 257, 17), (8192, 8192, 110)])
def test_fp8_products(R, m, n, l):
    """E4M3 products with power-of-two row / column scales: u = 2^-4 per
    operand, so a single product is held to 8e-2 normwise."""
    rng = np.random.default_rng(m + 7 * n + l)
    A = rng.standard_normal((m, n)) * (1.0 + 10.0 * rng.random((m, 1)))
    Om = rng.standard_normal((n, l))
    V = rng.standard_normal((m, l))
    assert _normrel(R.sketch(_t(A), _t(Om), prec="fp8"), O.sketch(A, Om)) <= 8e-2
    assert _normrel(R.project(_t(A), _t(V), prec="fp8"), O.adjoint_product(A, V)) <= 8e-2


def test_fp8_factorization_singular_values(R):
    pr = W.c2(m=2048, n=1536, k=60, p=10, q=1, d=2)
    Om = W.omega(pr.n, pr.l, 0)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=1, d=2, pivot2=False, prec="fp8")
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, q=1, d=2, pivot2=False)
    sg = np.linalg.svd(out["L"].cpu().numpy(), compute_uv=False)
    so = np.linalg.svd(ref["L"], compute_uv=False)
    keep = so >= 1e-3 * so[0]
    # reported, not a precision claim: the E4M3 sketch moves sigma(L) by a few percent
    assert (np.abs(sg - so)[keep] / so[keep]).max() <= 0.1
    Q = out["Q"].cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(pr.l)).max() <= 1e-12


# ------------------------------------------------------------------ FP64TC
@pytest.mark.parametrize("m,n,l", [(256, 192, 16), (1000, 700, 30), (2048, 1536, 110),
                                   (333, 257, 17), (130, 4100, 128), (8192, 8192, 110),
                                   (3000, 70, 64)])
def test_fp64tc_products_are_fp64_accurate(R, m, n, l):
    """Digit products on the tensor cores: each operand element is held to
    2^-48 of its row's scale (the power of two above the row's largest
    magnitude) and the digit pairs below 2^-48 of the leading pair are
    dropped, the leading four weight groups summed exactly; on Gaussian data,
    whose entries sit 3-5 times below the row maximum on both operands, that
    is about 1e-13 normwise (measured 4e-14 to 1.5e-13 at K = 8192), held to
    3e-13 (FP64 DFMA products: about 1e-16)."""
    rng = np.random.default_rng(m * 5 + n + l)
    A = rng.standard_normal((m, n)) * (1.0 + 10.0 * rng.random((m, 1)))
    Om = rng.standard_normal((n, l))
    V = rng.standard_normal((m, l))
    Y = R.sketch(_t(A), _t(Om), prec="fp64tc")
    Z = R.project(_t(A), _t(V), prec="fp64tc")
    ey, ez = _normrel(Y, O.sketch(A, Om)), _normrel(Z, O.adjoint_product(A, V))
    assert ey <= 3e-13 and ez <= 3e-13, (ey, ez)


def test_fp64tc_product_of_fp32_data_and_zero_rows(R):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((700, 500)).astype(np.float32)
    A[17, :] = 0.0
    A[:, 33] = 0.0
    Om = rng.standard_normal((500, 40))
    Y = R.sketch(_t(A), _t(Om), prec="fp64tc")
    ref = O.sketch(A.astype(np.float64), Om)
    assert _normrel(Y, ref) <= 3e-13
    assert np.all(Y.cpu().numpy()[17] == 0.0)


@pytest.mark.parametrize("variant", [(True, 1, 0), (False, 2, 1), (False, 3, 2)])
def test_fp64tc_factorization_holds_the_fp64_parity(R, variant):
    """The FP64TC form against the FP64 oracle at the FP64 form's tolerances:
    L and L-values 1e-10 relative, identical pivots, Q and P 1e-9."""
    pivot2, d, q = variant
    pr = W.c1()
    Om = W.omega(pr.n, pr.l, 0)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=q, d=d, pivot2=pivot2, prec="fp64tc")
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, q=q, d=d, pivot2=pivot2)
    L = out["L"].cpu().numpy()
    assert np.abs(L - ref["L"]).max() <= 1e-10 * np.abs(ref["L"]).max()
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / ref["Lvalues"]) <= 1e-10
    assert np.array_equal(out["piv0"].cpu().numpy()[:pr.l], ref["piv0"][:pr.l])
    assert np.array_equal(out["piv1"].cpu().numpy(), ref["piv1"])
    assert np.abs(out["Q"].cpu().numpy() - ref["Q"]).max() <= 1e-9
    assert np.abs(out["P"].cpu().numpy() - ref["P"]).max() <= 1e-9


def test_fp64tc_nonfinite_and_wide_sketch(R):
    A = np.random.default_rng(2).standard_normal((300, 200))
    A[5, 6] = np.inf
    with pytest.raises(R.RqlpError) as e:
        R.rqlp(_t(A), 10, 5, _t(W.omega(200, 15, 0)), prec="fp64tc")
    assert e.value.code == -2
    A[5, 6] = 0.0
    with pytest.raises(R.RqlpError) as e:  # l > 128 is not offered
        R.rqlp(_t(A), 130, 5, _t(W.omega(200, 135, 0)), prec="fp64tc")
    assert e.value.code == -7
