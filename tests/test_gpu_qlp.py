"""The deterministic truncated pivoted QLP on the GPU (rqlp_qlp, the
comparison method of Section 5) against the FP64 oracle at the FP64 parity
tolerances: L and the L-values 1e-10 relative, pivots identical, Q and P
1e-9."""
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


def _relmax(a, b):
    a = a.cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("m,n,t,pivot2", [(600, 400, 30, False), (600, 400, 30, True),
                                          (1500, 900, 125, False), (333, 257, 17, True),
                                          (700, 90, 90, True)])
def test_qlp_matches_oracle(R, m, n, t, pivot2):
    sigma = 0.97 ** np.arange(min(m, n))
    A = W.low_rank_from_spectrum(m, n, sigma, m + n + t)
    out = R.qlp(torch.from_numpy(A).cuda(), t, pivot2=pivot2)
    ref = O.qlp_truncated(A, t, pivot2=pivot2)
    assert np.array_equal(out["piv0"].cpu().numpy()[:t], ref["piv0"][:t])
    assert np.array_equal(out["piv1"].cpu().numpy(), ref["piv1"])
    assert _relmax(out["L"], ref["L"]) <= 1e-10
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])) <= 1e-10
    assert _relmax(out["Q"], ref["Q"]) <= 1e-9
    assert _relmax(out["P"], ref["P"]) <= 1e-9


def test_qlp_paper_matrix_error_matches_oracle(R):
    # the Example 5.1 pds matrix (n = 1000, k = 120, p = 5): the Section 5
    # error of the QLP L-values equals the oracle's
    pr = W.w6("pds", 1000)
    t = pr.k + pr.p
    out = R.qlp(torch.from_numpy(pr.A).cuda(), t, pivot2=True)
    ref = O.qlp_truncated(pr.A, t, pivot2=True)
    e_gpu = O.lvalue_err(pr.sigma, out["Lvalues"].cpu().numpy(), pr.k)
    e_ref = O.lvalue_err(pr.sigma, ref["Lvalues"], pr.k)
    assert abs(e_gpu - e_ref) <= 1e-12
