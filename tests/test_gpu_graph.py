"""One factorization recorded into a CUDA graph and replayed
(rqlp_graph_create / launch / destroy, through the C ABI).

A replay runs the same kernels on the same data as rqlp(), so its outputs
are compared with the direct call bit for bit; the direct call is itself
compared with the FP64 oracle by the parity tests, and here once more for
new data written into A between replays.
"""
import numpy as np
import pytest

from oracle import rqlp_ref as O
from paper_1811_09334_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("Q", "L", "P", "Lvalues", "piv0", "piv1")


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_09334_gb300 import rqlp
    rqlp.lib()
    return rqlp


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "fp64tc"])
def test_replays_equal_the_direct_call(R, prec):
    pr = W.c1(m=3000, n=2500, k=40, p=10)
    A = _t(pr.A)
    Om = _t(W.omega(pr.n, pr.l, 7))
    kw = dict(q=1, d=2, pivot2=False, prec=prec)
    ref = R.rqlp(A, pr.k, pr.p, Om, **kw)
    g = R.Graph(A, pr.k, pr.p, Om, **kw)
    assert g.kernels > 20
    for rep in range(3):
        for key in KEYS:
            g.out[key].fill_(-1)
        n0 = R.launch_count()
        g.launch()
        torch.cuda.synchronize()
        assert R.launch_count() - n0 == g.kernels
        assert g.status() == ref["status"] >= 0
        for key in KEYS:
            assert torch.equal(g.out[key], ref[key]), (rep, key)
    g.close()


def test_new_data_written_in_place_is_factored(R):
    pr = W.c1(m=2000, n=1600, k=30, p=10)
    pr2 = W.c1(m=2000, n=1600, k=30, p=10)
    A = _t(pr.A)
    A2 = pr2.A[::-1].copy() * 0.5  # another matrix of the same shape
    Om = _t(W.omega(pr.n, pr.l, 8))
    kw = dict(q=1, d=2, pivot2=True)
    g = R.Graph(A, pr.k, pr.p, Om, **kw)
    A.copy_(_t(A2))
    g.launch()
    torch.cuda.synchronize()
    direct = R.rqlp(_t(A2), pr.k, pr.p, Om, **kw)
    for key in KEYS:
        assert torch.equal(g.out[key], direct[key]), key
    # and against the oracle (FP64 parity tolerances)
    ref = O.rqlp(A2, pr.k, pr.p, W.omega(pr.n, pr.l, 8), q=1, d=2, pivot2=True)
    assert np.array_equal(g.out["piv0"].cpu().numpy()[:pr.l], ref["piv0"][:pr.l])
    lv = g.out["Lvalues"].cpu().numpy()
    assert np.abs(lv - ref["Lvalues"]).max() <= 1e-10 * np.abs(ref["Lvalues"]).max()
    assert np.abs(g.out["Q"].cpu().numpy() - ref["Q"]).max() <= 1e-9
    g.close()


def test_graphs_in_flight_on_several_streams(R):
    # three graphs (own inputs, workspaces and outputs, in_flight = 3)
    # replayed on three streams: each equals the single-stream direct call
    pr = W.c1(m=3000, n=2500, k=40, p=10)
    Om = _t(W.omega(pr.n, pr.l, 6))
    kw = dict(q=1, d=2, pivot2=False, prec="bf16x3")
    A = _t(pr.A)
    ref = R.rqlp(A, pr.k, pr.p, Om, **kw)
    streams = [torch.cuda.Stream() for _ in range(3)]
    graphs = [R.Graph(A.clone(), pr.k, pr.p, Om, in_flight=3, stream=s, **kw) for s in streams]
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    for rep in range(2):
        for g, s in zip(graphs, streams):
            g.launch(stream=s)
    torch.cuda.synchronize()
    for g in graphs:
        assert g.status() == ref["status"] >= 0
        for key in KEYS:
            assert torch.equal(g.out[key], ref[key]), key
        g.close()


def test_create_refuses_invalid_arguments(R):
    pr = W.c1(m=500, n=400, k=10, p=5)
    A = _t(pr.A)
    Om = _t(W.omega(pr.n, pr.l, 1))
    # blocks of 4 columns do not divide l = 15: rqlp() refuses before recording
    with pytest.raises(R.RqlpError):
        R.Graph(A, pr.k, pr.p, Om, block_b=4)
