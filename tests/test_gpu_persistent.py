"""The persistent batch engine (one kernel whose CTAs take (problem, stage,
tile) work items from an ordered device list) against the FP64 oracle and
against the graph engine, through the C ABI.

Tolerances are those of the batched graph tests: FP64 L-values 1e-10
relative with identical pivots and Q to 1e-9; BF16x3 L-values 1e-3 relative
while the pivots agree, then the pivot-free singular values of L.
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


def _batch(count, mmax, seed, f32_every=0):
    """Uneven problems shaped like the 512-matrix workload, smaller; every
    f32_every-th matrix is given in FP32."""
    shapes = W.c5_shapes(count=count, mmax=mmax, seed=seed)
    As, Ans, ks, Oms, Onp = [], [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        k = min(k, n - 8)
        A, _ = W.c5_matrix(i, m, n)
        if f32_every and i % f32_every == 0:
            A = A.astype(np.float32)
        Om = W.omega(n, k + 8, i)
        Ans.append(A.astype(np.float64))
        Onp.append(Om)
        As.append(torch.from_numpy(A).cuda())
        Oms.append(torch.from_numpy(Om).cuda())
        ks.append(k)
    return As, Ans, ks, Oms, Onp


def _check(prec, out, ref, l, where):
    lv = out["Lvalues"].cpu().numpy()
    if prec == "fp64":
        rel = np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])
        assert rel.max() <= 1e-10, (where, rel.max())
        assert np.array_equal(out["piv0"].cpu().numpy()[:l], ref["piv0"][:l]), where
        assert np.array_equal(out["piv1"].cpu().numpy(), ref["piv1"][:l]), where
        for key, tol in (("Q", 1e-9), ("P", 1e-9)):
            X = out[key].cpu().numpy()
            assert np.abs(X - ref[key]).max() <= tol, (where, key)
        Lg = out["L"].cpu().numpy()
        assert np.abs(Lg - ref["L"]).max() <= 1e-10 * np.abs(ref["L"]).max(), where
        return
    keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"].max()
    pg = out["piv0"].cpu().numpy()[:l]
    diff = np.nonzero(pg != ref["piv0"][:l])[0]
    t = int(diff[0]) if diff.size else l
    kt = keep[:t]
    if kt.any():
        rel = np.abs(lv[:t] - ref["Lvalues"][:t])[kt] / ref["Lvalues"][:t][kt]
        assert rel.max() <= 1e-3, (where, t, rel.max())
    sg = np.linalg.svd(out["L"].cpu().numpy(), compute_uv=False)
    so = np.linalg.svd(ref["L"], compute_uv=False)
    k2 = so >= 1e-3 * so[0]
    assert (np.abs(sg - so)[k2] / so[k2]).max() <= 1e-3, where


@pytest.mark.parametrize("prec,q,d,pivot2", [("fp64", 1, 2, False), ("fp64", 0, 1, True),
                                             ("fp64", 1, 3, False), ("fp64", 2, 4, False),
                                             ("bf16x3", 1, 2, False), ("bf16x3", 0, 1, True),
                                             ("bf16x3", 1, 3, False)])
def test_persistent_matches_oracle(R, prec, q, d, pivot2):
    As, Ans, ks, Oms, Onp = _batch(20, 700, 77, f32_every=5)
    b = R.Batch(As, ks, 8, Oms, q=q, d=d, pivot2=pivot2, prec=prec, engine="persistent")
    assert b.engine == "persistent"
    assert b.kernel_nodes == 1 and b.work_items > 20 * 10
    for rep in range(2):  # the graph (zeroing + the kernel) can be replayed
        b.launch()
        worst, st = b.status()
        assert worst >= 0 and all(s >= 0 for s in st), st
        for i in range(len(As)):
            ref = O.rqlp(Ans[i], ks[i], 8, Onp[i], q=q, d=d, pivot2=pivot2)
            _check(prec, b.out[i], ref, ks[i] + 8, (rep, i))
    b.close()


def test_persistent_equals_graph_engine_fp64(R):
    As, Ans, ks, Oms, Onp = _batch(12, 900, 81)
    kw = dict(q=1, d=2, pivot2=False, prec="fp64")
    bp = R.Batch(As, ks, 8, Oms, engine="persistent", **kw)
    bg = R.Batch(As, ks, 8, Oms, engine="graph", branches=4, **kw)
    bp.launch()
    bg.launch()
    assert bp.status()[0] >= 0 and bg.status()[0] >= 0
    for i in range(len(As)):
        for key in ("piv0", "piv1"):
            assert torch.equal(bp.out[i][key], bg.out[i][key]), (i, key)
        for key in ("L", "Q", "P"):
            a, g = bp.out[i][key], bg.out[i][key]
            assert float((a - g).abs().max()) <= 1e-12 * float(g.abs().max()), (i, key)
    bp.close()
    bg.close()


def test_persistent_status_per_problem(R):
    As, Ans, ks, Oms, Onp = _batch(6, 400, 78)
    As[3][5, 7] = float("nan")
    b = R.Batch(As, ks, 8, Oms, q=1, d=2, pivot2=False, engine="persistent")
    for _ in range(2):
        b.launch()
        worst, st = b.status()
        assert worst == -2
        assert st[3] == -2 and all(s >= 0 for i, s in enumerate(st) if i != 3)
    # the others are still right
    for i in (0, 5):
        ref = O.rqlp(Ans[i], ks[i], 8, Onp[i], q=1, d=2, pivot2=False)
        _check("fp64", b.out[i], ref, ks[i] + 8, i)
    b.close()


def test_persistent_engine_refuses_what_it_does_not_support(R):
    As, Oms = [], []
    for i in range(3):
        A, _ = W.c5_matrix(i, 600, 400)
        As.append(torch.from_numpy(A).cuda())
        Oms.append(torch.from_numpy(W.omega(400, 140, i)).cuda())
    ks = [132] * 3
    # l = 140 > 128: the persistent engine cannot run it, auto falls back to the graph
    with pytest.raises(R.RqlpError):
        R.Batch(As, ks, 8, Oms, q=0, d=1, pivot2=True, engine="persistent")
    b = R.Batch(As, ks, 8, Oms, q=0, d=1, pivot2=True, engine="auto", branches=3)
    assert b.engine == "graph"
    b.launch()
    assert b.status()[0] >= 0
    b.close()
    # a precision the persistent kernel does not implement
    Om = [torch.from_numpy(W.omega(400, 28, 0)).cuda()]
    with pytest.raises(R.RqlpError):
        R.Batch(As[:1], [20], 8, Om, prec="tf32x3", engine="persistent")
