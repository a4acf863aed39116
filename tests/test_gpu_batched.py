"""Batched factorizations in one CUDA-graph launch against the oracle (the
graph engine, and the full 512-problem workload on both engines)."""
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


def _batch(count, mmax, seed):
    """Uneven problems shaped like the 512-matrix workload, smaller."""
    shapes = W.c5_shapes(count=count, mmax=mmax, seed=seed)
    As, Ans, ks, Oms, Onp = [], [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        k = min(k, n - 8)
        A, _ = W.c5_matrix(i, m, n)
        Om = W.omega(n, k + 8, i)
        Ans.append(A)
        Onp.append(Om)
        As.append(torch.from_numpy(A).cuda())
        Oms.append(torch.from_numpy(Om).cuda())
        ks.append(k)
    return As, Ans, ks, Oms, Onp


@pytest.mark.parametrize("prec,q,d,pivot2", [("fp64", 1, 2, False), ("fp64", 0, 1, True),
                                             ("bf16x3", 1, 2, False)])
def test_batched_matches_oracle(R, prec, q, d, pivot2):
    As, Ans, ks, Oms, Onp = _batch(20, 700, 77)
    b = R.Batch(As, ks, 8, Oms, q=q, d=d, pivot2=pivot2, prec=prec, branches=6, engine="graph")
    for rep in range(2):  # the graph can be replayed
        b.launch()
        worst, st = b.status()
        assert worst >= 0 and all(s >= 0 for s in st)
        for i in range(len(As)):
            ref = O.rqlp(Ans[i], ks[i], 8, Onp[i], q=q, d=d, pivot2=pivot2)
            lv = b.out[i]["Lvalues"].cpu().numpy()
            l = ks[i] + 8
            keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"].max()
            rel = np.abs(lv - ref["Lvalues"])[keep] / ref["Lvalues"][keep]
            if prec == "fp64":
                assert rel.max() <= 1e-10, (i, rel.max())
                assert np.array_equal(b.out[i]["piv0"].cpu().numpy()[:l], ref["piv0"][:l])
                Q = b.out[i]["Q"].cpu().numpy()
                assert np.abs(Q - ref["Q"]).max() <= 1e-9
            else:
                # index-wise while the pivots agree; after a divergence (a
                # near-tie of column norms flipped by the ~1e-6 perturbation)
                # compare the pivot-independent singular values of L
                pg = b.out[i]["piv0"].cpu().numpy()[:l]
                diff = np.nonzero(pg != ref["piv0"][:l])[0]
                t = int(diff[0]) if diff.size else l
                if t > 0:
                    assert (np.abs(lv - ref["Lvalues"])[:t] / ref["Lvalues"][:t]).max() <= 1e-3
                sg = np.linalg.svd(b.out[i]["L"].cpu().numpy(), compute_uv=False)
                so = np.linalg.svd(ref["L"], compute_uv=False)
                keep = so >= 1e-3 * so[0]
                assert (np.abs(sg - so)[keep] / so[keep]).max() <= 1e-3, i
    assert b.kernel_nodes > 20 * 10
    b.close()


def test_batched_status_per_problem(R):
    As, Ans, ks, Oms, Onp = _batch(6, 400, 78)
    As[3][5, 7] = float("nan")
    b = R.Batch(As, ks, 8, Oms, q=1, d=2, pivot2=False, branches=3, engine="graph")
    b.launch()
    worst, st = b.status()
    assert worst == -2
    assert st[3] == -2 and all(s >= 0 for i, s in enumerate(st) if i != 3)
    b.close()


def test_autotuner_picks_and_caches(R, tmp_path, monkeypatch):
    from paper_1811_09334_gb300 import autotune
    monkeypatch.setenv("RQLP_TUNE_CACHE", str(tmp_path / "tune.json"))
    As, Ans, ks, Oms, Onp = _batch(12, 500, 79)
    t1 = autotune.tune(As, ks, 8, Oms, q=1, d=2, pivot2=False, prec="bf16x3", sample=12)
    assert t1["branches"] in autotune.BRANCHES
    assert (tmp_path / "tune.json").exists()
    t2 = autotune.tune(As, ks, 8, Oms, q=1, d=2, pivot2=False, prec="bf16x3", sample=12)
    assert t1 == t2


def _check_against_oracle(prec, out, ref, l, where):
    lv = out["Lvalues"].cpu().numpy()
    keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"].max()
    if prec == "fp64":
        rel = np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])
        assert rel.max() <= 1e-10, (where, rel.max())
        assert np.array_equal(out["piv0"].cpu().numpy()[:l], ref["piv0"][:l]), where
        Q = out["Q"].cpu().numpy()
        assert np.abs(Q - ref["Q"]).max() <= 1e-9, where
        return
    # index-wise while the pivots agree, then the pivot-free singular values of L
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


@pytest.mark.slow
@pytest.mark.parametrize("prec,engine", [("bf16x3", "persistent"), ("fp64", "persistent"),
                                         ("bf16x3", "graph")])
def test_full_512_problem_batch_sampled_against_the_oracle(R, prec, engine, tmp_path,
                                                            monkeypatch):
    """The whole 512-problem workload (m ~ U[256, 4096], n ~ U[128, m],
    k ~ U[8, 64], p = 8, ERQLP q = 1, d = 2) on each engine the benchmark
    times (autotuned shapes for the graph, one graph launch), with a seeded
    sample of 20 problems and the 4 largest compared with the FP64 oracle."""
    from paper_1811_09334_gb300 import autotune
    monkeypatch.setenv("RQLP_TUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = W.c5_shapes()
    As, ks, Oms = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, _ = W.c5_matrix(i, m, n, device="cuda", fast=True)
        As.append(A)
        ks.append(k)
        Oms.append(torch.from_numpy(W.omega(n, k + 8, i)).cuda())
    torch.cuda.synchronize()
    tune = autotune.tune(As, ks, 8, Oms, q=1, d=2, pivot2=False, prec=prec, sample=128)
    tune["engine"] = engine
    b = R.Batch(As, ks, 8, Oms, q=1, d=2, pivot2=False, prec=prec, **tune)
    assert b.engine == engine
    b.launch()
    worst, st = b.status()
    assert worst >= 0 and all(s >= 0 for s in st)
    cost = [m * n * (k + 8) for (m, n, k) in shapes]
    largest = sorted(range(len(shapes)), key=lambda i: -cost[i])[:4]
    rng = np.random.default_rng(512)
    sample = sorted(set(largest) | set(int(i) for i in rng.choice(len(shapes), 20, replace=False)))
    for i in sample:
        m, n, k = shapes[i]
        ref = O.rqlp(As[i].cpu().numpy(), k, 8, Oms[i].cpu().numpy(), q=1, d=2, pivot2=False)
        _check_against_oracle(prec, b.out[i], ref, k + 8, (i, m, n, k))
    b.close()
