"""Autotuner for batched factorizations.

Picks how a batch runs by timing candidates on the GPU on a sample of the
batch: the launch shapes of the graph engine (parallel branches, the CTA
target of the FP64 products, the K splits of the tensor-core products), one
knob at a time, then the persistent engine where it supports the batch; the
faster engine wins.  The choice is cached in a JSON file keyed by the
batch's shape bucket (number of problems, largest m, n and l, precision, q,
d).  The cache file is $RQLP_TUNE_CACHE, else ~/.cache/rqlp_gb300_tune.json.
"""
from __future__ import annotations

import json
import os

from . import rqlp as R

BRANCHES = (16, 32, 64, 128)
GEMM_TARGETS = (38, 76, 152)
MMA_SPLITS = (1, 2, 4)


def _cache_path():
    return os.environ.get("RQLP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rqlp_gb300_tune.json"))


def _bucket(n):
    b = 1
    while b < n:
        b *= 2
    return b


def shape_key(As, ks, p, prec, q, d, pivot2):
    mm = max(a.shape[0] for a in As)
    nn = max(a.shape[1] for a in As)
    ll = max(ks) + p
    return "count%d_m%d_n%d_l%d_%s_q%d_d%d_piv%d" % (_bucket(len(As)), _bucket(mm), _bucket(nn),
                                                     _bucket(ll), prec, q, d, int(pivot2))


def _time_batch(As, ks, p, Oms, q, d, pivot2, prec, tune, reps=3):
    import torch
    b = R.Batch(As, ks, p, Oms, q=q, d=d, pivot2=pivot2, prec=prec, **tune)
    try:
        b.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.launch()
        e1.record()
        torch.cuda.synchronize()
        worst, _ = b.status()
        if worst < 0:
            return float("inf")
        return e0.elapsed_time(e1) / reps
    finally:
        b.close()


def tune(As, ks, p, Oms, q=0, d=1, pivot2=True, prec="fp64", sample=64, use_cache=True,
         log=None) -> dict:
    """Engine and launch shapes for this batch: dict(branches, gemm_target_ctas,
    mma_max_splits, engine)."""
    key = shape_key(As, ks, p, prec, q, d, pivot2)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key]["tuning"])
    idx = list(range(0, len(As), max(1, len(As) // sample)))[:sample]
    sA = [As[i] for i in idx]
    sk = [ks[i] for i in idx]
    sO = [Oms[i] for i in idx]
    best = {"branches": 64, "gemm_target_ctas": 76, "mma_max_splits": 2, "engine": "graph"}
    trials = []
    for knob, values in (("branches", BRANCHES), ("gemm_target_ctas", GEMM_TARGETS),
                         ("mma_max_splits", MMA_SPLITS)):
        if knob == "mma_max_splits" and prec == "fp64":
            continue
        times = {}
        for v in values:
            cand = dict(best)
            cand[knob] = v
            times[v] = _time_batch(sA, sk, p, sO, q, d, pivot2, prec, cand)
            trials.append((dict(cand), times[v]))
            if log:
                log("autotune %s=%s: %.3f ms" % (knob, v, times[v]))
        best[knob] = min(times, key=times.get)
    graph_ms = min(ms for t, ms in trials if all(t[k] == best[k] for k in best))
    try:
        cand = dict(best)
        cand["engine"] = "persistent"
        pms = _time_batch(sA, sk, p, sO, q, d, pivot2, prec, cand)
        trials.append((dict(cand), pms))
        if log:
            log("autotune engine=persistent: %.3f ms (graph %.3f ms)" % (pms, graph_ms))
        if pms < graph_ms:
            best["engine"] = "persistent"
    except R.RqlpError:
        pass  # the persistent engine does not support this batch
    if use_cache:
        cache[key] = {"tuning": best, "sample": len(sA),
                      "trials": [{"tuning": t, "ms": ms} for t, ms in trials]}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except OSError:
            pass
    return best
