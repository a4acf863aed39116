"""Central differences of the oracle forward in worker processes (test
infrastructure for the adjoint tests).

Each worker holds A, Omega and the fixed pivots once (sent at start-up) and
evaluates both losses of the differentiable workload, sum_{j<k} L_jj and
||A - Q_k L_11 P_k^T||_F^2, at A +- h e_i e_c^T with the FP64 oracle at the
fixed pivots.  The pool is started with the spawn method, so that it never
inherits a CUDA context.
"""
import os

_S = {}


def _init(A, Om, k, p, q, piv0, piv1, h):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _S.update(A=A, Om=Om, k=k, p=p, q=q, piv0=piv0, piv1=piv1, h=h)


def _losses(Ap):
    import numpy as np
    from oracle import rqlp_ref as O
    k = _S["k"]
    t = O.rqlp_trace(Ap, k, _S["p"], _S["Om"], _S["q"], _S["piv0"], _S["piv1"])
    E = Ap - t["Q"][:, :k] @ t["L"][:k, :k] @ t["P"][:, :k].T
    return np.trace(t["L"][:k, :k]), float(np.sum(E * E))


def fd_entry(ic):
    """(d loss1 / dA[i, c], d loss2 / dA[i, c]) by central differences."""
    i, c = ic
    A, h = _S["A"], _S["h"]
    Ap = A.copy()
    Ap[i, c] += h
    lp = _losses(Ap)
    Ap[i, c] -= 2 * h
    lm = _losses(Ap)
    return (lp[0] - lm[0]) / (2 * h), (lp[1] - lm[1]) / (2 * h)


def fd_entries(A, Om, k, p, q, piv0, piv1, h, entries, procs=None):
    import multiprocessing as mp
    procs = procs or max(1, min(len(entries), (os.cpu_count() or 2)))
    # single-threaded BLAS in the workers (set before they start)
    old = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    for v in old:
        os.environ[v] = "1"
    try:
        # a worker that dies raises BrokenProcessPool here instead of hanging
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn"), initializer=_init,
                                 initargs=(A, Om, k, p, q, piv0, piv1, h)) as ex:
            return list(ex.map(fd_entry, entries,
                               chunksize=max(1, len(entries) // (4 * procs))))
    finally:
        for v, x in old.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
