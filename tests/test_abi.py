"""The C-ABI library loads and exports what include/rqlp.h declares (no GPU needed)."""
import ctypes

import pytest

from paper_1811_09334_gb300 import rqlp as R


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return R.lib()


def test_every_declared_symbol_is_exported(lib):
    names = R.header_symbols()
    assert "rqlp" in names and "rqlp_workspace_size" in names
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(names) <= set(R._SIGS)


def test_version_and_status_strings(lib):
    assert lib.rqlp_version() >= 100
    for code in R.STATUS:
        assert lib.rqlp_status_string(code)
    assert lib.rqlp_status_string(12345) == b"unknown status"


def test_argument_errors_are_synchronous(lib):
    o = R.opts()
    assert lib.rqlp_workspace_size(0, 10, 2, 2, ctypes.byref(o)) == 0
    assert lib.rqlp_workspace_size(10, 10, 8, 3, ctypes.byref(o)) == 0  # l > n
    assert lib.rqlp_workspace_size(1000, 500, 200, 60, ctypes.byref(o)) == 0  # l > 256
    assert lib.rqlp_workspace_size(100, 50, 5, 5, ctypes.byref(o)) > 0
    bad = R.opts(pivot2=False, d=0)
    assert lib.rqlp_workspace_size(100, 50, 5, 5, ctypes.byref(bad)) == 0
    # null pointers are rejected before any CUDA call
    code = lib.rqlp(None, 0, 100, 50, 50, 5, 5, None, 10, ctypes.byref(o), None, None, None, None,
                    None, None, None, 0, None)
    assert code == -1
    code = lib.rqlp_orth(None, 10, 4, 4, None, 4, None, None, 0, None)
    assert code == -1


def test_precision_names_match_the_header(lib):
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "rqlp.h")) as f:
        hdr = f.read()
    enum = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"RQLP_PREC_([A-Z0-9]+)\s*=\s*(\d+)", hdr)}
    assert enum == R.PREC
    # every precision is accepted, the next value is not
    sizes = {}
    for name, code in R.PREC.items():
        o = R.opts(q=1, d=2, pivot2=False, prec=name)
        sizes[name] = lib.rqlp_workspace_size(4096, 2048, 100, 10, ctypes.byref(o))
        assert sizes[name] > 0, name
    o = R.opts(q=1, d=2, pivot2=False)
    o.prec = max(R.PREC.values()) + 1
    assert lib.rqlp_workspace_size(4096, 2048, 100, 10, ctypes.byref(o)) == 0
    # the TF32 pairs take twice the bytes of the BF16 pairs, one TF32 copy
    # those of the BF16 pair; FP64 keeps no copies of A
    assert sizes["tf32x3"] > sizes["bf16x3"] > sizes["bf16"] > sizes["fp64"]
    assert sizes["tf32"] > sizes["bf16"]


def test_new_options_are_checked(lib):
    # fixed pivots and truncation are 0/1 switches; fixed pivots need the
    # pivot arrays and are not offered for the blocked form
    o = R.opts(fixed_pivots=True, truncate_k=True)
    assert lib.rqlp_workspace_size(100, 50, 5, 5, ctypes.byref(o)) > \
        lib.rqlp_workspace_size(100, 50, 5, 5, ctypes.byref(R.opts()))
    o.truncate_k = 2
    assert lib.rqlp_workspace_size(100, 50, 5, 5, ctypes.byref(o)) == 0
    o = R.opts(fixed_pivots=True)
    dummy = ctypes.c_void_p(256)  # never dereferenced: the call fails on its arguments
    code = lib.rqlp(dummy, 0, 100, 50, 50, 5, 5, dummy, 10, ctypes.byref(o), dummy, dummy, dummy,
                    None, None, None, dummy, 1 << 20, None)
    assert code == -1
    o = R.opts(fixed_pivots=True, block_b=5)
    code = lib.rqlp(dummy, 0, 100, 50, 50, 5, 5, dummy, 10, ctypes.byref(o), dummy, dummy, dummy,
                    None, dummy, dummy, dummy, 1 << 20, None)
    assert code == -7
    assert lib.rqlp_backward_workspace_size(100, 50, 5, 5, ctypes.byref(R.opts(truncate_k=True))) == 0
    assert lib.rqlp_version() >= 200


def _problems(shapes):
    # fake (never dereferenced) device pointers: the size queries only read shapes
    probs = (R.Problem * len(shapes))()
    for i, (m, n, k) in enumerate(shapes):
        f = ctypes.c_void_p(4096 * (i + 1))
        probs[i] = R.Problem(f, 0, k, m, n, n, 8, 0, f, k + 8, f, f, f, f, f, f)
    return probs


def test_batch_engine_selection_by_workspace_size(lib):
    shapes = [(700, 500, 40), (300, 200, 20), (1000, 900, 64)]
    probs = _problems(shapes)
    o = R.opts(q=1, d=2, pivot2=False, prec="bf16x3")
    size = {e: lib.rqlp_batched_workspace_size(probs, 3, ctypes.byref(o),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, c)))
            for e, c in R.ENGINES.items()}
    assert size["persistent"] > 0 and size["graph"] > 0
    assert size["auto"] == size["persistent"]
    # the persistent engine keeps every problem's BF16 copies of A at once
    assert size["persistent"] > 8 * sum(m * n for m, n, _ in shapes)
    # l = 136 > 128, a precision it lacks, a truncation: not for the persistent kernel
    big = _problems([(700, 500, 128)])
    for oo, pr in ((o, big), (R.opts(prec="tf32x3"), probs), (R.opts(truncate_k=True), probs)):
        n = 1 if pr is big else 3
        assert lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, 2))) == 0
        assert lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, 0))) == \
            lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                            ctypes.byref(R.BatchTuning(4, 0, 0, 1)))
    assert lib.rqlp_batched_workspace_size(probs, 3, ctypes.byref(o),
                                           ctypes.byref(R.BatchTuning(4, 0, 0, 7))) == 0


def _problems(shapes):
    # fake (never dereferenced) device pointers: the size queries only read shapes
    probs = (R.Problem * len(shapes))()
    for i, (m, n, k) in enumerate(shapes):
        f = ctypes.c_void_p(4096 * (i + 1))
        probs[i] = R.Problem(f, 0, k, m, n, n, 8, 0, f, k + 8, f, f, f, f, f, f)
    return probs


def test_batch_engine_selection_by_workspace_size(lib):
    shapes = [(700, 500, 40), (300, 200, 20), (1000, 900, 64)]
    probs = _problems(shapes)
    o = R.opts(q=1, d=2, pivot2=False, prec="bf16x3")
    size = {e: lib.rqlp_batched_workspace_size(probs, 3, ctypes.byref(o),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, c)))
            for e, c in R.ENGINES.items()}
    assert size["persistent"] > 0 and size["graph"] > 0
    assert size["auto"] == size["persistent"]
    # the persistent engine keeps every problem's BF16 copies of A at once
    assert size["persistent"] > 8 * sum(m * n for m, n, _ in shapes)
    # l = 136 > 128, a precision it lacks, a truncation: not for the persistent kernel
    big = _problems([(700, 500, 128)])
    for oo, pr in ((o, big), (R.opts(prec="tf32x3"), probs), (R.opts(truncate_k=True), probs)):
        n = 1 if pr is big else 3
        assert lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, 2))) == 0
        assert lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                               ctypes.byref(R.BatchTuning(4, 0, 0, 0))) == \
            lib.rqlp_batched_workspace_size(pr, n, ctypes.byref(oo),
                                            ctypes.byref(R.BatchTuning(4, 0, 0, 1)))
    assert lib.rqlp_batched_workspace_size(probs, 3, ctypes.byref(o),
                                           ctypes.byref(R.BatchTuning(4, 0, 0, 7))) == 0


def test_in_flight_option_needs_no_other_workspace(lib):
    # rqlp_opts.in_flight only changes the grid of the pivoted QR of B: the
    # workspace covers every grid; a negative count is invalid
    base = lib.rqlp_workspace_size(1000, 800, 20, 10, ctypes.byref(R.opts(q=1, d=2, pivot2=False)))
    assert base > 0
    for f in (1, 2, 8):
        o = R.opts(q=1, d=2, pivot2=False, in_flight=f)
        assert lib.rqlp_workspace_size(1000, 800, 20, 10, ctypes.byref(o)) == base
    assert lib.rqlp_workspace_size(1000, 800, 20, 10, ctypes.byref(R.opts(in_flight=-1))) == 0
    assert lib.rqlp_version() >= 201
