"""rqlp_cpqr_static(): the CPQR of B for callers that cannot allocate device memory.

Such callers (code under another runtime's memory manager that owns the
device memory, or loops where cudaMalloc's implicit synchronization is not
allowed) cannot pass a workspace; this entry point keeps its scratch in a
fixed array inside the library.  The test calls it through the C ABI twice
in a row, on different inputs, and checks each result against the
workspace-based rqlp_cpqr() entry point with the tolerance of the other CPQR
parity tests (pivots identical, R0 and Q0 to 1e-12 relative).
"""
import ctypes

import numpy as np
import pytest

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
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _static_cpqr(R, Bt, sync=1):
    n, l = Bt.shape
    R0t = torch.empty((n, l), dtype=torch.float64, device=Bt.device)
    piv = torch.empty((n,), dtype=torch.int32, device=Bt.device)
    Q0 = torch.empty((l, l), dtype=torch.float64, device=Bt.device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = R.lib().rqlp_cpqr_static(Bt.data_ptr(), n, l, l, R0t.data_ptr(), piv.data_ptr(),
                                    Q0.data_ptr(), sync, st)
    return code, R0t, piv, Q0


def _input(l, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((l, n)) * (0.999 ** np.arange(n))[None, :]
    return B, torch.from_numpy(np.ascontiguousarray(B.T)).cuda()


def test_static_cpqr_matches_workspace_entry_point(R):
    for call, (l, n) in enumerate([(30, 1000), (110, 8192)]):
        rng = np.random.default_rng(100 + call)
        B = rng.standard_normal((l, n)) * (0.999 ** np.arange(n))[None, :]
        Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
        code, R0t, piv, Q0 = _static_cpqr(R, Bt)
        assert code == 0, R.STATUS.get(code, code)
        Q0w, R0w, pivw = R.cpqr(Bt.t())
        assert torch.equal(piv.cpu(), pivw.cpu())
        assert _relmax(R0t.t(), R0w) <= 1e-12
        assert _relmax(Q0, Q0w) <= 1e-12


def test_static_cpqr_rejects_sizes_beyond_its_array(R):
    # slabs of 200000 x 256 doubles cannot sit in shared memory: rejected on the host
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = dummy.data_ptr()
    code = R.lib().rqlp_cpqr_static(p, 200000, 256, 256, p, p, p, 1, st)
    assert code == -6


def test_static_cpqr_queued_calls_share_the_array(R):
    # two calls enqueued back to back on one stream without waiting (sync = 0):
    # the second call clears the control block the first one used only after
    # the first has finished (same stream), so both results are right; they are
    # checked against the workspace entry point and the oracle's CPQR
    from oracle import rqlp_ref as O
    (B1, Bt1), (B2, Bt2) = _input(40, 3000, 7), _input(64, 2000, 8)
    c1, R1, p1, Q1 = _static_cpqr(R, Bt1, sync=0)
    c2, R2, p2, Q2 = _static_cpqr(R, Bt2, sync=0)
    assert c1 == 0 and c2 == 0
    torch.cuda.synchronize()
    for B, Bt, R0t, piv, Q0 in ((B1, Bt1, R1, p1, Q1), (B2, Bt2, R2, p2, Q2)):
        Q0w, R0w, pivw = R.cpqr(Bt.t())
        assert torch.equal(piv.cpu(), pivw.cpu())
        assert _relmax(R0t.t(), R0w) <= 1e-12
        Qo, Ro, po = O.cpqr(B)
        assert np.array_equal(piv.cpu().numpy(), po)
        assert _relmax(R0t.t(), torch.from_numpy(Ro)) <= 1e-12
        assert _relmax(Q0, torch.from_numpy(Qo)) <= 1e-12
