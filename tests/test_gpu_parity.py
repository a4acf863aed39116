"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path): L and the L-values to 1e-10 relative (the target the
method's FP64 form is held to); pivots identical; Q and P elementwise to
1e-9 (they inherit the conditioning of the sketch, about 1e4 at most here);
the single products Y = A Omega and A^T V to 1e-13 relative (K <= 8192 terms
of FP64 rounding).
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


DEV = "cuda"


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _relmax(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# ------------------------------------------------------------------ products
@pytest.mark.parametrize("m,n,l", [(2000, 1000, 30), (333, 257, 17), (64, 64, 1), (1025, 130, 129)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_sketch_and_projection(R, m, n, l, dt):
    rng = np.random.default_rng(m + n + l)
    A = rng.standard_normal((m, n))
    if dt == "f32":
        A = A.astype(np.float32)
    Om = rng.standard_normal((n, l))
    V = rng.standard_normal((m, l))
    Y = R.sketch(_t(A), _t(Om))
    Z = R.project(_t(A), _t(V))
    A64 = A.astype(np.float64)
    assert _relmax(Y, O.sketch(A64, Om)) <= 1e-13
    assert _relmax(Z, O.adjoint_product(A64, V)) <= 1e-13


# ------------------------------------------------------------------ thin QR
@pytest.mark.parametrize("rows,l", [(2000, 30), (8192, 110), (300, 256), (7, 7), (129, 1)])
def test_orth_matches_householder(R, rows, l):
    A = W.low_rank_from_spectrum(rows, l, np.linspace(1.0, 0.01, l), 5)
    Q, Rr, status = R.orth(_t(A))
    Qo, Ro = O.householder_qr(A)
    assert status == 0
    assert _relmax(Q, Qo) <= 1e-11
    assert _relmax(Rr, Ro) <= 1e-12
    Qn = Q.cpu().numpy()
    assert np.abs(Qn.T @ Qn - np.eye(l)).max() <= 1e-14 * max(10, l)


def test_orth_shifted_pass_on_ill_conditioned_input(R):
    # condition number ~1e12: the first Gram matrix is numerically singular,
    # the shifted pass plus two more passes still give an orthonormal basis.
    sigma = np.logspace(0, -12, 40)
    A = W.low_rank_from_spectrum(3000, 40, sigma, 6)
    Q, Rr, status = R.orth(_t(A))
    assert status == R.RQLP_WARN_SHIFTED_CHOLQR
    Qn, Rn = Q.cpu().numpy(), Rr.cpu().numpy()
    assert np.abs(Qn.T @ Qn - np.eye(40)).max() <= 1e-13
    assert np.abs(Qn @ Rn - A).max() <= 1e-12 * np.abs(A).max()
    assert np.all(np.diag(Rn) > 0)


# ------------------------------------------------------------------ CPQR
@pytest.mark.parametrize("l,n", [(30, 1000), (110, 8192), (17, 17), (5, 3000), (256, 1200)])
def test_cpqr_matches_oracle(R, l, n):
    rng = np.random.default_rng(l * 7 + n)
    B = rng.standard_normal((l, n)) * (0.999 ** np.arange(n))[None, :]
    Q0, R0, piv = R.cpqr(_t(B))
    Qo, Ro, po = O.cpqr(B)
    assert np.array_equal(piv.cpu().numpy(), po)
    assert _relmax(R0, Ro) <= 1e-12
    assert _relmax(Q0, Qo) <= 1e-12


# ------------------------------------------------------------------ whole method
def _compare(out, ref, l, tolL=1e-10, tolQP=1e-9):
    Lg = out["L"].cpu().numpy()
    assert _relmax(Lg, ref["L"]) <= tolL
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])) <= tolL
    assert np.array_equal(out["piv0"].cpu().numpy()[:l], ref["piv0"][:l])
    assert np.array_equal(out["piv1"].cpu().numpy(), ref["piv1"])
    assert _relmax(out["Q"], ref["Q"]) <= tolQP
    assert _relmax(out["P"], ref["P"]) <= tolQP


@pytest.mark.parametrize("variant", [(True, 1), (False, 1), (False, 2), (False, 3)])
def test_c1_rqlp_fp64_parity(R, variant):
    """RQLP / ERQLP on the 2000 x 1000 sigma_j = j^-2 workload, k = 20, p = 10, q = 0."""
    pr = W.c1()
    Om = W.omega(pr.n, pr.l, 0)
    pivot2, d = variant
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=0, d=d, pivot2=pivot2)
    ref = O.rqlp(pr.A, pr.k, pr.p, Om, q=0, d=d, pivot2=pivot2)
    _compare(out, ref, pr.l)
    assert out["status"] == 0


@pytest.mark.parametrize("m,n,k,p,q,d,pivot2", [
    (777, 513, 13, 6, 1, 2, False),
    (1000, 1000, 100, 10, 1, 2, False),
    (513, 300, 40, 9, 2, 1, True),
    (4096, 640, 60, 4, 1, 4, False),
    (300, 200, 2, 0, 0, 1, True),
])
def test_ragged_shapes_with_power_steps(R, m, n, k, p, q, d, pivot2):
    sigma = 10.0 ** (-np.arange(1, min(m, n) + 1) / 100.0)
    A = W.low_rank_from_spectrum(m, n, sigma, m + n)
    Om = W.omega(n, k + p, 3)
    out = R.rqlp(_t(A), k, p, _t(Om), q=q, d=d, pivot2=pivot2)
    ref = O.rqlp(A, k, p, Om, q=q, d=d, pivot2=pivot2)
    _compare(out, ref, k + p)


def test_full_width_sketch_is_deterministic_qlp(R):
    # l = n (square Omega): the result is Stewart's pivoted QLP of A (Section 1).
    A, _ = W.low_rank_from_spectrum(90, 40, 0.85 ** np.arange(40), 9), None
    Om = W.omega(40, 40, 1)
    out = R.rqlp(_t(A), 30, 10, _t(Om), pivot2=True)
    ref = O.rqlp(A, 30, 10, Om, pivot2=True)
    _compare(out, ref, 40)
    s = np.linalg.svd(A, compute_uv=False)
    Ln = out["L"].cpu().numpy()
    assert np.allclose(np.linalg.svd(Ln, compute_uv=False), s, rtol=1e-11)


def test_factorization_invariants_on_gpu(R):
    pr = W.c1(m=1500, n=700, k=25, p=7)
    Om = W.omega(pr.n, pr.l, 2)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=1, d=2, pivot2=False)
    Q, L, P = (out[x].cpu().numpy() for x in ("Q", "L", "P"))
    l = pr.l
    assert np.abs(Q.T @ Q - np.eye(l)).max() <= 1e-13
    assert np.abs(P.T @ P - np.eye(l)).max() <= 1e-13
    assert np.abs(np.tril(L, -1)).max() == 0.0  # even d: upper middle factor
    E = pr.A - Q @ L @ P.T
    B = Q.T @ pr.A
    assert abs(np.linalg.norm(E) ** 2 - (np.linalg.norm(pr.A) ** 2 - np.linalg.norm(B) ** 2)) <= 1e-12


# ------------------------------------------------------------------ status paths
def test_nonfinite_input_is_reported(R):
    A = np.random.default_rng(1).standard_normal((200, 100))
    A[17, 3] = np.nan
    with pytest.raises(R.RqlpError) as e:
        R.rqlp(_t(A), 5, 5, _t(W.omega(100, 10, 0)))
    assert e.value.code == -2


def test_device_wait_timeout_is_reported_and_context_survives(R):
    # The first grid-wide exchange of the CPQR kernel waits for an exchange
    # number that never comes; the bounded wait gives up after 50 ms and
    # reports a status.
    pr = W.c1(m=400, n=300, k=10, p=5)
    Om = _t(W.omega(pr.n, pr.l, 0))
    A = _t(pr.A)
    with pytest.raises(R.RqlpError) as e:
        R.rqlp(A, pr.k, pr.p, Om, debug_flags=1, spin_limit_ns=50_000_000)
    assert e.value.code == -4
    out = R.rqlp(A, pr.k, pr.p, Om)
    assert out["status"] == 0


def test_host_entry_point_matches_device_path(R):
    pr = W.c1(m=1200, n=500, k=15, p=5)
    Om = W.omega(pr.n, pr.l, 4)
    dev = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=1, d=2, pivot2=False)
    host = R.rqlp_host(torch.from_numpy(pr.A).pin_memory(), pr.k, pr.p,
                       torch.from_numpy(Om).pin_memory(), q=1, d=2, pivot2=False)
    for key in ("Q", "L", "P", "Lvalues", "piv0", "piv1"):
        assert torch.equal(dev[key].cpu(), host[key]), key


def test_host_async_two_streams_match_device_path(R):
    """Two problems in flight on two streams (the double-buffered host path):
    every result equals that problem's device-path result, including when a
    slot's workspace and host buffers are reused for the next problem."""
    probs = []
    for seed, (m, n) in enumerate(((900, 400), (700, 500))):
        pr = W.c1(m=m, n=n, k=12, p=4)
        Om = W.omega(pr.n, pr.l, seed)
        dev = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), q=1, d=2, pivot2=False, prec="bf16x3")
        probs.append((torch.from_numpy(pr.A).pin_memory(), torch.from_numpy(Om).pin_memory(),
                      pr, {k: dev[k].cpu() for k in ("Q", "L", "P", "Lvalues", "piv0", "piv1")}))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    slots = [None, None]
    for i in range(4):
        A_h, Om_h, pr, ref = probs[i % 2]
        sl = slots[i % 2]
        if sl is not None:
            R.host_wait(sl)
            for key, v in ref.items():
                assert torch.equal(sl[key], v), (i, key)
        slots[i % 2] = R.rqlp_host_async(
            A_h, pr.k, pr.p, Om_h, q=1, d=2, pivot2=False, prec="bf16x3",
            ws=None if sl is None else sl["ws"],
            out=None if sl is None else {k: sl[k] for k in ref}, stream=streams[i % 2])
    for i, sl in enumerate(slots):
        R.host_wait(sl)
        for key, v in probs[i][3].items():
            assert torch.equal(sl[key], v), (i, key)


@pytest.fixture(scope="module")
def c2_full():
    pr = W.c2(device=DEV)
    return pr, pr.A.cpu().numpy(), W.omega(pr.n, pr.l, 0)


@pytest.mark.slow
@pytest.mark.parametrize("q", [1, 2])
def test_c2_full_size_fp64_parity(R, c2_full, q):
    """The 8192 x 8192 ERQLP workload (q = 1 and 2, d = 2) in the launch
    configuration the benchmark times, against the oracle run on the same matrix."""
    pr, A_np, Om = c2_full
    out = R.rqlp(pr.A, pr.k, pr.p, _t(Om), q=q, d=2, pivot2=False)
    ref = O.rqlp(A_np, pr.k, pr.p, Om, q=q, d=2, pivot2=False)
    _compare(out, ref, pr.l)
    # the FP64TC form (digit products on the tensor cores) at the same tolerances
    tc = R.rqlp(pr.A, pr.k, pr.p, _t(Om), q=q, d=2, pivot2=False, prec="fp64tc")
    _compare(tc, ref, pr.l)
    if q == 2:
        # the same matrix in BF16x3 at q = 2: pivots identical, L-values to 1e-3
        mx = R.rqlp(pr.A, pr.k, pr.p, _t(Om), q=q, d=2, pivot2=False, prec="bf16x3")
        assert np.array_equal(mx["piv0"].cpu().numpy()[:pr.l], ref["piv0"][:pr.l])
        lv = mx["Lvalues"].cpu().numpy()
        keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"][0]
        assert (np.abs(lv - ref["Lvalues"])[keep] / ref["Lvalues"][keep]).max() <= 1e-3


# ------------------------------------------------------------------ BRQLP
@pytest.mark.parametrize("b,pivot2,d", [(10, True, 1), (6, True, 1), (15, False, 2), (30, True, 1),
                                        (5, False, 1)])
def test_brqlp_parity(R, b, pivot2, d):
    """Algorithm 4.1 on the 2000 x 1000 workload (l = 30) against the oracle,
    which forms the deflated A(j) literally."""
    pr = W.c1()
    Om = W.omega(pr.n, pr.l, 5)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), pivot2=pivot2, d=d, block_b=b)
    ref = O.brqlp(pr.A, pr.k, pr.p, b, Om, pivot2=pivot2, d=d)
    Lg = out["L"].cpu().numpy()
    assert _relmax(Lg, ref["L"]) <= 1e-10
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / np.abs(ref["Lvalues"])) <= 1e-10
    assert _relmax(out["Q"], ref["Q"]) <= 1e-9
    assert _relmax(out["P"], ref["P"]) <= 1e-9
    # A - Q L P^T = A - V B (eq. 4.5): the residual identity of eq. 2.1
    Q, P = out["Q"].cpu().numpy(), out["P"].cpu().numpy()
    E = pr.A - Q @ Lg @ P.T
    Bn = np.linalg.norm(Q.T @ pr.A)
    assert abs(np.linalg.norm(E) ** 2 - (np.linalg.norm(pr.A) ** 2 - Bn ** 2)) <= 1e-12


def test_brqlp_large_blocks_bf16x3(R):
    pr = W.c2(m=4096, n=3000, k=90, p=10)
    Om = W.omega(pr.n, pr.l, 6)
    out = R.rqlp(_t(pr.A), pr.k, pr.p, _t(Om), pivot2=True, block_b=20, prec="bf16x3")
    ref = O.brqlp(pr.A, pr.k, pr.p, 20, Om, pivot2=True)
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"]) / ref["Lvalues"]) <= 1e-3


def _block_residuals(A, B, b):
    """||A - V V^T A||_F / ||A||_F after each block, from eq. 2.1 (oracle B)."""
    a2 = float(np.sum(A * A))
    return [np.sqrt(max(a2 - float(np.sum(B[:(j + 1) * b] ** 2)), 0.0) / a2)
            for j in range(B.shape[0] // b)]


@pytest.mark.parametrize("tol,l_expect", [(0.03, 16), (5e-3, 40), (1e-3, 64)])
def test_brqlp_tol_parity(R, tol, l_expect):
    """Fixed-accuracy BRQLP (blocks of 8, at most 64 columns) on the
    900 x 600 sigma_j = j^-2 matrix: the same number of blocks as the oracle
    and the same factorization; every tolerance is at least 10 % away from
    the residual after any block, so the stopping block is unambiguous."""
    pr = W.c1(m=900, n=600, k=20, p=10)
    b, l_max = 8, 64
    Om = W.omega(pr.n, l_max, 5)
    full = O.brqlp_tol(pr.A, b, l_max, 0.0, Om)
    assert all(abs(r - tol) > 0.1 * tol for r in _block_residuals(pr.A, full["B"], b))
    ref = O.brqlp_tol(pr.A, b, l_max, tol, Om)
    assert ref["l"] == l_expect
    out = R.brqlp_tol(_t(pr.A), b, l_max, tol, _t(Om))
    assert out["l"] == ref["l"]
    Lg = out["L"].cpu().numpy()
    assert _relmax(Lg, ref["L"]) <= 1e-10
    # L-values normwise (relative to the largest): the GPU forms B_j = V_j^T A
    # where the oracle deflates A(j-1) literally (reading A8), so the
    # smallest L-values of the deeper blocks (3.5e-4 of the largest at
    # l = 64) differ by rounding of order 1e-14 absolute
    lv = out["Lvalues"].cpu().numpy()
    assert np.max(np.abs(lv - ref["Lvalues"])) <= 1e-10 * np.max(np.abs(ref["Lvalues"]))
    assert _relmax(out["Q"], ref["Q"]) <= 1e-9
    assert _relmax(out["P"], ref["P"]) <= 1e-9
    # below l_max the tolerance holds for the returned factors, computed directly
    if out["l"] < l_max:
        Q, P = out["Q"].cpu().numpy(), out["P"].cpu().numpy()
        assert np.linalg.norm(pr.A - Q @ Lg @ P.T) <= tol * np.linalg.norm(pr.A)


def test_brqlp_tol_zero_is_the_fixed_block_count(R):
    pr = W.c1(m=900, n=600, k=20, p=10)
    b, l_max = 8, 32
    Om = _t(W.omega(pr.n, l_max, 5))
    A = _t(pr.A)
    out = R.brqlp_tol(A, b, l_max, 0.0, Om)
    fix = R.rqlp(A, l_max, 0, Om, block_b=b)
    assert out["l"] == l_max
    for key in ("Q", "L", "P", "Lvalues", "piv0", "piv1"):
        assert torch.equal(out[key], fix[key]), key


def test_brqlp_tol_bf16x3(R):
    # the mixed form's products carry ~1e-5 relative errors, so ||A||^2 -
    # ||B||^2 is known to about 1e-5 ||A||^2: tolerances well above
    # sqrt(1e-5) ~ 3e-3 keep the stopping block unambiguous
    pr = W.c1(m=900, n=600, k=20, p=10)
    b, l_max = 8, 64
    Om = W.omega(pr.n, l_max, 5)
    ref = O.brqlp_tol(pr.A, b, l_max, 0.03, Om)
    out = R.brqlp_tol(_t(pr.A), b, l_max, 0.03, _t(Om), prec="bf16x3")
    assert out["l"] == ref["l"] == 16
    lv = out["Lvalues"].cpu().numpy()
    keep = ref["Lvalues"] >= 1e-3 * ref["Lvalues"].max()
    assert np.max(np.abs(lv - ref["Lvalues"])[keep] / ref["Lvalues"][keep]) <= 1e-3


# ------------------------------------------------------------------ device helpers
def test_device_arithmetic_helpers_match_cuda(R):
    # integer-pipe FP64/FP32 roundings bit-exact, FP32-seeded reciprocal and
    # reciprocal square root within 2^-51 relative, on 2^20 inputs each
    assert R.selftest(1 << 20) == [0, 0, 0, 0]
