"""The seeded input generators against their definitions (no GPU): the
spectra of Example 5.1, the singular values of the generated matrices, and
determinism of the seeds."""
import numpy as np

from paper_1811_09334_gb300 import workloads as W


def test_pds_and_eds_spectra_follow_example_5_1():
    n, t = 12, 4
    # pds: t ones, then 2^-s, 3^-s, ..., (n - t + 1)^-s
    s = 2.0
    want = [1.0] * t + [j ** -s for j in range(2, n - t + 2)]
    assert np.allclose(W.pds_spectrum(n, t, s), want, rtol=0, atol=0)
    # eds: t ones, then 2^-s, 2^-2s, ..., 2^-(n - t)s
    s = 0.05
    want = [1.0] * t + [2.0 ** (-i * s) for i in range(1, n - t + 1)]
    assert np.allclose(W.eds_spectrum(n, t, s), want, rtol=1e-15, atol=0)


def test_generated_matrix_has_the_requested_singular_values():
    sigma = W.pds_spectrum(60, 5, 2.0)
    A = W.low_rank_from_spectrum(80, 60, sigma, 3)
    assert A.shape == (80, 60)
    got = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(got, np.sort(sigma)[::-1], rtol=1e-12, atol=1e-14)


def test_seeds_are_deterministic_and_distinct():
    a = W.omega(50, 7, 0)
    assert np.array_equal(a, W.omega(50, 7, 0))
    assert not np.array_equal(a, W.omega(50, 7, 1))
    assert abs(a.mean()) < 0.2 and 0.8 < a.std() < 1.2
