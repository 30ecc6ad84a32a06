"""The per-node comparison the GPU parity tests use catches what a norm-wise one misses."""
import numpy as np

from nodewise import rel


def test_single_node_error_fails_per_node():
    rng = np.random.default_rng(0)
    ref = rng.standard_normal(73 * 73) + 1j * rng.standard_normal(73 * 73)
    a = ref.copy()
    a[5] += 2e-5 * np.abs(ref).max()  # one node off by 2e-5 of the largest value
    normwise = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    assert normwise < 2e-6  # would pass a norm-wise complex64 tolerance
    assert rel(a, ref) > 2e-6


def test_dirichlet_zero_must_be_exact():
    ref = np.array([0.0, 1.0, 2.0], dtype=complex)
    assert rel(np.array([0.0, 1.0, 2.0], dtype=complex), ref) == 0.0
    assert rel(np.array([1e-30, 1.0, 2.0], dtype=complex), ref) == float("inf")


def test_rounding_level_differences_pass():
    rng = np.random.default_rng(1)
    ref = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    a = (ref.astype(np.complex64)).astype(np.complex128)
    assert rel(a, ref) < 1e-7
