"""The entry-wise parity measure the GPU tests use (CPU, no GPU needed).

It must catch what a normwise error hides: one small entry wrong by far more
than the tolerance while the 2-norm error stays below it.
"""
import numpy as np

from _parity import entrywise_err, grad_entrywise_err, per_rhs_entrywise_err


def test_entrywise_catches_a_small_component_that_normwise_misses():
    ref = np.ones((1000, 2))
    ref[:, 1] = 1e3
    x = ref.copy()
    x[7, 0] += 5e-9                     # column 0: entry error 5e-9 relative to max |ref| = 1
    normwise = np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert normwise[0] < 1e-9           # 5e-9 / sqrt(1000) = 1.6e-10
    assert abs(entrywise_err(x, ref) - 5e-9) < 1e-15
    assert per_rhs_entrywise_err(x, ref)[1] == 0.0


def test_entrywise_scales_each_column_by_its_own_largest_entry():
    ref = np.array([[1.0, 1e6], [0.5, 2e6]])
    x = ref + np.array([[0.0, 2.0], [1e-3, 0.0]])
    np.testing.assert_allclose(per_rhs_entrywise_err(x, ref), [1e-3, 1e-6])


def test_nonfinite_entries_fail_and_gradient_measure():
    assert entrywise_err(np.array([np.nan, 1.0]), np.array([1.0, 1.0])) == float("inf")
    g = np.array([3.0, -4.0, 1e-9])
    assert abs(grad_entrywise_err(g + np.array([0.0, 0.0, 4e-9]), g) - 1e-9) < 1e-15
