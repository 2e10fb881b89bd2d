"""Gauss-Jordan inversion with partial pivoting and no row exchanges, as the condensation's
prep kernel performs it in FP32 registers: step k pivots on the unused row p_k with the
largest |entry| in column k (lowest row on ties), scales it by 1/pivot (storing 1/pivot in
column k) and eliminates column k from every other row (storing -f/pivot there). The
tableau then holds the inverse with rows and columns in pivot order, inv[k][p_j] = T[p_k][j].
Checked here in FP64 against a library inverse, on matrices that need pivoting."""
import numpy as np
import pytest


def gj_virtual_pivot(A):
    n = A.shape[0]
    T = A.astype(np.float64).copy()
    used = np.zeros(n, bool)
    p_of, k_of = np.zeros(n, int), np.zeros(n, int)
    for k in range(n):
        cand = [r for r in range(n) if not used[r]]
        pr = max(cand, key=lambda r: (abs(T[r, k]), -r))
        ip = 1.0 / T[pr, k]
        p_of[k], k_of[pr], used[pr] = pr, k, True
        prow = T[pr] * ip
        prow[k] = ip
        for r in range(n):
            if r == pr:
                T[r] = prow
            else:
                f = T[r, k]
                T[r] = T[r] - f * prow
                T[r, k] = -f * ip
    inv = np.empty_like(T)
    for r in range(n):
        inv[k_of[r], p_of] = T[r]
    return inv, p_of


@pytest.mark.parametrize("n", [1, 5, 37, 100])
def test_virtual_pivot_inverse(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A[:, 0] *= 1e-6  # column 0's best pivot is not on the diagonal after a row shuffle
    A = A[rng.permutation(n)]
    inv, p_of = gj_virtual_pivot(A)
    ref = np.linalg.inv(A)
    assert np.abs(inv - ref).max() <= 1e-9 * np.abs(ref).max()
    assert sorted(p_of.tolist()) == list(range(n))


def test_zero_leading_entry_needs_pivoting():
    A = np.array([[0.0, 2.0, 1.0], [3.0, 1.0, 0.0], [1.0, 0.0, 4.0]])
    inv, p_of = gj_virtual_pivot(A)
    assert p_of[0] == 1  # |3| is the largest entry of column 0
    assert np.allclose(inv @ A, np.eye(3), atol=1e-14)
