"""CPU pin of the algebra of the tensor-core MLP forward: an FP32 activation a enters the bf16
products as hi = bf16(a) and lo = bf16(a - hi) (round to nearest even). Then hi + lo equals a to
2^-16 relative, and a layer's sum over 64 terms of (hi + lo) w with bf16 weights w stays within
the bound that follows (2^-16 of sum |a w|), far inside the forward test's tolerance against the
FP64 oracle (1e-4 of the largest output)."""
import numpy as np


def _bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_bf16_rounding_emulation_is_exact_on_representable_values():
    x = np.array([1.0, -2.5, 0.15625, 3.0e-3], dtype=np.float32)
    xb = _bf16(x)
    assert np.array_equal(_bf16(xb), xb)                     # idempotent
    assert np.all(np.abs(xb - x) <= 2.0 ** -8 * np.abs(x))    # 8 significant bits
    assert _bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0          # a tie rounds to even


def test_hi_lo_split_carries_activations_to_two_to_the_minus_16():
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(200_000) * np.exp(rng.uniform(-6, 6, 200_000))).astype(np.float32)
    hi = _bf16(a)
    lo = _bf16(a.astype(np.float64) - hi.astype(np.float64))
    err = np.abs(a.astype(np.float64) - (hi.astype(np.float64) + lo.astype(np.float64)))
    assert np.all(err <= 2.0 ** -16 * np.abs(a))


def test_layer_sum_with_split_activations_meets_its_bound():
    rng = np.random.default_rng(5)
    K, N, B = 64, 64, 256
    a = np.tanh(rng.standard_normal((B, K))).astype(np.float32)
    w = _bf16(rng.standard_normal((N, K)).astype(np.float32) * 0.2).astype(np.float64)
    hi = _bf16(a).astype(np.float64)
    lo = _bf16(a.astype(np.float64) - hi).astype(np.float64)
    exact = a.astype(np.float64) @ w.T
    split = hi @ w.T + lo @ w.T
    bound = 2.0 ** -16 * (np.abs(a).astype(np.float64) @ np.abs(w).T)
    assert np.all(np.abs(split - exact) <= bound)
    assert np.abs(split - exact).max() <= 1e-4 * np.abs(exact).max()
