"""The FP64 norm of the fluence term (Section 2's |E x Hbar|) on the device:
one Newton step on s^2 = x from the single-precision reciprocal square root,
with the correctly rounded square root outside float's normal range.

Against numpy's correctly rounded square root: relative error below 2.5e-13
(the step's -3 e^2 / 2 for the seed's e < 2^-21.4, plus the rounding of its
three FP64 operations) across float's normal range and at its ends, exact
zeros, and the library's own result (bit for bit) for denormals, values past
2^128, infinity and NaN."""
import numpy as np
import pytest
import torch

from paper_2102_12978_gb300 import fdtd

pytestmark = pytest.mark.gpu

BOUND = 2.5e-13


def _norm(x: np.ndarray) -> np.ndarray:
    return fdtd.debug_vec_norm(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()).cpu().numpy()


def _rel(got, x):
    ref = np.sqrt(x)
    return np.abs(got - ref) / ref


def test_random_values_across_the_float_range():
    rng = np.random.default_rng(11)
    x = np.exp2(rng.uniform(-126.0, 128.0, 1 << 20))
    err = _rel(_norm(x), x)
    print("worst", err.max(), "mean", err.mean())
    assert err.max() < BOUND
    assert err.mean() < BOUND / 4


def test_every_mantissa_pattern_of_the_seed():
    """All 2^23 float mantissas of x in [1, 4) (both exponent parities of
    the square root), plus one random low mantissa word each."""
    m = np.arange(1 << 23, dtype=np.uint64)
    rng = np.random.default_rng(5)
    for e in (1023, 1024):
        bits = (np.uint64(e) << np.uint64(52)) | (m << np.uint64(29)) | rng.integers(0, 1 << 29, m.size,
                                                                                     dtype=np.uint64)
        x = bits.view(np.float64)
        err = _rel(_norm(x), x)
        assert err.max() < BOUND, (e, err.max())


def test_range_ends_and_exact_squares():
    lo, hi = 2.0 ** -126, 2.0 ** 128
    x = np.array([lo, np.nextafter(lo, 2.0), np.nextafter(hi, 0.0), 1.0, 4.0, 0.25, 2.0 ** 100, 2.0 ** -100,
                  9.0, 1e-30, 1e30, 3.0])
    err = _rel(_norm(x), x)
    assert err.max() < BOUND, err


def test_zero_and_library_cases():
    x = np.array([0.0, 5e-324, 1e-310, np.nextafter(2.0 ** -126, 0.0), 2.0 ** -127, 1e-300, 2.0 ** 128, 1e300,
                  np.inf, np.nan, 1.7976931348623157e308])
    got = _norm(x)
    ref = np.sqrt(x)
    assert got[0] == 0.0 and not np.signbit(got[0])
    np.testing.assert_array_equal(got, ref)


def test_empty_and_invalid_arguments():
    assert _norm(np.zeros(0)).size == 0
    with pytest.raises(TypeError):
        fdtd.debug_vec_norm(torch.zeros(4, dtype=torch.float32, device="cuda"))
