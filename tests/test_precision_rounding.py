"""Host checks of the IEEE facts the 16-bit step kernels rely on (no GPU).

* The internal-energy balance of the temperature recovery, e - rho u^2 / 2,
  is one subtraction of two FP32 numbers.  FP32's correctly rounded
  subtraction gives the value that converting both to FP64, subtracting and
  rounding back would: the exact difference is an FP64 number when the
  exponents differ by at most 28, and otherwise lies within 2^-28 of the
  larger operand, far from any FP32 rounding tie.
* The range tests of the software stochastic rounding (the register-pull
  kernel and the wall values written into ghost slots; the pulled-row
  kernels round in hardware and test nothing) select the values they are
  meant to: FP16 |v| < 255.875 <=> |256 v| < 65504, BF16 |v| <= FLT_MAX <=>
  v finite.
"""
import numpy as np

F32_MAX = np.float32(3.40282347e38)


def _random_f32(rng, n, emin, emax):
    mant = rng.uniform(1.0, 2.0, n)
    exp = rng.integers(emin, emax, n)
    sign = rng.choice([-1.0, 1.0], n)
    return (sign * np.ldexp(mant, exp)).astype(np.float32)


def test_fp32_subtraction_equals_fp64_rounded_back():
    rng = np.random.default_rng(11)
    n = 2_000_000
    a = _random_f32(rng, n, -30, 10)
    # b spans exponent gaps of 0 .. 60 below and above a, and near-equal values
    gap = rng.integers(-60, 61, n)
    b = (a * np.ldexp(rng.uniform(0.5, 2.0, n), gap)).astype(np.float32)
    b[: n // 8] = np.nextafter(a[: n // 8], np.float32(np.inf))  # cancellation
    b[n // 8: n // 4] = -b[n // 8: n // 4]  # opposite signs: a carry
    with np.errstate(over="ignore", under="ignore"):
        r32 = a - b
        r64 = (a.astype(np.float64) - b.astype(np.float64)).astype(np.float32)
    fin = np.isfinite(r32)
    assert fin.mean() > 0.99
    np.testing.assert_array_equal(r32[fin].view(np.uint32), r64[fin].view(np.uint32))


def test_energy_balance_form_of_the_kernel():
    # e = rho (Es - b/6) and the kinetic term, both small, as the kernel forms them
    rng = np.random.default_rng(12)
    n = 1_000_000
    rho = (1 + 1e-3 * rng.standard_normal(n)).astype(np.float32)
    ux = (0.1 * rng.standard_normal(n)).astype(np.float32)
    uy = (0.1 * rng.standard_normal(n)).astype(np.float32)
    kin = np.float32(0.5) * (rho * (ux * ux + uy * uy))
    e = (kin + (1e-2 * rng.standard_normal(n)).astype(np.float32)).astype(np.float32)
    e[: n // 10] = kin[: n // 10]  # exact balance: theta = 1
    r32 = e - kin
    r64 = (e.astype(np.float64) - kin.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(r32.view(np.uint32), r64.view(np.uint32))


def test_stochastic_rounding_range_tests():
    rng = np.random.default_rng(13)
    v = np.concatenate([
        _random_f32(rng, 1_000_000, -40, 12),
        np.float32([255.875, 255.87498, 255.87502, -255.875, 0.0, -0.0, np.inf, -np.inf, np.nan]),
        np.nextafter(np.float32(255.875), np.float32([0, np.inf, -np.inf])).astype(np.float32),
    ]).astype(np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        per_value = np.abs(v * np.float32(256)) < np.float32(65504)
        per_node = np.abs(v) < np.float32(255.875)
    np.testing.assert_array_equal(per_value, per_node)
    u = np.concatenate([v, np.float32([F32_MAX, -F32_MAX, 1e38])]).view(np.uint32)
    w = u.view(np.float32)
    with np.errstate(invalid="ignore"):
        np.testing.assert_array_equal((u & 0x7F800000) != 0x7F800000, np.abs(w) <= F32_MAX)
