"""Integer-only conversions of the mixed-precision node update (cem_probe_split):
the FP32 pair (hi, lo) of a double and the float-to-double conversion, bit for
bit against NumPy's IEEE conversions, over magnitudes from subnormal to
overflow, signed zeros and non-finite values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOW29 = np.uint64((1 << 29) - 1)


def _doubles(rng):
    n = 200_000
    mag = 10.0 ** rng.uniform(-45, 45, n)
    x = np.where(rng.random(n) < 0.5, -mag, mag)
    # exactly representable floats (zero remainder) and remainders with every leading bit
    exact = rng.standard_normal(2000).astype(np.float32).astype(np.float64)
    lead = np.array([(1.0 + 2.0 ** -(24 + k)) * 2.0 ** e for k in range(29) for e in (-74, -20, 0, 127)])
    special = np.array([0.0, -0.0, 2.0 ** -74, np.nextafter(2.0 ** -74, 0), 2.0 ** -75, np.nextafter(2.0 ** 128, 0),
                        2.0 ** 128, -(2.0 ** 127), 1e-310, -1e-310, np.inf, -np.inf, np.nan, 1e300, 1.0, -1.0])
    return np.concatenate([x, exact, -exact, lead, -lead, special])


def _floats(rng, n):
    mag = (10.0 ** rng.uniform(-44, 38, n)).astype(np.float32)
    f = np.where(rng.random(n) < 0.5, -mag, mag).astype(np.float32)
    special = np.array([0.0, -0.0, 1e-40, -1e-40, 1.4e-45, np.inf, -np.inf, np.nan, 3.4e38, 1.17549435e-38],
                       dtype=np.float32)
    f[: special.size] = special
    return f


def _expected_split(x):
    b = x.view(np.uint64)
    E = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    zero = (b << np.uint64(1)) == 0
    fast = (E >= -74) & (E <= 127) & ~zero
    with np.errstate(invalid="ignore", over="ignore"):
        hi_t = (b & ~LOW29).view(np.float64)             # x truncated to 24 significant bits
        r = x - hi_t                                     # exact
        lo_t = (r.view(np.uint64) & ~LOW29).view(np.float64)
        hi_r = x.astype(np.float32)
        lo_r = (x - hi_r.astype(np.float64)).astype(np.float32)
        hi = np.where(fast, hi_t.astype(np.float32), hi_r)
        lo = np.where(fast, lo_t.astype(np.float32), lo_r)
    signed_zero = np.where(np.signbit(x), np.float32(-0.0), np.float32(0.0))
    return np.where(zero, signed_zero, hi), np.where(zero, signed_zero, lo), fast


def _same_bits(a, b):
    return (a.view(np.uint32 if a.dtype == np.float32 else np.uint64) ==
            b.view(np.uint32 if b.dtype == np.float32 else np.uint64)) | (np.isnan(a) & np.isnan(b))


def test_split_and_widen_are_bit_exact():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2508_04076_gb300 import probe_split
    rng = np.random.default_rng(11)
    x = _doubles(rng)
    f = _floats(rng, x.size)
    hi, lo, fd = probe_split(x, f)
    ehi, elo, fast = _expected_split(x)
    assert _same_bits(hi, ehi).all(), x[~_same_bits(hi, ehi)][:5]
    assert _same_bits(lo, elo).all(), x[~_same_bits(lo, elo)][:5]
    # the pair carries x to 2^-47 relative on the integer path
    err = np.abs(x[fast] - hi[fast].astype(np.float64) - lo[fast].astype(np.float64))
    assert (err <= 2.0 ** -47 * np.abs(x[fast])).all()
    assert fast.sum() > 100_000 and (~fast).sum() > 10
    assert _same_bits(fd, f.astype(np.float64)).all()
