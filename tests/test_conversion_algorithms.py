"""The integer-pipe format conversions of the mixed form's RK stage
(widen_f32 and narrow_f64_rn in csrc/hx_common.cuh) restated step for step
on the bit patterns in Python and checked against IEEE 754 conversions
(numpy's float32 <-> float64 casts, round to nearest, ties to even) on
random values and on the edge cases: ties, carries into the exponent,
overflow to infinity, subnormal results, zeros, infinities and NaNs.  The
device code itself is checked bit for bit on the GPU (the FP32 stage copy
equals CUDA's cast of the FP64 state)."""
import numpy as np


def widen_f32(b):
    """FP32 bit pattern -> FP64 bit pattern, the steps of widen_f32."""
    s, em = b & 0x80000000, b & 0x7FFFFFFF
    if 0x00800000 <= em < 0x7F800000:
        hi = s | ((em >> 3) + (896 << 20))
        lo = (em << 29) & 0xFFFFFFFF
        return (hi << 32) | lo
    if em == 0:
        return s << 32
    if em >= 0x7F800000:
        return (s | (0x7FF00000 if em == 0x7F800000 else 0x7FF80000)) << 32
    n = em.bit_length() - 1
    m = (em << (52 - n)) & 0x000FFFFFFFFFFFFF
    return (s << 32) | ((n + 874) << 52) | m


def narrow_f64_rn(b):
    """FP64 bit pattern -> FP32 bit pattern, the steps of narrow_f64_rn."""
    hi, lo = b >> 32, b & 0xFFFFFFFF
    s = hi & 0x80000000
    e = (hi >> 20) & 0x7FF
    if e == 0x7FF:
        return s | 0x7F800000 | (0x400000 if ((hi & 0xFFFFF) | lo) else 0)
    fe = e - 896
    if fe >= 0xFF:
        return s | 0x7F800000
    if fe > 0:
        mant = ((hi & 0xFFFFF) << 3) | (lo >> 29)
        rem = lo & 0x1FFFFFFF
        up = 1 if (rem > 0x10000000 or (rem == 0x10000000 and (mant & 1))) else 0
        return s | (((fe << 23) | mant) + up)
    if e == 0:
        return s
    m = ((hi & 0xFFFFF) << 32 | lo) | (1 << 52)
    sh = 926 - e
    if sh >= 64:
        return s
    q, rem, half = m >> sh, m & ((1 << sh) - 1), 1 << (sh - 1)
    return s | (q + (1 if (rem > half or (rem == half and (q & 1))) else 0))


def _f32_bits(x):
    return int(np.array(x, dtype=np.float32).view(np.uint32))


def _f64_bits(x):
    return int(np.array(x, dtype=np.float64).view(np.uint64))


def _check_narrow(values):
    for v in values:
        v = np.float64(v)
        got = narrow_f64_rn(_f64_bits(v))
        with np.errstate(over="ignore"):
            ref = np.float32(v)
        if np.isnan(v):
            assert (got & 0x7F800000) == 0x7F800000 and (got & 0x7FFFFF)
        else:
            assert got == _f32_bits(ref), (v, hex(got), hex(_f32_bits(ref)))


def test_widen_is_exact_on_every_class():
    rng = np.random.default_rng(7)
    bits = list(rng.integers(0, 2 ** 32, size=20000, dtype=np.uint64))
    bits += [0, 0x80000000, 1, 0x80000001, 0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000,
             0x3F800000, 0x00400000, 0x00000100]
    for b in bits:
        b = int(b)
        f = np.array(b, dtype=np.uint32).view(np.float32)
        got = widen_f32(b)
        if np.isnan(f):
            assert (got >> 52) & 0x7FF == 0x7FF and (got & 0x000FFFFFFFFFFFFF)
        else:
            assert got == _f64_bits(np.float64(f)), hex(b)


def test_narrow_rounds_to_nearest_even_on_random_values():
    rng = np.random.default_rng(11)
    vals = np.concatenate([rng.normal(size=5000), rng.normal(size=2000) * 1e-3,
                           np.exp(rng.uniform(-100, 100, size=5000)) * rng.choice([-1, 1], size=5000)])
    _check_narrow(vals)


def test_narrow_ties_carries_and_limits():
    vals = []
    for f in (1.0, 1.5, 3.0, 1.9999998807907104, 1e-30, 3.4e38):
        b = _f64_bits(np.float64(np.float32(f)))
        for d in (-1, 0, 1):   # exactly halfway between two FP32 neighbours, and just around it
            vals.append(np.array(b + (1 << 28) + d, dtype=np.uint64).view(np.float64))
            vals.append(np.array(b + (3 << 28) + d, dtype=np.uint64).view(np.float64))
    fmax = float(np.finfo(np.float32).max)
    vals += [fmax, np.nextafter(fmax, np.inf), fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), 1e39, -1e300,
             np.inf, -np.inf, np.nan, 0.0, -0.0, 5e-324, 1e-310]
    _check_narrow(vals)


def test_narrow_to_fp32_subnormals():
    tiny = float(np.finfo(np.float32).tiny)        # 2^-126
    sub = 2.0 ** -149                              # smallest FP32 subnormal
    vals = [tiny, tiny * (1 - 2.0 ** -24), tiny * (1 - 2.0 ** -25), tiny / 3, sub, sub / 2, sub * 0.5000001,
            sub * 1.5, sub * 2.5, sub * 0.49, -sub * 3.5, 1e-40, -2.5e-39, 2.0 ** -150, 2.0 ** -151]
    rng = np.random.default_rng(3)
    vals += list(np.exp(rng.uniform(np.log(2.0 ** -160), np.log(tiny), size=3000)))
    _check_narrow(vals)
