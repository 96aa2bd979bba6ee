"""CPU model of the FP32-pair ("double-float") arithmetic of dfloat.cuh.

The complex128 tile passes can compute in pairs of floats. This test replays
the same steps with numpy float32 (IEEE round-to-nearest; fmaf emulated by an
exact float64 product rounded once to float32 after the add) and checks the
properties the kernels rely on: the bit-pattern split of a double and the join
give back the double to 2^-46 relative; pair products and pair
multiply-adds keep about 2^-44 relative accuracy over random inputs; the
float -> double widening by bit pattern equals the hardware conversion.
"""
import numpy as np

f32 = np.float32


def fmaf(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def df_mul(a, b):
    p = f32(a[0] * b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    e = fmaf(a[1], b[0], e)
    return fast_two_sum(p, e)


def df_fma(a, b, c):
    p = f32(a[0] * b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    e = fmaf(a[1], b[0], e)
    s, t = two_sum(p, c[0])
    t = f32(t + f32(e + c[1]))
    return fast_two_sum(s, t)


M32, M64 = 0xFFFFFFFF, 0xFFFFFFFFFFFFFFFF


def u32(x):
    """A uint32 intermediate of the C code: wraps like the hardware."""
    return x & M32


def split(d):
    b = int(np.array([d], dtype=np.float64).view(np.uint64)[0])
    hi, lo = b >> 32, b & M32
    ex, sign = (hi >> 20) & 0x7FF, hi & 0x80000000
    u2f = lambda u: np.array([u32(u)], dtype=np.uint32).view(np.float32)[0]   # noqa: E731
    if ex <= 896:
        return f32(0), f32(0)
    h = u2f(sign | u32(u32(ex - 896) << 23) | u32((hi & 0xFFFFF) << 3) | (lo >> 29))
    if ex < 920:
        return h, f32(0)
    eb = u32(u32(ex - 919) << 23)
    return h, f32(u2f(sign | eb | ((lo & 0x1FFFFFFF) >> 6)) - u2f(sign | eb))


def widen(f):
    u = int(np.array([f], dtype=np.float32).view(np.uint32)[0])
    s = ((u & 0x80000000) << 32) & M64
    if (u & 0x7F800000) == 0:
        return np.array([s], dtype=np.uint64).view(np.float64)[0]
    # 64-bit intermediate, as in the C code (896 << 23 needs 34 bits)
    return np.array([s | ((((u & 0x7FFFFFFF) + (896 << 23)) << 29) & M64)], dtype=np.uint64).view(np.float64)[0]


def join(p):
    return widen(p[0]) + widen(p[1])


def test_split_join_and_widen():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-30, 0, 2000), [1.0, -1.0, 0.5, 2 ** -100]])
    for d in vals:
        h, l = split(float(d))
        assert abs(join((h, l)) - d) <= 2.0 ** -46 * abs(d) + 2.0 ** -125   # flush below 2^-126
        assert abs(l) <= abs(h) * 2.0 ** -22
        for f in (h, l):
            if f == 0 or abs(f) >= 2.0 ** -126:
                assert widen(f) == np.float64(f)
    assert split(1e-40) == (0, 0)


def test_pair_products_and_multiply_adds():
    rng = np.random.default_rng(1)
    worst_mul = worst_fma = 0.0
    for _ in range(3000):
        a, b, c = (float(x) for x in rng.uniform(-1, 1, 3))
        pa, pb, pc = split(a), split(b), split(c)
        m = join(df_mul(pa, pb))
        worst_mul = max(worst_mul, abs(m - a * b) / abs(a * b))
        r = join(df_fma(pa, pb, pc))
        worst_fma = max(worst_fma, abs(r - (a * b + c)) / max(abs(a * b), abs(c)))
    assert worst_mul < 2.0 ** -44 and worst_fma < 2.0 ** -44, (worst_mul, worst_fma)
