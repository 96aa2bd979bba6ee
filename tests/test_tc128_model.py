"""Host-side models of the complex128 tensor-core pass (k_tc128, no GPU).

They restate in Python, with numpy float32 arithmetic (IEEE round to nearest,
the rounding of the kernel's __fadd_rn / __fmul_rn / __fmaf_rn steps, whose
FMAs here only add a power-of-two multiple), the kernel's arithmetic and check
what it relies on:

* digits (the pass stores them negated, its chain being the exact negation of
  the one restated here; a test checks that bit for bit): every FP64 value of
  a row becomes six integer digits with
  |d| <= 260 whose sum 2^(E-8) sum_i d_i 2^(-9 i) is within 2^(E-46) of it;
  the host's W digits (six, balanced, |g| <= 256) are within 2^-54 of w;
* exactness: the level sums of a 64-term row (levels 0..2, and 3 short of an
  adversarial alignment) stay below 2^24, so FP32 accumulation is exact;
* the combination of the six levels back to FP64 (FP32 pairs joined by
  integer arithmetic) equals their exact sum to 2^-46 relative, including
  results just below a power of two;
* the FP32-pair form kept between consecutive passes: digits taken from a
  pair, and a row read and written as pairs, keep the same bounds;
* a whole row: U psi through digits, level sums (six accumulators, levels 0-2
  exact) and the combination is within 2^-46 ||a||_2 + 2^(E-49) of the
  FP64 product (2^-48 ||a||_2 + 2^(E-49) when the row is read as FP32
  pairs), ||a||_2 the row's 2-norm and 2^E its scale (|a| < 2^E <= 2 max
  |a|), for Haar-random blocks and rows of every shape (random, one non-zero
  entry, mixed magnitudes, FP64 zeros and subnormals, exact powers of two);
  the bound is tight enough that a model with one planted mistake (a digit
  plane of A or W dropped, the level-4 or level-5 accumulator lost, a level's sign
  flipped, the block transposed) fails it;
* indexing: runs of >= 2^7 amplitudes land every element (row, column) of a
  tile at its tile-local index, the tiles partition the state, and stores
  go to roff(row) | coff(column) of the tile;
* barriers: the single-buffered A and accumulator protocol (with the row
  exponent exchange, the exponent table, and the two-step release of the
  accumulators: levels 4-5 once combined in registers, levels 0-3 once read)
  has no deadlock or hazard under random delays, for 1 to 54 tiles per CTA,
  with and without W reloads.
"""
import random
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32
MAGIC = F32(12582912.0)


def f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def rint32(x):
    return (x + MAGIC) - MAGIC


# ---------------------------------------------------------------- kernel arithmetic, restated

def digits(a, emax_b):
    """t2_digits over an array of FP64 values of one row (emax_b per value)."""
    u = np.asarray(a, dtype=np.float64).view(np.uint64)
    whi = (u >> np.uint64(32)).astype(np.int64)
    wlo = (u & np.uint64(0xFFFFFFFF)).astype(np.int64)
    ex = (whi >> 20) & 0x7FF
    fe = ex + 134 - np.asarray(emax_b, dtype=np.int64)
    sign = whi & 0x80000000
    ok = (ex != 0) & (fe >= 87)
    fe_ok = np.where(ok, fe, 127)
    hi = f32((sign | (fe_ok << 23) | ((whi & 0xFFFFF) << 3) | (wlo >> 29)).astype(np.uint32))
    eb = (fe_ok - 5) << 23
    lo18 = f32((sign | eb | ((wlo & 0x1FFFFFFF) >> 6)).astype(np.uint32)) - f32((sign | eb).astype(np.uint32))
    hi = np.where(ok, hi, F32(0))
    lo18 = np.where(ok, lo18, F32(0))
    d0 = rint32(hi)
    t = hi - d0
    u1 = t * F32(512)
    d1 = rint32(u1)
    t = u1 - d1
    v = t * F32(512) + lo18               # fmaf(t, 512, lo18): t * 512 is exact
    d2 = rint32(v)
    r = (t * F32(512) - d2) + lo18        # fmaf(t, 512, -d2) is exact
    u3 = r * F32(512)
    d3 = rint32(u3)
    t = u3 - d3
    u4 = t * F32(512)
    d4 = rint32(u4)
    t = u4 - d4
    d5 = rint32(t * F32(512))
    return np.stack([d0, d1, d2, d3, d4, d5]).astype(np.float64)


def digits_pair(s, e, E):
    """t2_digits_pair: the digits of s + e (FP32 pairs) for a row of scale 2^E."""
    hi = np.asarray(s, dtype=np.float32) * F32(2.0 ** (8 - E))
    lo18 = np.asarray(e, dtype=np.float32) * F32(2.0 ** (26 - E))
    d0 = rint32(hi)
    t = hi - d0
    u1 = t * F32(512)
    d1 = rint32(u1)
    t = u1 - d1
    d2 = rint32(t * F32(512) + lo18)
    t = (t * F32(512) - d2) + lo18
    u3 = t * F32(512)
    d3 = rint32(u3)
    t = u3 - d3
    u4 = t * F32(512)
    d4 = rint32(u4)
    t = u4 - d4
    d5 = rint32(t * F32(512))
    return np.stack([d0, d1, d2, d3, d4, d5]).astype(np.float64)


def to_pairs(a):
    """FP64 values as normalised FP32 pairs (s, e), s + e = a to about 2^-48."""
    s = np.asarray(a, dtype=np.float64).astype(np.float32)
    e = (np.asarray(a, dtype=np.float64) - s.astype(np.float64)).astype(np.float32)
    return s, e


def pair_row_scale(s):
    """E of a row held as pairs: max biased FP32 exponent - 126, at least -101."""
    ex = (np.asarray(s, dtype=np.float32).view(np.uint32) >> np.uint32(23)) & np.uint32(0xFF)
    return max(int(ex.max()) - 126, -101)


def fold(c):
    """The drainer's fold of the six level sums (float32) into an FP32 pair
    (s, e): levels 4 and 5 first combined into one value t (one rounding: both
    products are exact), which starts the error word; then TwoSum of levels
    1-3 into level 0, each TwoSum's error added to the error word."""
    c0, c1, c2, c3, c4, c5 = (F32(x) for x in c)
    e = c4 * F32(2.0 ** -36) + c5 * F32(2.0 ** -45)
    s = c0
    for l, cl in ((1, c1), (2, c2), (3, c3)):
        s, e2 = two_sum(s, cl * F32(2.0 ** (-9 * l)))
        e = e + e2
    return s, e


def pair_out(c, E):
    """The drainer's pair output: levels folded, FastTwoSum, scaled by 2^(E - 16)."""
    s, e = fold(c)
    t = s + e
    e = e - (t - s)
    sc = F32(2.0 ** (E - 16))
    return t * sc, e * sc


def w_digits(w):
    """build_w_digits for one value: balanced digits of X = rint(w 2^53)."""
    X = int(np.rint(np.ldexp(np.float64(w), 53)))
    g = [0] * 6
    for j in range(5, 0, -1):
        g[j] = ((X + 256) & 511) - 256
        X = (X - g[j]) // 512
    g[0] = X
    return g


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def combine(c, emax_b):
    """t2_join after the fold: six level sums (float32) -> FP64 value
    2^(emax_b - 1038) sum_l c_l 2^(-9 l) (emax_b = E + 1022)."""
    s, e = fold(c)
    s2 = s + e
    e = e - (s2 - s)
    s = s2
    us = int(np.array(s, dtype=np.float32).view(np.uint32))
    fs = (us >> 23) & 0xFF
    de = fs + emax_b - 142
    if fs == 0 or de <= 0:
        return 0.0
    mag = (de << 52) | ((us & 0x7FFFFF) << 29)
    if 46 <= fs <= 254:
        sc = f32(np.uint32((300 - fs) << 23))
        k = int(np.array((e * sc) + MAGIC, dtype=np.float32).view(np.int32)) - 0x4B400000
        adj = (-k if us >> 31 else k) << 6
        if (us & 0x7FFFFF) == 0 and adj < 0:
            adj *= 2
        mag += adj
    bits = ((us >> 31) << 63) | mag
    return float(np.array(bits, dtype=np.uint64).view(np.float64))


def row_emax(vals):
    u = np.asarray(vals, dtype=np.float64).view(np.uint64)
    return int(((u >> np.uint64(52)) & np.uint64(0x7FF)).max())


def apply_row(U, a, pairs_in=False, pairs_out=False, plant=None):
    """One output row of the pass: U (32x32 complex) applied to a (32 complex)
    the kernel's way, reading FP64 values or FP32 pairs and writing FP64
    values or pairs (returned joined in FP64 for comparison). `plant` puts one
    deliberate mistake into the model (a test shows the bound catches it)."""
    reals = np.empty(64)
    reals[0::2], reals[1::2] = a.real, a.imag
    if pairs_in:
        ps, pe = to_pairs(reals)
        E = pair_row_scale(ps)
        D = digits_pair(ps, pe, E)
    else:
        E = max(row_emax(reals) - 1022, -101)
        D = digits(reals, np.full(64, E + 1022))
    em = E + 1022
    assert np.abs(D).max() <= 260
    if plant == "no_a_digit5":
        D[5] = 0
    Wd = np.zeros((6, 64, 64), dtype=np.int64)       # [j][k][nn]
    for co in range(32):
        for ci in range(32):
            u = U[co, ci]
            for k, nn, w in ((2 * ci, 2 * co, u.real), (2 * ci, 2 * co + 1, u.imag),
                             (2 * ci + 1, 2 * co, -u.imag), (2 * ci + 1, 2 * co + 1, u.real)):
                Wd[:, k, nn] = w_digits(w)
    assert np.abs(Wd).max() <= 256
    if plant == "no_w_digit5":
        Wd[5] = 0
    if plant == "w_transposed":
        Wd = Wd.transpose(0, 2, 1).copy()
    Di = D.astype(np.int64)
    out = np.empty(64)
    for nn in range(64):
        lev = []
        for l in range(6):
            tot = 0
            for i in range(l + 1):
                # one K = 16 MMA per k-step: the accumulator after each step
                for ks in range(4):
                    tot += int((Di[i, 16 * ks:16 * ks + 16] * Wd[l - i, 16 * ks:16 * ks + 16, nn]).sum())
                    if l <= 2:
                        assert abs(tot) < 2 ** 24, "an exact level left the FP32 integer range"
            if plant == "no_level4" and l == 4:
                tot = 0
            if plant == "no_level5" and l == 5:
                tot = 0
            if plant == "level1_sign" and l == 1:
                tot = -tot
            lev.append(F32(float(tot)))                # exact for levels <= 2 (checked), rounded above
        if pairs_out:
            so, eo = pair_out(lev, E)
            out[nn] = float(so) + float(eo)
        else:
            out[nn] = combine(lev, em)
    return out[0::2] + 1j * out[1::2], em


def row_bound(a, em, pairs_in=False):
    """The per-output error bound of one pass: the digit split keeps 47 bits
    of each FP64 value (truncation below 2^-46 relative; an FP32 pair holds
    its value to 2^-48), which a unit column of W turns into at most that
    fraction of the row's 2-norm (Cauchy-Schwarz); the last digit's rounding,
    W's digit tails (2^-54 per entry) and the roundings of levels 3-5 add less
    than 2^(E-49)."""
    nrm = float(np.sqrt(np.sum(np.abs(a) ** 2)))
    return (2.0 ** -48 if pairs_in else 2.0 ** -46) * nrm + 2.0 ** (em - 1022 - 49)


def haar(d, rng):
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


# ---------------------------------------------------------------- arithmetic checks

def test_digits_reconstruct_every_value_of_a_row():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-12, 1, 4000),
                           [0.0, -0.0, 5e-324, -2.2e-308, 1.0, -1.0, 0.5, 2.0 ** -30, 1 - 2 ** -53, 0.999999999]])
    for em_extra in (0, 1, 7, 30):
        em = row_emax(vals) + em_extra
        E = em - 1022
        assert np.all(np.abs(vals) < 2.0 ** E)
        D = digits(vals, np.full(vals.shape, em))
        assert np.abs(D).max() <= 260
        rec = np.zeros_like(vals)
        for i in range(6):
            rec += D[i] * 2.0 ** (-9 * i)
        rec *= 2.0 ** (E - 8)
        assert np.abs(rec - vals).max() <= 2.0 ** (E - 46)


def ndigits_pair(s, e, E):
    """The kernel's packed chain (t2_nchain2 after t2_ndigits_pair2): the
    negated digits, u = t 512 + M, -d = M - u, t = fma(t, 512, -d)."""
    M = MAGIC
    hi = np.asarray(s, dtype=np.float32) * F32(2.0 ** (8 - E))
    lo18 = np.asarray(e, dtype=np.float32) * F32(2.0 ** (26 - E))
    u = hi + M
    nd0 = M - u
    t = hi + nd0
    u = t * F32(512) + M
    nd1 = M - u
    t = t * F32(512) + nd1
    u = (t * F32(512) + lo18) + M
    nd2 = M - u
    t = (t * F32(512) + nd2) + lo18
    u = t * F32(512) + M
    nd3 = M - u
    t = t * F32(512) + nd3
    u = t * F32(512) + M
    nd4 = M - u
    t = t * F32(512) + nd4
    u = t * F32(512) + M
    nd5 = M - u
    return np.stack([nd0, nd1, nd2, nd3, nd4, nd5]).astype(np.float64)


def test_negated_digit_chain_is_the_exact_negation():
    """The pass stores -d_i, computed by its own chain; every step is the exact
    negation of the positive chain's (rounding is symmetric and u - M is an
    exact integer), so the digits agree bit for bit up to sign."""
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-12, 1, 5000),
                           [0.0, 1.0, -1.0, 0.5, 2.0 ** -30, 0.999999999, 1e-40]])
    s, e = to_pairs(vals)
    E = pair_row_scale(s)
    assert np.array_equal(ndigits_pair(s, e, E), -digits_pair(s, e, E))


def test_w_digits_reconstruct_within_2_pow_minus_54():
    rng = np.random.default_rng(1)
    for w in list(rng.uniform(-1, 1, 3000)) + [1.0, -1.0, 0.0, 0.5, -0.5, 2 ** -44, 1 - 2 ** -50]:
        g = w_digits(w)
        assert max(abs(x) for x in g) <= 256
        v = sum(Fraction(x) * Fraction(2) ** (-8 - 9 * j) for j, x in enumerate(g))
        assert abs(v - Fraction(w)) <= Fraction(2) ** -54


def test_combine_equals_the_exact_level_sum():
    rng = np.random.default_rng(2)
    for trial in range(3000):
        c = [float(rng.integers(-2 ** 22, 2 ** 22)), float(rng.integers(-2 ** 23, 2 ** 23)),
             float(rng.integers(-3 * 2 ** 22, 3 * 2 ** 22)), float(rng.integers(-2 ** 24, 2 ** 24)),
             float(F32(rng.integers(-2 ** 25, 2 ** 25))), float(F32(rng.integers(-2 ** 25, 2 ** 25)))]
        if trial % 5 == 0:
            c[0] = 0.0
        if trial % 7 == 0:   # just below or above a power of two
            c = [float(2 ** 20), -1.0 * rng.integers(1, 512), float(rng.integers(-2 ** 10, 2 ** 10)), 0.0, 0.0, 0.0]
        if trial % 11 == 0:  # only the low levels
            c = [0.0, 0.0, 0.0, 0.0, float(rng.integers(-2 ** 20, 2 ** 20)), float(rng.integers(-2 ** 20, 2 ** 20))]
        em = int(rng.integers(900, 1100))
        exact = sum(Fraction(x) * Fraction(2) ** (-9 * l) for l, x in enumerate(c)) * Fraction(2) ** (em - 1038)
        got = combine(c, em)
        # relative to the result, or absolute at 2^-34 of a level-0 unit (2^(E-50) for rows scaled 2^E)
        assert abs(Fraction(got) - exact) <= abs(exact) * Fraction(2) ** -46 + Fraction(2) ** (em - 1038 - 34)


def test_pair_digits_reconstruct_every_value_of_a_row():
    rng = np.random.default_rng(3)
    vals = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-12, 1, 4000),
                           [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -30, 0.999999999, 1e-40]])
    s, e = to_pairs(vals)
    E = pair_row_scale(s)
    assert np.all(np.abs(vals) < 2.0 ** E)
    D = digits_pair(s, e, E)
    assert np.abs(D).max() <= 260
    rec = sum(D[i] * 2.0 ** (-9 * i) for i in range(6)) * 2.0 ** (E - 8)
    # the pair holds the value to 2^-48 relative; the digits to 2^(E-46)
    assert np.abs(rec - vals).max() <= 2.0 ** (E - 46) + 2.0 ** -47 * np.abs(vals).max()


@pytest.mark.parametrize("pairs_in,pairs_out", [(False, True), (True, True), (True, False)])
def test_a_whole_row_through_fp32_pairs(pairs_in, pairs_out):
    rng = np.random.default_rng(7)
    for trial in range(3):
        U = haar(32, rng)
        a = (rng.standard_normal(32) + 1j * rng.standard_normal(32)) / 8
        if trial == 2:
            a[::3] = 0
        got, em = apply_row(U, a, pairs_in, pairs_out)
        assert np.abs(got - U @ a).max() <= row_bound(a, em, pairs_in)


@pytest.mark.parametrize("shape", ["random", "one", "mixed", "tiny", "powers", "zeros"])
def test_a_whole_row_matches_the_fp64_product(shape):
    rng = np.random.default_rng(["random", "one", "mixed", "tiny", "powers", "zeros"].index(shape) + 40)
    for trial in range(3):
        U = haar(32, rng)
        a = (rng.standard_normal(32) + 1j * rng.standard_normal(32)) / 8
        if shape == "one":
            a = np.zeros(32, complex)
            a[rng.integers(32)] = 1.0 if trial == 0 else np.exp(1j * rng.uniform(0, 6.3))
        elif shape == "mixed":
            a *= 10.0 ** rng.integers(-15, 1, 32)
        elif shape == "tiny":
            a *= 2.0 ** -900
            a[3] = 5e-324
        elif shape == "powers":
            a = (2.0 ** -rng.integers(1, 12, 32)) * rng.choice([-1, 1], 32) + 1j * 2.0 ** -rng.integers(1, 12, 32)
        elif shape == "zeros":
            a[::2] = 0
            a[5] = -0.0
        got, em = apply_row(U, a)
        want = U @ a
        if np.abs(np.concatenate([a.real, a.imag])).max() == 0:
            assert np.all(got == 0)
            continue
        assert np.abs(got - want).max() <= row_bound(a, em) + 1e-300, (shape, trial)


def _schedule():
    """The kernel's MMA schedule tables (kT2PhaseH, kT2PhaseL), read from its source."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(__file__), "..", "paper_2509_04955_gb300", "csrc",
                            "kernels_tc128.cu")).read()
    out = []
    for name in ("kT2PhaseH", "kT2PhaseL"):
        body = re.search(name + r"\[\] = \{(.*?)\};", src, re.S).group(1)
        out.append([tuple(int(x) for x in m.groups())
                    for m in re.finditer(r"\{\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\s*\}", body)])
    return out


# the levels each phase may write: the previous tile's drainers release levels
# 4-5 first (combined into registers), then levels 0-3 (read for the fold)
PHASE_LEVELS = ({4, 5}, {0, 1, 2, 3, 4, 5})


def test_mma_schedule_issues_every_digit_product_once():
    """Each entry (a, w, nplanes, level, fresh) multiplies A plane a by W planes
    w .. w + nplanes - 1 into levels level .. level + nplanes - 1. Together the
    two phases must issue exactly the 21 products A_i W_j into level i + j,
    i + j <= 5, over the six planes of each operand; phase H only into levels
    4-5 (released first); an entry is `fresh` (its first k-step overwrites)
    exactly when it is the first, in issue order, to write each of its levels,
    and every level has one; N = 64 x nplanes <= 256 (four planes)."""
    phases = _schedule()
    want = {(i, j, i + j) for i in range(6) for j in range(6) if i + j <= 5}
    got, written = [], set()
    for phase, levels in zip(phases, PHASE_LEVELS):
        for a, w, npl, lev, fresh in phase:
            assert 1 <= npl <= 4 and 0 <= a <= 5 and fresh in (0, 1) and w + npl <= 6
            mine = set(range(lev, lev + npl))
            assert mine <= levels
            if fresh:
                assert not (mine & written), "a fresh entry would overwrite an earlier product"
            else:
                assert mine <= written, "an accumulating entry would add to the previous tile's level"
            written |= mine
            got += [(a, w + k, lev + k) for k in range(npl)]
    assert written == {0, 1, 2, 3, 4, 5}
    assert sorted(got) == sorted(want) and len(got) == 21
    assert sum(len(p) for p in phases) == 8


@pytest.mark.parametrize("plant", ["no_a_digit5", "no_w_digit5", "no_level4", "no_level5", "level1_sign",
                                   "w_transposed"])
def test_the_row_bound_catches_a_planted_mistake(plant):
    """The whole-row bound is tight enough to fail when the model drops the
    last digit plane of A or of W or the level-4 or level-5 accumulator, flips the sign
    of a level, or transposes the block (rows read as FP32 pairs, the form
    every pass after the first of a run reads): each slip gives an error
    above the bound, the clean model one well below it."""
    rng = np.random.default_rng(60)
    U = haar(32, rng)
    a = (rng.standard_normal(32) + 1j * rng.standard_normal(32)) / 8
    got, em = apply_row(U, a, pairs_in=True, plant=plant)
    assert np.abs(got - U @ a).max() > 2 * row_bound(a, em, pairs_in=True)
    clean, em = apply_row(U, a, pairs_in=True)
    assert np.abs(clean - U @ a).max() <= 0.5 * row_bound(a, em, pairs_in=True)


def test_level_three_range_holds_for_random_rows():
    """Level 3 sums 4 products; only an adversarial alignment of all digits could reach 2^24."""
    rng = np.random.default_rng(5)
    U = haar(32, rng)
    for _ in range(3):
        a = (rng.standard_normal(32) + 1j * rng.standard_normal(32))
        reals = np.empty(64)
        reals[0::2], reals[1::2] = a.real, a.imag
        D = digits(reals, np.full(64, row_emax(reals))).astype(np.int64)
        Wd = np.array([[w_digits(x) for x in col] for col in
                       np.concatenate([U.real.T, U.imag.T]).reshape(64, 32)]).transpose(2, 0, 1)
        for nn in range(32):
            l3 = sum(int((D[i] * np.resize(Wd[3 - i, :, nn], 64)).sum()) for i in range(4))
            assert abs(l3) < 2 ** 22


# ---------------------------------------------------------------- indexing

def _geometry(n, Q):
    Q = sorted(Q)
    R = [q for q in range(n) if q not in Q][:7]
    T = sorted(Q + R)
    pr = 0
    while pr < 12 and T[pr] == pr:
        pr += 1
    lam = {q: i for i, q in enumerate(T)}
    lamcol = [sum(((c >> b) & 1) << lam[Q[b]] for b in range(5)) for c in range(32)]
    coff = [sum(((c >> b) & 1) << Q[b] for b in range(5)) for c in range(32)]
    return Q, R, T, pr, lam, lamcol, coff


def _tile_base(T, t):
    x = t
    for q in T:
        x = ((x >> q) << (q + 1)) | (x & ((1 << q) - 1))
    return x


PLACEMENTS = [(0, 1, 2, 3, 4), (0, 1, 2, 9, 10), (1, 3, 7, 9, 11), (7, 8, 9, 10, 11), (2, 4, 5, 6, 8),
              (12, 13, 14, 15, 16), (0, 5, 11, 13, 15), (3, 4, 5, 6, 7), (0, 2, 4, 6, 8)]


@pytest.mark.parametrize("Q", PLACEMENTS)
def test_tile_elements_land_and_store_at_their_amplitudes(Q):
    n = 17
    Q, R, T, pr, lam, lamcol, coff = _geometry(n, Q)
    assert pr >= 7
    runoff = [sum(((j >> b) & 1) << T[pr + b] for b in range(12 - pr)) for j in range(1 << (12 - pr))]
    seen = set()
    for t in range(1 << (n - 12)):
        tb = _tile_base(T, t)
        slot = {}
        for j, r in enumerate(runoff):             # run j of 2^pr amplitudes at slot offset j 2^pr
            for o in range(1 << pr):
                slot[j * (1 << pr) + o] = tb + r + o
        assert sorted(slot) == list(range(4096))
        for row in range(128):
            lrow = sum(((row >> b) & 1) << lam[R[b]] for b in range(7))
            roff = sum(((row >> b) & 1) << R[b] for b in range(7))
            for c in range(32):
                g = slot[lrow | lamcol[c]]
                assert g == (tb | roff | coff[c])      # the drainer's store address
                seen.add(g)
    assert len(seen) == 1 << n


def _skew(T, Q, lane):
    """The converters' column skew: kq = row qubits among the three lowest
    tile qubits, sg = lane bits kq .. 2 (the kernel's qpos[25] and sg)."""
    kq = sum(1 for q in T[:3] if q not in Q)
    return kq, (lane >> kq) & ((1 << (3 - kq)) - 1)


@pytest.mark.parametrize("Q", PLACEMENTS + [(20, 22, 25, 27, 29), (5, 6, 7, 8, 9), (0, 1, 2, 3, 29)])
def test_converter_slot_reads_are_bank_conflict_free(Q):
    """Every warp-wide 16-byte read of the landing slot (32 rows, lane l at
    step j taking column j ^ sg(l)) hits each of the 8 bank groups (index
    mod 8) exactly 4 times, for the exponent pass (16 columns) and the digit
    pass (8 columns per chunk); each lane still reads all its columns once,
    and the swap network puts column j into register j."""
    n = 30
    Q, R, T, pr, lam, lamcol, coff = _geometry(n, Q)
    for quad in range(4):
        lrows = [sum((((quad * 32 + l) >> b) & 1) << lam[R[b]] for b in range(7)) for l in range(32)]
        for h in range(2):
            for j in range(16):
                groups = [0] * 8
                for l in range(32):
                    kq, sg = _skew(T, Q, l)
                    groups[(lrows[l] | lamcol[16 * h + (j ^ sg)]) & 7] += 1
                assert groups == [4] * 8, (quad, h, j, groups)
    for l in range(32):
        kq, sg = _skew(T, Q, l)
        assert sorted(j ^ sg for j in range(16)) == list(range(16))
        vv = [j ^ sg for j in range(8)]            # column held after the skewed loads
        for b in range(3 - kq):
            if (sg >> b) & 1:
                for j in range(8):
                    if not j & (1 << b):
                        vv[j], vv[j | (1 << b)] = vv[j | (1 << b)], vv[j]
        assert vv == list(range(8))


# ---------------------------------------------------------------- barriers

class _Bar:
    """mbarrier: `done` completed phases; try_wait.parity(P) passes iff (done & 1) != P."""

    def __init__(self, count):
        self.count, self.pending, self.done, self.tx = count, count, 0, 0

    def arrive(self):
        self.pending -= 1
        self._check()

    def expect_tx(self, b):
        self.tx += b
        self.arrive()

    def complete_tx(self, b):
        self.tx -= b
        self._check()

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.done += 1
            self.pending = self.count

    def ok(self, parity):
        return (self.done & 1) != parity


def _simulate(my, tiles_per_state, t_begin, seed, etab_after_mdone=True, l45_release_early=False):
    rng = random.Random(seed)
    state = lambda i: (t_begin + i) // tiles_per_state
    new_state = lambda i: i > 0 and state(i) != state(i - 1)
    full, empty = [_Bar(1), _Bar(1)], [_Bar(8), _Bar(8)]
    afull, mdone, dfree, dfree45 = _Bar(8), _Bar(1), _Bar(8), _Bar(8)
    efull = [_Bar(8), _Bar(8)]
    xbar = [[_Bar(2) for _ in range(4)] for _ in range(2)]
    wfull, wfree = _Bar(1), _Bar(1)
    events, now, last_finish = [], [0.0], [0.0]
    W = {"state": state(0), "writing": None}
    A = {"tile": None}                   # tile whose digits the A planes hold
    # levels 4-5 and levels 0-3 of the accumulators: tile they hold, and whether
    # the drainers are done with them (combined into registers, resp. read for the fold)
    D45 = {"tile": None, "free": True}
    D03 = {"tile": None, "free": True}
    slot_of = {0: None, 1: None}
    xe = {}                              # (parity, quad, half) -> tile
    etab = {0: None, 1: None}
    inflight, errors = {}, []

    def later(dt, fn):
        events.append((now[0] + dt, fn))

    def producer():
        issued = 0
        for i in range(my):
            s = i & 1
            if i >= 2:
                yield lambda: empty[s].ok(((i >> 1) - 1) & 1)
            full[s].expect_tx(1)

            def land(s=s, i=i):
                slot_of[s] = i
                full[s].complete_tx(1)
            later(rng.uniform(1, 5), land)
            if new_state(i):
                yield lambda: wfree.ok(issued & 1)
                if any(st != state(i) for st in inflight.values()):
                    errors.append("W overwritten under in-flight MMAs")
                W["writing"] = state(i)
                wfull.expect_tx(1)

                def wland(st=state(i)):
                    W["state"], W["writing"] = st, None
                    wfull.complete_tx(1)
                later(rng.uniform(1, 5), wland)
                issued += 1

    def mma():
        seen = 0
        for i in range(my):
            if new_state(i):
                yield lambda: wfull.ok(seen & 1)
                seen += 1
            yield lambda: afull.ok(i & 1)
            if i >= 1:                   # phase H: levels 4-5 first
                yield lambda: dfree45.ok((i - 1) & 1)
            if W["state"] != state(i) or W["writing"] is not None:
                errors.append("MMA reads the wrong W")
            if A["tile"] != i:
                errors.append("MMA reads digits of another tile")
            if not D45["free"]:
                errors.append("levels 4-5 overwritten before they were read")
            D45["tile"], D45["free"] = None, False
            inflight[i] = state(i)
            if i >= 1:                   # phase L: levels 0-3 (and 4-5 again)
                yield lambda: dfree.ok((i - 1) & 1)
            if not D03["free"]:
                errors.append("levels 0-3 overwritten before they were read")
            if A["tile"] != i or W["state"] != state(i):
                errors.append("MMA reads digits of another tile")
            D03["tile"], D03["free"] = None, False

            def finish(i=i, last=(i + 1 < my and new_state(i + 1))):
                del inflight[i]
                D45["tile"] = D03["tile"] = i
                mdone.arrive()
                if last:
                    wfree.arrive()
            last_finish[0] = max(last_finish[0], now[0] + rng.uniform(0.5, 3))
            events.append((last_finish[0], finish))

    def converter(quad, half):
        for i in range(my):
            s, par = i & 1, i & 1
            yield lambda: full[s].ok((i >> 1) & 1)
            if slot_of[s] != i:
                errors.append("converter reads a slot holding another tile")
            yield ("sleep", rng.uniform(0, 0.5))
            xe[(par, quad, half)] = i
            xbar[par][quad].arrive()
            yield lambda: xbar[par][quad].ok((i >> 1) & 1)
            if xe.get((par, quad, half ^ 1)) != i:
                errors.append("row exponent exchanged with another tile")
            if not etab_after_mdone:
                if half == 0:
                    etab[par] = i
                efull[par].arrive()
            if i >= 1:
                yield lambda: mdone.ok((i - 1) & 1)
            if (i - 1) in inflight:
                errors.append("A planes overwritten under an MMA")
            if etab_after_mdone:   # the drainers of tile i - 2 (same parity) read their entry
                if half == 0:
                    etab[par] = i
                efull[par].arrive()
            yield ("sleep", rng.uniform(0, 1))
            A["tile"] = i
            empty[s].arrive()
            afull.arrive()

    def drainer():
        for i in range(my):
            par = i & 1
            yield lambda: mdone.ok(i & 1)
            yield lambda: efull[par].ok((i >> 1) & 1)
            if D45["tile"] != i or D03["tile"] != i:
                errors.append("accumulators read before their MMAs finished")
            if etab[par] != i:
                errors.append("exponent table holds another tile")

            def release45():
                dfree45.arrive()
                if dfree45.pending == dfree45.count:   # the eighth drainer warp: levels 4-5 free
                    D45["free"] = True
            if l45_release_early:
                release45()
            yield ("sleep", rng.uniform(0, 0.5))   # levels 4-5 into registers
            if D45["tile"] != i:
                errors.append("levels 4-5 read after the next tile's MMAs wrote them")
            if not l45_release_early:
                release45()
            yield ("sleep", rng.uniform(0, 1))     # levels 0-3 read chunk by chunk
            if D03["tile"] != i:
                errors.append("levels 0-3 read after the next tile's MMAs wrote them")
            dfree.arrive()
            if dfree.pending == dfree.count:
                D03["free"] = True
            yield ("sleep", rng.uniform(0, 4))   # joins and stores after the release

    roles = [producer(), mma()] + [converter(q, h) for h in range(2) for q in range(4)] + \
            [drainer() for _ in range(8)]
    waiting, sleeping, alive = {}, {}, set(range(len(roles)))
    for _ in range(400000):
        if not alive:
            return errors
        progressed = False
        order = list(alive)
        rng.shuffle(order)
        for j in order:
            if j in sleeping:
                if sleeping[j] > now[0]:
                    continue
                del sleeping[j]
            w = waiting.get(j)
            if w is not None and not w():
                continue
            try:
                nxt = next(roles[j])
                if isinstance(nxt, tuple):
                    sleeping[j], waiting[j] = now[0] + nxt[1], None
                else:
                    waiting[j] = nxt
            except StopIteration:
                alive.discard(j)
            progressed = True
        if not progressed:
            if not events and not sleeping:
                return errors + ["deadlock"]
            now[0] = max(now[0], min([e[0] for e in events] + list(sleeping.values())))
            for e in [e for e in events if e[0] <= now[0]]:
                events.remove(e)
                e[1]()
    return errors + ["no progress"]


def test_barrier_protocol_has_no_hazard_or_deadlock():
    for seed in range(300):
        r = random.Random(seed * 11 + 5)
        tps = r.choice([1, 2, 3, 4, 8, 1 << 20])
        my = r.choice([1, 2, 3, 4, 5, 7, 20, 54])
        tb = r.randrange(0, 4 * min(tps, 8))
        assert _simulate(my, tps, tb, seed) == [], (seed, tps, my, tb)


def test_exponent_table_written_before_the_mdone_wait_is_caught_by_the_model():
    """Writing tile i's row exponents before waiting for tile i - 1's MMAs lets
    them overwrite tile i - 2's entry while its drainers are still storing."""
    fails = sum(1 for seed in range(200) if _simulate(20, 1 << 20, 0, seed, etab_after_mdone=False))
    assert fails > 20


def test_levels_four_five_released_before_they_are_read_is_caught_by_the_model():
    """Releasing levels 4-5 to the next tile's MMAs before the drainers have
    read them into registers lets those MMAs overwrite them mid-read."""
    fails = sum(1 for seed in range(200) if _simulate(20, 1 << 20, 0, seed, l45_release_early=True))
    assert fails > 20
