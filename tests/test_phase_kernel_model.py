"""CPU model of the diagonal phase pass's arithmetic (kernels_phase.cu).

The kernel splits the index into lo = bits 0..11 and hi, forms per-CTA and
per-chunk factor tables and reads them with per-lane index arithmetic that
differs between complex64 (a lane holds amplitudes 2f, 2f + 1 of float4 f =
lane + 32 i) and complex128 (a lane holds amplitude lane + 32 i). This model
replays exactly those steps in numpy, on the terms a real plan hands the
kernel (class order from qs_plan_phase_terms), and checks the product against
the phase polynomial evaluated directly. It runs without a GPU.
"""
import numpy as np
import pytest

import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

LBITS = 12
LOW = (1 << LBITS) - 1


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def parity(v):
    return bin(int(v)).count("1") & 1


def classes(masks):
    """Class boundaries as the kernel reads them: LOW, LIN per bit, HIGH, MIXED."""
    def cls(m):
        k = bin(m & LOW).count("1")
        if k == 0:
            return LBITS + 1
        if k == 1:
            return 1 + (m & LOW).bit_length() - 1
        return LBITS + 2 if m & ~LOW else 0
    c = [cls(m) for m in masks]
    assert c == sorted(c), "terms must arrive in class order"
    nlow = sum(1 for v in c if v == 0)
    lin_off = [sum(1 for v in c if v < 1 + u) for u in range(LBITS + 1)]
    high_begin = sum(1 for v in c if v <= LBITS)
    mixed_begin = sum(1 for v in c if v <= LBITS + 1)
    assert lin_off[0] == nlow and lin_off[LBITS] == high_begin
    return nlow, lin_off, high_begin, mixed_begin


def kernel_model(n, terms, theta, c128):
    masks = [t[0] for t in terms]
    alpha = [a0 + (cf * theta[pi] if pi >= 0 else 0.0) for _, pi, a0, cf in terms]
    z = np.exp(1j * np.array(alpha))
    nlow, lin_off, high_begin, mixed_begin = classes(masks)
    cj = lambda v, f: np.conj(v) if f else v   # noqa: E731
    E = np.ones(1 << LBITS, dtype=complex)
    for lo in range(1 << LBITS):
        for j in range(nlow):
            E[lo] *= cj(z[j], parity(masks[j] & lo))
    out = np.empty(1 << n, dtype=complex)
    for ch in range(1 << (n - LBITS)):
        base = ch << LBITS
        cst = np.prod([cj(z[j], parity(masks[j] & base)) for j in range(high_begin, mixed_begin)] or [1.0])
        w = [np.prod([cj(z[j], parity(masks[j] & base)) for j in range(lin_off[u], lin_off[u + 1])] or [1.0])
             for u in range(LBITS)]
        ab = np.empty(128, dtype=complex)
        for e in range(64):
            a, b = cst, 1.0
            for u in range(6):
                a *= cj(w[u], (e >> u) & 1)
                b *= cj(w[6 + u], (e >> u) & 1)
            ab[e], ab[64 + e] = a, b
        mx = [cj(z[j], parity(masks[j] & base)) for j in range(mixed_begin, len(masks))]
        for lane in range(32):
            if not c128:
                a01 = (ab[2 * lane], ab[2 * lane + 1])
                for i in range(64):
                    for bb in range(2):
                        lo = 2 * (lane + 32 * i) + bb
                        f = E[lo] * ab[64 + i] * a01[bb]
                        for j, m in enumerate(mx):
                            f *= cj(m, parity(masks[mixed_begin + j] & lo))
                        out[base + lo] = f
            else:
                for i in range(128):
                    lo = lane + 32 * i
                    f = E[lo] * ab[64 + (i >> 1)] * (ab[lane + 32] if i & 1 else ab[lane])
                    for j, m in enumerate(mx):
                        f *= cj(m, parity(masks[mixed_begin + j] & lo))
                    out[base + lo] = f
    return out


def direct(n, terms, theta):
    x = np.arange(1 << n, dtype=np.int64)
    ang = np.zeros(1 << n)
    for mask, pi, a0, cf in terms:
        a = a0 + (cf * theta[pi] if pi >= 0 else 0.0)
        par = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            if (mask >> q) & 1:
                par ^= (x >> q) & 1
        ang += a * (1 - 2 * par)
    return np.exp(1j * ang)


@pytest.mark.parametrize("c128", [False, True])
def test_phase_kernel_decomposition_equals_the_phase_polynomial(c128):
    n = 13
    gates, p = W.phase_run_circuit(n, 2, 40, seed=11)
    theta = W.thetas_uniform(max(p, 1), 12)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts())
    try:
        runs = [op for op in Q.qs_plan_ops(plan) if op["type"] == 4]
    finally:
        Q.qs_plan_free(plan)
    assert runs
    seen = set()
    for op in runs:
        terms = op["terms"]
        nlow, lin_off, high_begin, mixed_begin = classes([t[0] for t in terms])
        seen |= {k for k, v in (("low", nlow), ("lin", high_begin - nlow), ("high", mixed_begin - high_begin),
                                ("mixed", len(terms) - mixed_begin)) if v}
        got = kernel_model(n, terms, theta, c128)
        assert np.abs(got - direct(n, terms, theta)).max() < 1e-12
    assert seen == {"low", "lin", "high", "mixed"}
