"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, through properties that hold at any size or on outputs the
oracle computes one by one:

* the 30-qubit random circuit (complex64, tensor-core plan) followed by its
  inverse returns |0..0>, and the norm stays 1;
* the 32-qubit CZ circuit (32 GiB complex64) on tensor cores: circuit x
  inverse = identity;
* complex128 on the tensor-core plan (the benchmark's headline
  configuration): the 30-qubit circuit and the 32-qubit CZ circuit (64 GiB)
  times their inverses = identity, bar derived from the per-pass bound of the
  digit products; QFT n = 30 on 2^16 sampled amplitudes against the closed
  form.
Round-trip bar: each tensor-core block application perturbs the state by a
relative error e per pass: bf16x3 split products keep about 16 significant
bits (e = 2^-16: hi and lo of 8 bits each, the dropped lo*lo term 2^-16);
the fp16 split (precision 4) keeps 22 (hi and lo of 11 bits, lo*lo 2^-22,
so e = 2^-21 with a factor 2 for the sum of the terms). Over B applications
these add like a random walk, so the test requires
||psi - |0..0>||_2 <= 4 sqrt(B) e (and the same for max |delta amp|, which
after a round trip sits on the amplitude of size 1, unlike the forward
results checked against 2e-5 elsewhere);
* the batched UCC workload (20 qubits, 400 terms, 64 parameter vectors, one
  CUDA graph): sampled states' <H> against the oracle;
* QAOA at 30 qubits (8 GiB complex64, 16 GiB complex128): depth 1 gives the
  expected cut of the published p = 1 closed form (pinned against the oracle
  on small graphs); depth 4 times its inverse returns |0..0>.
"""
import numpy as np
import pytest

import oracle as O
import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


EPS = {3: 2.0 ** -16, 4: 2.0 ** -21}


def roundtrip(n, gates, opts, dt=Q.QS_C64):
    inv = W.inverse_circuit(gates)
    h = Q.qs_state_alloc(n, dt)
    try:
        p1 = Q.qs_plan_create(n, dt, gates, opts)
        p2 = Q.qs_plan_create(n, dt, inv, opts)
        nblocks = sum(1 for p in (p1, p2) for op in Q.qs_plan_ops(p) if op["type"] == 3)
        try:
            Q.qs_plan_execute(p1, h)
            norm_mid = Q.qs_norm(h)
            Q.qs_plan_execute(p2, h)
            norm_end = Q.qs_norm(h)
        finally:
            Q.qs_plan_free(p1)
            Q.qs_plan_free(p2)
        z = Q.qs_state_alloc(n, dt)
        try:
            Q.qs_state_set_basis(z, 0)
            max_abs, l2 = Q.qs_state_diff(h, z)
        finally:
            Q.qs_state_free(z)
    finally:
        Q.qs_state_free(h)
    if dt == Q.QS_C128:
        # per pass and output at most (2^-46 + 2^-48) of the row's 2-norm, so
        # ||delta||_2 <= sqrt(32) (2^-46 + 2^-48) per pass, added up linearly
        return norm_mid, norm_end, max_abs, l2, nblocks * np.sqrt(32) * (2.0 ** -46 + 2.0 ** -48)
    return norm_mid, norm_end, max_abs, l2, 4.0 * np.sqrt(max(1, nblocks)) * EPS[opts.tc_precision or 4]


@pytest.mark.parametrize("tc_min,prec", [(2, 4), (6, 4), (2, 3)])
def test_n30_random_circuit_tensor_plan_times_inverse(tc_min, prec):
    n = 30
    gates = W.random_layered(n, 20, seed=0)
    mid, end, max_abs, l2, bar = roundtrip(n, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=tc_min,
                                                                  tc_precision=prec))
    assert abs(mid - 1) < 1e-4 and abs(end - 1) < 1e-4
    assert max_abs <= bar and l2 <= bar, (max_abs, l2, bar)


@pytest.mark.parametrize("prec", [4, 3])
def test_n32_cz_circuit_tensor_plan_times_inverse(prec):
    n = 32
    gates = W.random_layered(n, 40, seed=0, entangler="cz")
    mid, end, max_abs, l2, bar = roundtrip(n, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2,
                                                                  tc_precision=prec))
    assert abs(mid - 1) < 1e-4 and abs(end - 1) < 1e-4
    assert max_abs <= bar and l2 <= bar, (max_abs, l2, bar)


@pytest.mark.parametrize("n,depth,ent", [(30, 20, "cnot"), (32, 40, "cz")])
def test_c128_tensor_plan_times_inverse_at_full_size(n, depth, ent):
    """Complex128 on the default tensor-core plan, the launch configuration
    of the benchmark: the 30-qubit headline circuit (16 GiB) and the 32-qubit
    CZ circuit (64 GiB), each followed by its inverse, return |0..0>. Bar: the
    derived worst case of the digit-product passes for the l2 error, and the
    complex128 bar 1e-12 for every amplitude."""
    gates = W.random_layered(n, depth, seed=0, entangler=ent)
    mid, end, max_abs, l2, bar = roundtrip(n, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR), Q.QS_C128)
    assert abs(mid - 1) < 1e-12 and abs(end - 1) < 1e-12
    assert l2 <= bar and max_abs <= min(bar, 1e-12), (max_abs, l2, bar)


def test_c128_tensor_plan_qft_n30_sampled_closed_form():
    """QFT on 30 qubits (16 GiB complex128) on the tensor-core plan from a
    seeded basis state: 2^16 sampled amplitudes, gathered on the device,
    against the closed form 2^-15 e^(2 pi i x y / 2^30), bar 1e-12."""
    n = 30
    x = W.random_basis_index(n, 30)
    rng = np.random.default_rng(3)
    idx = np.unique(rng.integers(0, 1 << n, size=1 << 16).astype(np.uint64))
    h = Q.qs_state_alloc(n, Q.QS_C128)
    try:
        Q.qs_state_set_basis(h, x)
        Q.qs_apply_circuit(h, W.qft(n), None, Q.make_opts(mode=Q.QS_MODE_TENSOR))
        got = Q.qs_state_get_amplitudes(h, idx, Q.QS_C128)
        assert abs(Q.qs_norm(h) - 1) < 1e-12
    finally:
        Q.qs_state_free(h)
    y = idx.astype(object)
    ph = np.array([float((x * int(v)) % (1 << n)) for v in y]) / (1 << n)
    want = np.exp(2j * np.pi * ph) / 2.0 ** (n / 2)
    assert np.abs(got - want).max() <= 1e-12


@pytest.mark.parametrize("dtname,mode", [("c64", Q.QS_MODE_FUSED), ("c64", Q.QS_MODE_TENSOR),
                                         ("c128", Q.QS_MODE_FUSED)])
def test_qaoa_n30_p1_expected_cut_closed_form(dtname, mode):
    from closed_forms import qaoa_p1_maxcut
    dt = {"c64": Q.QS_C64, "c128": Q.QS_C128}[dtname]
    n = 30
    edges = W.random_regular_graph(n, 3, seed=0)
    gates, p = W.qaoa(n, 1, edges)
    H = W.maxcut_hamiltonian(edges)
    th = np.array([0.37, -0.81])
    opts = Q.make_opts(mode=mode, tc_min_gates=4, fuse_parametric=1)
    plan = Q.qs_plan_create(n, dt, gates, opts)
    h = Q.qs_state_alloc(n, dt)
    try:
        assert sum(op["type"] == 4 for op in Q.qs_plan_ops(plan)) == 1
        Q.qs_plan_execute(plan, h, th)
        e = Q.qs_expval_pauli_sum(h, *H)
        assert abs(Q.qs_norm(h) - 1) < (1e-12 if dt == Q.QS_C128 else 1e-5)
        bar = (1e-10 if dt == Q.QS_C128 else 2e-5) * np.abs(H[0]).sum()
        assert abs(e - qaoa_p1_maxcut(n, edges, *th)) <= bar, (e, qaoa_p1_maxcut(n, edges, *th))
    finally:
        Q.qs_state_free(h)
        Q.qs_plan_free(plan)


def test_qaoa_n30_p4_times_inverse():
    n = 30
    edges = W.random_regular_graph(n, 3, seed=0)
    gates, p = W.qaoa(n, 4, edges)
    th = W.thetas_uniform(p, 1)
    fixed = W.inverse_circuit(W.inverse_circuit(gates, th))     # the same circuit with resolved angles
    mid, end, max_abs, l2, bar = roundtrip(n, fixed, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4))
    assert abs(mid - 1) < 1e-4 and abs(end - 1) < 1e-4
    # phase passes and tile passes are FP32 products: about 1e-6 per pass
    assert max_abs <= 2e-4 and l2 <= 2e-4, (max_abs, l2)


def test_ucc_batched_n20_b64_sampled_against_oracle():
    n, Bsz = 20, 64
    gates, _ = W.ucc(n, 400, seed=0)
    th = W.thetas_normal(400, 1, sigma=0.1, batch=Bsz)
    H = W.random_pauli_sum(n, 300, seed=3)
    psi17 = O.apply_circuit(O.basis(n, 0), n, gates, th[17])
    want = O.expval(psi17, n, *H).real
    for opts in (Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1), Q.make_opts(fuse_k=1)):
        plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
        try:
            for rep_ in range(2):        # capture, then graph replay
                for s in states:
                    Q.qs_state_set_basis(s, 0)
                ex = Q.qs_plan_execute_batched(plan, states, th, H)
            # the state of row 17 element by element (complex64 bar), and <H> against the
            # oracle to 1e-5 of the coefficient sum (about 1 % of the value here)
            out = np.empty(1 << n, dtype=np.complex64)
            Q.qs_state_copy_to_host(states[17], out)
            assert np.abs(out - psi17).max() <= 2e-5
            assert abs(ex[17] - want) <= 1e-5 * np.abs(H[0]).sum()
            assert np.all(np.isfinite(ex))
        finally:
            for s in states:
                Q.qs_state_free(s)
            Q.qs_plan_free(plan)
