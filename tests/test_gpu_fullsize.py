"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, through properties that hold at any size or on outputs the
oracle computes one by one:

* the 30-qubit random circuit (complex64, tensor-core plan) followed by its
  inverse returns |0..0>, and the norm stays 1;
* the 32-qubit CZ circuit (32 GiB complex64) on tensor cores: circuit x
  inverse = identity.
Round-trip bar: each tensor-core block application (bf16x3 split products,
FP32 accumulation) perturbs the state by a relative error of about 2^-16;
over B applications these add like a random walk, so the test requires
||psi - |0..0>||_2 <= 4 sqrt(B) 2^-16 (and the same for max |delta amp|,
which after a round trip sits on the amplitude of size 1, unlike the forward
results checked against 2e-5 elsewhere);
* the batched UCC workload (20 qubits, 400 terms, 64 parameter vectors, one
  CUDA graph): sampled states' <H> against the oracle.
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


def roundtrip(n, gates, opts):
    inv = W.inverse_circuit(gates)
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        p1 = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        p2 = Q.qs_plan_create(n, Q.QS_C64, inv, opts)
        nblocks = sum(1 for p in (p1, p2) for op in Q.qs_plan_ops(p) if op["type"] == 3)
        try:
            Q.qs_plan_execute(p1, h)
            norm_mid = Q.qs_norm(h)
            Q.qs_plan_execute(p2, h)
            norm_end = Q.qs_norm(h)
        finally:
            Q.qs_plan_free(p1)
            Q.qs_plan_free(p2)
        z = Q.qs_state_alloc(n, Q.QS_C64)
        try:
            Q.qs_state_set_basis(z, 0)
            max_abs, l2 = Q.qs_state_diff(h, z)
        finally:
            Q.qs_state_free(z)
    finally:
        Q.qs_state_free(h)
    return norm_mid, norm_end, max_abs, l2, 4.0 * np.sqrt(max(1, nblocks)) * 2.0 ** -16


@pytest.mark.parametrize("tc_min", [2, 6])
def test_n30_random_circuit_tensor_plan_times_inverse(tc_min):
    n = 30
    gates = W.random_layered(n, 20, seed=0)
    mid, end, max_abs, l2, bar = roundtrip(n, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=tc_min))
    assert abs(mid - 1) < 1e-4 and abs(end - 1) < 1e-4
    assert max_abs <= bar and l2 <= bar, (max_abs, l2, bar)


def test_n32_cz_circuit_tensor_plan_times_inverse():
    n = 32
    gates = W.random_layered(n, 40, seed=0, entangler="cz")
    mid, end, max_abs, l2, bar = roundtrip(n, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2))
    assert abs(mid - 1) < 1e-4 and abs(end - 1) < 1e-4
    assert max_abs <= bar and l2 <= bar, (max_abs, l2, bar)


def test_ucc_batched_n20_b64_sampled_against_oracle():
    n, Bsz = 20, 64
    gates, _ = W.ucc(n, 400, seed=0)
    th = W.thetas_normal(400, 1, sigma=0.1, batch=Bsz)
    H = W.random_pauli_sum(n, 300, seed=3)
    want = O.expval_of_circuit(O.basis(n, 0), n, gates, th[17], *H)
    for opts in (Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1), Q.make_opts(fuse_k=1)):
        plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
        try:
            ex = Q.qs_plan_execute_batched(plan, states, th, H)
            assert abs(ex[17] - want) <= 2e-5 * np.abs(H[0]).sum()
            assert np.all(np.isfinite(ex))
        finally:
            for s in states:
                Q.qs_state_free(s)
            Q.qs_plan_free(plan)
