"""GPU parity of the complex128 tensor-core pass (k_tc128) and the bounded-wait
timeout path of both tensor-core passes, through the C ABI against the FP64
oracle.

Bar: complex128 max |delta amp| <= 1e-12 element by element (a pass adds at
most 2^-46 of a 32-amplitude row's 2-norm plus 2^-49 of its scale to each
output, 2^-48 of the norm between passes that hand over FP32 pairs, so the bar
leaves a wide margin at these depths).
"""
import numpy as np
import pytest

import oracle as O
import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
TENSOR = Q.make_opts(mode=Q.QS_MODE_TENSOR)


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    import torch
    assert torch.cuda.is_available()


def execute(plan, n, dt, psi0=None, theta=None, basis=0):
    h = Q.qs_state_alloc(n, dt)
    try:
        if psi0 is not None:
            Q.qs_state_copy_from_host(h, np.ascontiguousarray(psi0, dtype=Q.NP_DTYPE[dt]))
        else:
            Q.qs_state_set_basis(h, basis)
        Q.qs_plan_execute(plan, h, theta)
        out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
        Q.qs_state_copy_to_host(h, out)
        return out
    finally:
        Q.qs_state_free(h)


def tc_ops(plan):
    return [op for op in Q.qs_plan_ops(plan) if op["type"] == 3]


# 5-qubit placements: all, some or none of the block qubits among qubits 0-6
# (the lowest qubits, which hold the tile rows when the block avoids them),
# blocks spread out, and blocks above every row qubit.
BLOCK_SETS5 = [(0, 1, 2, 3, 4), (0, 1, 2, 9, 10), (1, 3, 7, 9, 11), (0, 7, 8, 9, 10), (7, 8, 9, 10, 11),
               (2, 4, 5, 6, 8), (0, 2, 4, 6, 8), (3, 4, 5, 6, 7)]


@pytest.mark.parametrize("n", [12, 13, 16])
def test_c128_tensor_core_every_block_placement(n):
    """Dense 5-qubit blocks on the placements above (and on the five highest
    qubits) applied to a random state: every amplitude against the oracle."""
    sets = list(BLOCK_SETS5) + ([tuple(range(n - 5, n))] if n > 12 else [])
    gates = W.block_circuit(sets, 10, seed=n)
    psi0 = W.random_state(n, 5)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=5))
    try:
        placed = [tuple(sorted(op["qubits"])) for op in tc_ops(plan)]
        assert len(placed) == len(sets)
        # the contraction may regroup overlapping sets, but the placements keep
        # 5, 3, 2, 1 and 0 block qubits below qubit 7
        assert {5, 3, 2, 1, 0} <= {sum(q < 7 for q in qs) for qs in placed}
        out = execute(plan, n, Q.QS_C128, psi0=psi0)
    finally:
        Q.qs_plan_free(plan)
    assert np.abs(out - O.apply_circuit(psi0, n, gates)).max() <= TOL


@pytest.mark.parametrize("n,depth", [(12, 10), (14, 20), (18, 12), (21, 8), (22, 6)])
def test_c128_tensor_core_random_layers_many_tiles(n, depth):
    """The layered random circuit on tensor-core plans; from n = 21 a CTA walks
    several tiles (2^(n-12) tiles over at most one CTA per SM), with both
    landing slots and the single-buffered operand and accumulator hand-offs in
    use. Every amplitude against the oracle."""
    gates = W.random_layered(n, depth, seed=n + 100)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, TENSOR)
    try:
        assert tc_ops(plan)
        out = execute(plan, n, Q.QS_C128)
    finally:
        Q.qs_plan_free(plan)
    assert np.abs(out - O.apply_circuit(O.basis(n, 0), n, gates)).max() <= TOL


def test_c128_tensor_core_qft_closed_form_and_oracle():
    """QFT n = 16 on a basis state: amplitudes 2^-8 e^(2 pi i x y / 2^16)."""
    n = 16
    x = W.random_basis_index(n, 7)
    gates = W.qft(n)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, TENSOR)
    try:
        out = execute(plan, n, Q.QS_C128, basis=x)
    finally:
        Q.qs_plan_free(plan)
    y = np.arange(1 << n)
    closed = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    assert np.abs(out - closed).max() <= TOL
    assert np.abs(out - O.apply_circuit(O.basis(n, x), n, gates)).max() <= TOL


def test_c128_tensor_core_with_phase_passes_and_tile_passes():
    """QAOA (phase runs as their own passes) and tensor-core thresholds that
    leave some blocks to CUDA-core tile passes, in FP32 pairs (the default)
    and in FP64."""
    n = 14
    qg, p = W.qaoa(n, 2, W.random_regular_graph(n, 3, seed=1))
    th = W.thetas_uniform(p, 3)
    want = O.apply_circuit(O.basis(n, 0), n, qg, th)
    for tmin, pairs in ((1, 0), (4, 2), (4, 1)):
        plan = Q.qs_plan_create(n, Q.QS_C128, qg, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=tmin,
                                                               c128_pairs=pairs))
        try:
            assert tc_ops(plan)
            out = execute(plan, n, Q.QS_C128, theta=th)
        finally:
            Q.qs_plan_free(plan)
        assert np.abs(out - want).max() <= TOL, (tmin, pairs)


def test_c128_tensor_core_basis_states_keep_full_precision():
    """States with one amplitude near 1 (the largest row scale): a short
    circuit from every basis index of a small register stays at the bar."""
    n = 12
    gates = W.block_circuit([(0, 1, 2, 3, 4), (3, 5, 7, 9, 11), (6, 7, 8, 10, 11)], 8, seed=2)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, TENSOR)
    try:
        for x in (0, 1, 2 ** 11 + 5, 2 ** 12 - 1):
            out = execute(plan, n, Q.QS_C128, basis=x)
            assert np.abs(out - O.apply_circuit(O.basis(n, x), n, gates)).max() <= TOL, x
    finally:
        Q.qs_plan_free(plan)


@pytest.mark.parametrize("n,Bsz", [(13, 7), (14, 77)])
def test_c128_tensor_core_batched_with_device_built_digit_planes(n, Bsz):
    """Batched complex128 tensor-core passes: blocks holding parametric gates
    are rebuilt from each row's theta on the device as digit planes (checked
    against the host's FP64 products), per-state W planes reloaded when a
    CTA's tile range crosses a state; rows against the oracle after a graph
    capture and a replay."""
    nterms = 8
    gates, _ = W.ucc(n, nterms, seed=n)
    thetas = W.thetas_normal(nterms, 20 + n, sigma=0.5, batch=Bsz)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, fuse_parametric=1))
    states = [Q.qs_state_alloc(n, Q.QS_C128) for _ in range(Bsz)]
    try:
        assert tc_ops(plan)
        diff, nblk = Q.qs_plan_check_device_blocks(plan, states[0], thetas[0])
        assert nblk >= 1 and diff <= 1e-15
        for _ in range(2):               # capture, then graph replay
            for s in states:
                Q.qs_state_set_basis(s, 0)
            Q.qs_plan_execute_batched(plan, states, thetas)
        for b in sorted({0, 1, Bsz // 2, Bsz - 1}):
            out = np.empty(1 << n, dtype=np.complex128)
            Q.qs_state_copy_to_host(states[b], out)
            assert np.abs(out - O.apply_circuit(O.basis(n, 0), n, gates, thetas[b])).max() <= TOL, b
    finally:
        for s in states:
            Q.qs_state_free(s)
        Q.qs_plan_free(plan)


def test_c128_adjoint_gradient_with_a_tensor_core_forward_plan():
    """The adjoint gradient with a complex128 tensor-core forward plan: <H>
    and every gradient entry against the oracle's adjoint."""
    n = 12
    gates, p = W.hea(n, 2)
    th = W.thetas_uniform(p, 11)
    coeff, xm, zm = W.random_pauli_sum(n, 20, seed=12)
    h = Q.qs_state_alloc(n, Q.QS_C128)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, th, coeff, xm, zm, opts=TENSOR)
    finally:
        Q.qs_state_free(h)
    e_ref, g_ref = O.adjoint_grad(O.basis(n, 0), n, gates, th, coeff, xm, zm)
    bar = TOL * float(np.abs(coeff).sum())
    assert abs(e - e_ref) <= bar
    assert np.abs(g - g_ref).max() <= bar


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_tensor_core_wait_timeout_returns_error_and_recovers(dtname):
    """Failure detection: with a wait limit of 2 immediate polls the pipeline
    waits run out (the first accumulator is minutes of polls away, not two);
    the pass stops, lets its copies and MMAs land, frees its tensor memory and
    the execution returns QS_ERR_TIMEOUT. The same plan with the default
    limit then runs normally in the same process and matches the oracle."""
    dt = Q.QS_C64 if dtname == "c64" else Q.QS_C128
    n = 16
    gates = W.random_layered(n, 6, seed=31)
    opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2 if dt == Q.QS_C64 else 0)
    plan = Q.qs_plan_create(n, dt, gates, opts)
    try:
        assert tc_ops(plan)
        Q.qs_plan_set_wait_limit(plan, 2)
        with pytest.raises(Q.QsError) as e:
            execute(plan, n, dt)
        assert e.value.status == Q.QS_ERR_TIMEOUT
        Q.qs_plan_set_wait_limit(plan, 0)
        out = execute(plan, n, dt)
    finally:
        Q.qs_plan_free(plan)
    tol = 1e-12 if dt == Q.QS_C128 else 2e-5
    assert np.abs(out - O.apply_circuit(O.basis(n, 0), n, gates)).max() <= tol
