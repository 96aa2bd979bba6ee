"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (written into every comparison): complex128 max |delta amp| <= 1e-12,
complex64 max |delta amp| <= 2e-5; expectation values and gradients to the
same absolute bars scaled by the Hamiltonian's coefficient sum.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {Q.QS_C128: 1e-12, Q.QS_C64: 2e-5}
DT = {"c128": Q.QS_C128, "c64": Q.QS_C64}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    import torch
    assert torch.cuda.is_available()


def run(n, dt, gates, theta=None, psi0=None, opts=None, basis=0):
    h = Q.qs_state_alloc(n, dt)
    try:
        if psi0 is not None:
            Q.qs_state_copy_from_host(h, np.ascontiguousarray(psi0, dtype=Q.NP_DTYPE[dt]))
        else:
            Q.qs_state_set_basis(h, basis)
        Q.qs_apply_circuit(h, gates, theta, opts)
        out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
        Q.qs_state_copy_to_host(h, out)
        return out
    finally:
        Q.qs_state_free(h)


def ref(n, gates, theta=None, psi0=None, basis=0):
    psi = O.basis(n, basis) if psi0 is None else np.asarray(psi0, dtype=np.complex128)
    return O.apply_circuit(psi, n, gates, theta)


FUSED = [None, Q.make_opts(fuse_k=1, tile_qubits=6, low_qubits=2), Q.make_opts(fuse_k=2, tile_qubits=8, low_qubits=3),
         Q.make_opts(fuse_k=3), Q.make_opts(fuse_k=4, tile_qubits=10, low_qubits=4),
         Q.make_opts(fuse_k=5, tile_qubits=11, low_qubits=3), Q.make_opts(paper_mode=1)]


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_random_depth20_n12_per_gate_matches_oracle(dtname):
    """n = 12 from |0..0>, depth-20 random layers with CNOT matchings, per-gate."""
    dt = DT[dtname]
    n = 12
    gates = W.random_layered(n, 20, seed=0)
    got = run(n, dt, gates)
    want = ref(n, gates)
    assert np.abs(got - want).max() <= TOL[dt]


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("oi", range(len(FUSED)))
def test_every_gate_kind_every_mode(dtname, oi):
    dt = DT[dtname]
    n = 9
    gates = W.random_gate_mix(n, 120, seed=7 + oi) + W.random_layered(n, 3, seed=oi)
    psi0 = W.random_state(n, 3)
    got = run(n, dt, gates, psi0=psi0, opts=FUSED[oi])
    assert np.abs(got - ref(n, gates, psi0=psi0)).max() <= TOL[dt]


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_tiny_states_ragged_tiles(dtname, n):
    dt = DT[dtname]
    gates = W.random_gate_mix(n, 40, seed=n)
    psi0 = W.random_state(n, n)
    for opts in (None, Q.make_opts(fuse_k=2), Q.make_opts(fuse_k=min(n, 5), tile_qubits=n, low_qubits=n)):
        got = run(n, dt, gates, psi0=psi0, opts=opts)
        assert np.abs(got - ref(n, gates, psi0=psi0)).max() <= TOL[dt]


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_fused_random_n18_spans_many_tiles(dtname):
    dt = DT[dtname]
    n = 18
    gates = W.random_layered(n, 6, seed=4)
    want = ref(n, gates)
    for opts in (Q.make_opts(fuse_k=4), Q.make_opts(fuse_k=2, tile_qubits=9, low_qubits=5),
                 Q.make_opts(fuse_k=3, tile_qubits=13, low_qubits=2)):
        got = run(n, dt, gates, opts=opts)
        assert np.abs(got - want).max() <= TOL[dt]


@pytest.mark.parametrize("n", [2, 7, 13])
def test_ghz_closed_form(n):
    gates = [W.Gate("h", (0,))] + [W.Gate("x", (q,), controls=(q - 1,)) for q in range(1, n)]
    for opts in (None, Q.make_opts(fuse_k=3)):
        got = run(n, Q.QS_C128, gates, opts=opts)
        want = np.zeros(1 << n, dtype=complex)
        want[0] = want[-1] = 1 / math.sqrt(2)
        assert np.abs(got - want).max() <= 1e-12


def qft_closed_form(n, x, idx):
    return np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)


def test_qft_n14_all_modes_vs_oracle_and_closed_form():
    n = 14
    x = W.random_basis_index(n, 1)
    gates = W.qft(n)
    want = ref(n, gates, basis=x)
    y = np.arange(1 << n)
    assert np.abs(want - qft_closed_form(n, x, y)).max() < 1e-12
    for opts in (None, Q.make_opts(fuse_k=2), Q.make_opts(fuse_k=4), Q.make_opts(fuse_k=5)):
        got = run(n, Q.QS_C128, gates, opts=opts, basis=x)
        assert np.abs(got - want).max() <= 1e-12


def test_qft_n28_c128_full_size_sampled_closed_form():
    """QFT on 28 qubits (4 GiB complex128) from a seeded basis state; the
    closed form gives every amplitude, checked on 2^16 sampled indices, and
    the norm is checked on the device in FP64."""
    n = 28
    x = W.random_basis_index(n, 28)
    gates = W.qft(n)
    rng = np.random.default_rng(0)
    idx = np.unique(rng.integers(0, 1 << n, size=1 << 16))
    for opts in (Q.make_opts(fuse_k=4), None, Q.make_opts(fuse_k=2, c128_pairs=2)):
        h = Q.qs_state_alloc(n, Q.QS_C128)
        try:
            Q.qs_state_set_basis(h, x)
            Q.qs_apply_circuit(h, gates, None, opts)
            out = np.empty(1 << n, dtype=np.complex128)
            Q.qs_state_copy_to_host(h, out)
            assert abs(Q.qs_norm(h) - 1) < 1e-12
        finally:
            Q.qs_state_free(h)
        assert np.abs(out[idx] - qft_closed_form(n, x, idx)).max() <= 1e-12
        assert np.abs(np.abs(out) - 2.0 ** (-n / 2)).max() <= 1e-12


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_norm_expval_pauli_apply_inner(dtname):
    dt = DT[dtname]
    n = 12
    psi = W.random_state(n, 5)
    coeff, xm, zm = W.random_pauli_sum(n, 40, seed=2)
    # add a few diagonal and repeated-x strings
    coeff = np.concatenate([coeff, [0.7, -0.3, 1.1]])
    xm = np.concatenate([xm, np.array([0, 0, xm[0]], dtype=np.uint64)])
    zm = np.concatenate([zm, np.array([5, 3, 9], dtype=np.uint64)])
    h = Q.qs_state_alloc(n, dt)
    h2 = Q.qs_state_alloc(n, dt)
    try:
        Q.qs_state_copy_from_host(h, psi.astype(Q.NP_DTYPE[dt]))
        psi_dev = psi.astype(Q.NP_DTYPE[dt]).astype(np.complex128)   # what the device holds
        tol = TOL[dt]
        assert abs(Q.qs_norm(h) - O.norm2(psi_dev, n)) <= tol
        e = Q.qs_expval_pauli_sum(h, coeff, xm, zm)
        assert abs(e - O.expval(psi_dev, n, coeff, xm, zm).real) <= tol * np.abs(coeff).sum()
        Q.qs_apply_pauli_sum(h, coeff, xm, zm, h2)
        out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
        Q.qs_state_copy_to_host(h2, out)
        assert np.abs(out - O.apply_pauli_sum(psi_dev, n, coeff, xm, zm)).max() <= tol * np.abs(coeff).sum()
        ip = Q.qs_inner(h, h2)
        want = np.vdot(psi_dev, O.apply_pauli_sum(psi_dev, n, coeff, xm, zm))
        assert abs(ip - want) <= tol * np.abs(coeff).sum()
    finally:
        Q.qs_state_free(h)
        Q.qs_state_free(h2)


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("maker", ["hea", "ucc", "controlled"])
def test_adjoint_gradient_matches_oracle(dtname, maker):
    dt = DT[dtname]
    n = 10
    if maker == "hea":
        gates, p = W.hea(n, 3)
        theta = W.thetas_uniform(p, 1)
    elif maker == "ucc":
        gates, _ = W.ucc(n, 20, 2, wmin=2, wmax=6)
        p = 20
        theta = W.thetas_normal(p, 3, sigma=0.4)
    else:
        gates = W.random_layered(n, 2, 1) + [
            W.Gate("ry", (3,), (1,), param_index=0), W.Gate("p", (2,), (5, 6), param_index=1),
            W.Gate("rx", (0,), (9,), param_index=0, scale=-0.5), W.Gate("rz", (7,), param_index=2, scale=3.0),
            W.Gate("swap", (2, 8)), W.Gate("u2", (1, 4), matrix=tuple(W.random_unitary(4, np.random.default_rng(1)).reshape(-1)))]
        p = 3
        theta = np.array([0.3, -1.1, 0.7])
    H = W.random_pauli_sum(n, 30, seed=6)
    h = Q.qs_state_alloc(n, dt)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, theta, *H)
    finally:
        Q.qs_state_free(h)
    e_ref, g_ref = O.adjoint_grad(O.basis(n, 0), n, gates, theta, *H)
    scale = np.abs(H[0]).sum()
    assert abs(e - e_ref) <= TOL[dt] * scale * 10
    assert np.abs(g - g_ref).max() <= TOL[dt] * scale * 10


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("maker", ["mix", "hea"])
def test_adjoint_gradient_over_many_tiles(dtname, maker):
    """15 qubits: the reverse sweep runs as several tile passes of 2^12
    (complex64) or 2^11 (complex128) amplitudes over 8 or 16 tiles, with
    gradient parts summed over tiles and CTAs; every gate form, controlled
    rotations and two-target gates (mix), or the hardware-efficient ansatz."""
    dt = DT[dtname]
    n = 15
    if maker == "mix":
        gates, p = _parametrized_gate_mix(n, 140, seed=21)
        theta = W.thetas_uniform(p, 22)
    else:
        gates, p = W.hea(n, 4)
        theta = W.thetas_uniform(p, 23)
    H = W.random_pauli_sum(n, 25, seed=24)
    h = Q.qs_state_alloc(n, dt)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, theta, *H)
    finally:
        Q.qs_state_free(h)
    e_ref, g_ref = O.adjoint_grad(O.basis(n, 0), n, gates, theta, *H)
    scale = np.abs(H[0]).sum()
    assert abs(e - e_ref) <= TOL[dt] * scale * 10
    assert np.abs(g - g_ref).max() <= TOL[dt] * scale * 10


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_parametric_circuits_both_fusion_policies(dtname):
    """Parametric rotations resolved on the device (default) or folded into
    dense blocks rebuilt on the host at each execution (fuse_parametric=1)."""
    dt = DT[dtname]
    n = 11
    gates, p = W.hea(n, 4)
    ucc, _ = W.ucc(n, 10, 3, wmin=2, wmax=5)
    gates = gates + [W.Gate(g.kind, g.targets, g.controls, g.angle, g.param_index + p if g.param_index >= 0 else -1,
                            g.scale) for g in ucc]
    theta = W.thetas_uniform(p + 10, 5)
    want = ref(n, gates, theta)
    for opts in (Q.make_opts(fuse_k=3), Q.make_opts(fuse_k=4, fuse_parametric=1)):
        h = Q.qs_state_alloc(n, dt)
        plan = Q.qs_plan_create(n, dt, gates, opts)
        try:
            for th, w in ((theta, want), (theta * 0.5, ref(n, gates, theta * 0.5))):
                Q.qs_state_set_basis(h, 0)
                Q.qs_plan_execute(plan, h, th)
                out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
                Q.qs_state_copy_to_host(h, out)
                assert np.abs(out - w).max() <= TOL[dt]
        finally:
            Q.qs_plan_free(plan)
            Q.qs_state_free(h)


def test_parametric_tensor_core_blocks_built_on_device():
    """Rotations folded into 6-qubit tensor-core blocks whose W images are
    rebuilt on the device from theta at every execution."""
    n = 14
    gates, p = W.hea(n, 3)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4,
                                                            fuse_parametric=1))
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        assert any(op["type"] == 3 for op in Q.qs_plan_ops(plan))
        for seed in (1, 2):
            theta = W.thetas_uniform(p, seed)
            Q.qs_state_set_basis(h, 0)
            Q.qs_plan_execute(plan, h, theta)
            out = np.empty(1 << n, dtype=np.complex64)
            Q.qs_state_copy_to_host(h, out)
            assert np.abs(out - ref(n, gates, theta)).max() <= 2e-5
    finally:
        Q.qs_state_free(h)
        Q.qs_plan_free(plan)


def _parametrized_gate_mix(n, ngates, seed):
    """Every gate kind and form (permutations, diagonals, real, RX-like,
    dense, SWAP, dense two-target) with each parametric gate reading theta."""
    import dataclasses
    gates, p = [], 0
    for g in W.random_gate_mix(n, ngates, seed):
        if g.kind in W.PARAMETRIC_KINDS:
            g = dataclasses.replace(g, param_index=p, scale=1.0)
            p += 1
        gates.append(g)
    return gates, p


@pytest.mark.parametrize("mode", ["fused", "tensor"])
def test_device_built_blocks_equal_host_products(mode):
    """Blocks rebuilt on the device from theta (FP64 products, structured
    forms) against the host's FP64 products of the same members: dense and
    diagonal blocks to 1e-13; tensor-core W images compared as hi + lo (the
    value the MMAs multiply), each side within 2^-18 |w| of w, so 2^-16."""
    n = 13
    gates, p = _parametrized_gate_mix(n, 160, seed=11)
    if mode == "fused":   # the paper's merges: many 2-qubit dense blocks over every form
        opts = Q.make_opts(paper_mode=1, fuse_parametric=1)
        bar = 1e-13
    else:
        opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=3, fuse_parametric=1)
        bar = 2.0 ** -16
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        kinds = {op["type"] for op in Q.qs_plan_ops(plan)}
        assert (3 in kinds) if mode == "tensor" else (1 in kinds)
        for seed in (3, 4):
            worst, nb = Q.qs_plan_check_device_blocks(plan, h, W.thetas_uniform(p, seed))
            assert nb > 0
            assert worst <= bar
        theta = W.thetas_uniform(p, 5)
        Q.qs_state_set_basis(h, 0)
        Q.qs_plan_execute(plan, h, theta)
        out = np.empty(1 << n, dtype=np.complex64)
        Q.qs_state_copy_to_host(h, out)
        assert np.abs(out - ref(n, gates, theta)).max() <= 2e-5
    finally:
        Q.qs_state_free(h)
        Q.qs_plan_free(plan)


def test_adjoint_hea_n24_full_size_against_device_parameter_shift():
    """Hardware-efficient ansatz at its full size (24 qubits, 12 layers, 576
    parameters, 150-term H): the adjoint gradient equals the two-term shift
    rule evaluated with the device's own forward + expectation on 8 sampled
    parameters (a property that holds at any size)."""
    n = 24
    gates, p = W.hea(n, 12)
    theta = W.thetas_uniform(p, 4)
    H = W.random_pauli_sum(n, 150, seed=4)
    h = Q.qs_state_alloc(n, Q.QS_C128)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, theta, *H)
        plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(fuse_k=2))
        try:
            def f(th):
                Q.qs_state_set_basis(h, 0)
                Q.qs_plan_execute(plan, h, th)
                return Q.qs_expval_pauli_sum(h, *H)
            assert abs(f(theta) - e) < 1e-10
            for j in np.random.default_rng(0).choice(p, size=8, replace=False):
                tp, tm = theta.copy(), theta.copy()
                tp[j] += math.pi / 2
                tm[j] -= math.pi / 2
                assert abs(0.5 * (f(tp) - f(tm)) - g[j]) < 1e-10
        finally:
            Q.qs_plan_free(plan)
    finally:
        Q.qs_state_free(h)


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_batched_graph_matches_sequential_and_oracle(dtname):
    dt = DT[dtname]
    n, nterms, Bsz = 14, 16, 4
    gates, _ = W.ucc(n, nterms, 5, wmin=2, wmax=6)
    thetas = W.thetas_normal(nterms, 6, sigma=0.3, batch=Bsz)
    H = W.random_pauli_sum(n, 25, seed=8)
    modes = [None, Q.make_opts(fuse_k=1), Q.make_opts(fuse_k=3), Q.make_opts(fuse_k=4, fuse_parametric=1)]
    if dt == Q.QS_C64:
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2))
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1))
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1, tc_pipeline=1))
    for opts in modes:
        plan = Q.qs_plan_create(n, dt, gates, opts)
        states = [Q.qs_state_alloc(n, dt) for _ in range(Bsz)]
        try:
            for rep in range(2):      # second call replays the captured graph
                for s in states:
                    Q.qs_state_set_basis(s, 0)
                th = thetas if rep == 0 else thetas[::-1].copy()
                ex = Q.qs_plan_execute_batched(plan, states, th, H)
                for b in range(Bsz):
                    want = O.expval_of_circuit(O.basis(n, 0), n, gates, th[b], *H)
                    assert abs(ex[b] - want) <= TOL[dt] * np.abs(H[0]).sum() * 10
        finally:
            for s in states:
                Q.qs_state_free(s)
            Q.qs_plan_free(plan)


@pytest.mark.parametrize("n,depth,ent", [(13, 6, "cnot"), (15, 8, "cz"), (17, 5, "cnot")])
def test_tensor_core_mode_split_products_match_oracle(n, depth, ent):
    """6-qubit blocks on tensor cores (fp16 and bf16 hi/lo split products,
    FP32 accumulation) interleaved with CUDA-core tile passes, complex64 bar
    2e-5, both pipelines."""
    gates = W.random_layered(n, depth, seed=n, entangler=ent)
    psi0 = W.random_state(n, 2)
    want = ref(n, gates, psi0=psi0.astype(np.complex64).astype(complex))
    for tmin, pipe, prec in ((6, 0, 4), (10, 0, 4), (6, 1, 4), (6, 0, 3), (6, 1, 3)):
        opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_precision=prec, tc_min_gates=tmin, tc_pipeline=pipe)
        plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        try:
            assert any(op["type"] == 3 for op in Q.qs_plan_ops(plan))
            h = Q.qs_state_alloc(n, Q.QS_C64)
            try:
                Q.qs_state_copy_from_host(h, psi0.astype(np.complex64))
                Q.qs_plan_execute(plan, h)
                out = np.empty(1 << n, dtype=np.complex64)
                Q.qs_state_copy_to_host(h, out)
            finally:
                Q.qs_state_free(h)
        finally:
            Q.qs_plan_free(plan)
        assert np.abs(out - want).max() <= 2e-5


# Block placements covering 4, 3, 2, 1 and 0 block qubits among qubits 0-3
# (the shared-memory bank bits of the bulk-copy kernel's slot reads), plus
# blocks entirely above the row qubits.
BLOCK_SETS = [(0, 1, 2, 3, 4, 5), (0, 1, 2, 9, 10, 11), (1, 3, 7, 9, 11, 12), (0, 7, 8, 9, 10, 11),
              (7, 8, 9, 10, 11, 12), (2, 4, 5, 6, 8, 12)]


@pytest.mark.parametrize("n", [13, 14, 17])
def test_tensor_core_pipelines_on_every_block_placement(n):
    """Dense 6-qubit blocks on the placements above (and, for n = 17, on the
    six highest qubits): the bulk-copy and the register-staged tensor-core
    kernels against the oracle (complex64 bar 2e-5) and against each other.
    Both round the same operands to bf16 and issue the same MMAs, so they
    agree to FP32 accumulation-order level (2^-20 of the largest amplitude)."""
    sets = list(BLOCK_SETS) + ([tuple(range(n - 6, n))] if n > 13 else [])
    gates = W.block_circuit(sets, 12, seed=n)
    psi0 = W.random_state(n, 4).astype(np.complex64)
    want = ref(n, gates, psi0=psi0.astype(complex))
    outs = []
    for pipe in (0, 1):
        opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=6, tc_pipeline=pipe)
        plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        try:
            tc_sets = [tuple(sorted(op["qubits"])) for op in Q.qs_plan_ops(plan) if op["type"] == 3]
            assert len(tc_sets) == len(sets)
            h = Q.qs_state_alloc(n, Q.QS_C64)
            try:
                Q.qs_state_copy_from_host(h, psi0)
                Q.qs_plan_execute(plan, h)
                out = np.empty(1 << n, dtype=np.complex64)
                Q.qs_state_copy_to_host(h, out)
            finally:
                Q.qs_state_free(h)
        finally:
            Q.qs_plan_free(plan)
        assert np.abs(out - want).max() <= 2e-5
        outs.append(out)
    assert np.abs(outs[0] - outs[1]).max() <= 2.0 ** -20 * np.abs(want).max()


def test_tensor_core_plain_bf16_error_bound():
    """Plain bf16 products (one MMA per k-step): error within the bf16
    rounding bound, about 2^-8 of the largest amplitude per block."""
    n = 14
    gates = W.random_layered(n, 6, seed=5)
    want = ref(n, gates)
    opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_precision=1)
    out = run(n, Q.QS_C64, gates, opts=opts)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
    ntc = sum(1 for op in Q.qs_plan_ops(plan) if op["type"] == 3)
    Q.qs_plan_free(plan)
    assert ntc >= 1
    assert np.abs(out - want).max() <= ntc * 2.0 ** -8 * np.abs(want).max()


def test_tensor_core_config2_shape_n20_depth40_cz():
    """The layer structure of the 32-qubit tensor-core workload (CZ
    entanglers, depth 40) at 20 qubits, where the oracle finishes in seconds."""
    n = 20
    gates = W.random_layered(n, 40, seed=0, entangler="cz")
    want = ref(n, gates)
    out = run(n, Q.QS_C64, gates, opts=Q.make_opts(mode=Q.QS_MODE_TENSOR))
    assert np.abs(out - want).max() <= 2e-5


class oracle_threads:
    """Runs the oracle on every host core inside the block (its gate loops
    split the amplitudes among threads; results are bit-identical to one
    thread), one thread again after."""

    def __enter__(self):
        O.lib().or_set_threads(0)

    def __exit__(self, *exc):
        O.lib().or_set_threads(1)


# 6-qubit placements at 23 qubits: inside the lowest rows, across the tile
# boundary (tile widths 12-13), spread from qubit 0 to the top, and entirely
# among the highest qubits (the tile-index bits of the address).
BLOCK_SETS_N23 = [(0, 1, 2, 3, 4, 5), (9, 10, 11, 12, 13, 14), (0, 5, 11, 13, 17, 22),
                  (17, 18, 19, 20, 21, 22), (3, 4, 12, 19, 20, 21), (1, 2, 3, 14, 15, 16)]


@pytest.mark.parametrize("pipe", [0, 1])
def test_tensor_core_single_state_n23_every_block_placement(pipe):
    """A single 2^23 complex64 state (2^11 tiles, several per CTA) through
    dense 6-qubit blocks on the placements above, on both tensor-core
    pipelines: every amplitude against the oracle, bar 2e-5."""
    n = 23
    gates = W.block_circuit(BLOCK_SETS_N23, 12, seed=23)
    psi0 = W.random_state(n, 9).astype(np.complex64)
    with oracle_threads():
        want = ref(n, gates, psi0=psi0.astype(complex))
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=6,
                                                            tc_pipeline=pipe))
    try:
        tc_sets = [tuple(sorted(op["qubits"])) for op in Q.qs_plan_ops(plan) if op["type"] == 3]
        assert len(tc_sets) == len(BLOCK_SETS_N23)
        h = Q.qs_state_alloc(n, Q.QS_C64)
        try:
            Q.qs_state_copy_from_host(h, psi0)
            Q.qs_plan_execute(plan, h)
            out = np.empty(1 << n, dtype=np.complex64)
            Q.qs_state_copy_to_host(h, out)
        finally:
            Q.qs_state_free(h)
    finally:
        Q.qs_plan_free(plan)
    assert np.abs(out - want).max() <= 2e-5


@pytest.mark.parametrize("n", [22, 24])
def test_tensor_core_default_plan_random_layers_n22_n24(n):
    """The default tensor-core plan of the layered random circuit at 22 and
    24 qubits (a single state, one persistent CTA per SM walking many tiles):
    every amplitude against the oracle, complex64 bar 2e-5 and complex128
    bar 1e-12."""
    gates = W.random_layered(n, 12, seed=n)
    with oracle_threads():
        want = ref(n, gates)
    for dt in (Q.QS_C64, Q.QS_C128):
        out = run(n, dt, gates, opts=Q.make_opts(mode=Q.QS_MODE_TENSOR))
        assert np.abs(out - want).max() <= TOL[dt], dt


_CZ26 = {}


def _cz26():
    """The 32-qubit tensor-core workload's structure (random layers, CZ
    entanglers, depth 40) at 26 qubits and its oracle state (computed once)."""
    if not _CZ26:
        n = 26
        gates = W.random_layered(n, 40, seed=0, entangler="cz")
        with oracle_threads():
            _CZ26["v"] = (n, gates, ref(n, gates))
    return _CZ26["v"]


@pytest.mark.parametrize("dtname,prec", [("c64", 4), ("c64", 3), ("c128", 0)])
def test_tensor_core_cz_depth40_n26_against_the_oracle(dtname, prec):
    """Depth 40 of CZ layers at 26 qubits (1560 gates, 2^14 tiles) on the
    tensor-core plan: complex64 with the fp16 and the bf16 split products (bar
    2e-5) and complex128 with exact digit products (bar 1e-12), every
    amplitude against the oracle."""
    n, gates, want = _cz26()
    dt = DT[dtname]
    kw = dict(mode=Q.QS_MODE_TENSOR)
    if prec:
        kw["tc_precision"] = prec
    out = run(n, dt, gates, opts=Q.make_opts(**kw))
    assert np.abs(out - want).max() <= TOL[dt]


def _structured_pauli_sum(n, seed):
    """Every x-mask case of the batched expectation kernel: x = 0 (Z
    strings), x = 1, odd and even x with a high bit, and 11 strings sharing one
    x (more than one launch group of 8), plus random strings."""
    rng = np.random.default_rng(seed)
    xs, zs = [], []
    for x in (0, 0, 1, 3, (1 << (n - 1)) | 1, 2, 6, 1 << (n - 1)):
        xs.append(x & ((1 << n) - 1))
        zs.append(int(rng.integers(0, 1 << n)))
    shared = int(rng.integers(1, 1 << n))
    for _ in range(11):
        xs.append(shared)
        zs.append(int(rng.integers(0, 1 << n)))
    c, xr, zr = W.random_pauli_sum(n, 12, seed)
    coeff = np.concatenate([rng.standard_normal(len(xs)), c])
    return coeff, np.array(xs + list(xr), dtype=np.uint64), np.array(zs + list(zr), dtype=np.uint64)


@pytest.mark.parametrize("n", [2, 13])
def test_batched_expectation_every_mask_case(n):
    """Batched <H> (one launch per wave of states, 16-byte pair loads) on a
    sum that hits every x-mask case, against the oracle per state: bar 2e-5
    times the coefficient sum (complex64)."""
    Bsz = 5
    gates = W.random_layered(n, 3, seed=n)
    H = _structured_pauli_sum(n, seed=7)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(fuse_k=2, tile_qubits=min(n, 8), low_qubits=1))
    states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
    try:
        for b, s in enumerate(states):
            Q.qs_state_set_basis(s, (b * 2654435761) % (1 << n))
        ex = Q.qs_plan_execute_batched(plan, states, None, H)
        for b in range(Bsz):
            psi = O.apply_circuit(O.basis(n, (b * 2654435761) % (1 << n)), n, gates, None)
            want = O.expval(psi, n, *H).real
            assert abs(ex[b] - want) <= 2e-5 * np.abs(H[0]).sum()
    finally:
        for s in states:
            Q.qs_state_free(s)
        Q.qs_plan_free(plan)


@pytest.mark.parametrize("n,Bsz", [(15, 77), (16, 40)])
@pytest.mark.parametrize("pipe", [0, 1])
def test_batched_tensor_core_ranges_cross_states(n, Bsz, pipe):
    """Per-CTA tile ranges of 3 tiles over states of 4 (n = 15) or 8 (n = 16)
    tiles: most CTAs cross a state boundary mid-range and reload that state's
    W image (rebuilt from its own theta) while earlier tiles are in flight.
    States of every row against the oracle, complex64 bar 2e-5 (the states
    keep most weight on |0..0>, amplitude about 0.76: the default fp16 split
    holds the bar there, the bf16 split, about 2^-16 per pass, does not)."""
    nterms = 8
    gates, _ = W.ucc(n, nterms, seed=n)
    thetas = W.thetas_normal(nterms, 10 + n, sigma=0.5, batch=Bsz)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4,
                                                            fuse_parametric=1, tc_pipeline=pipe))
    states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
    try:
        assert any(op["type"] == 3 for op in Q.qs_plan_ops(plan))
        for rep_ in range(2):            # capture, then graph replay
            for s in states:
                Q.qs_state_set_basis(s, 0)
            Q.qs_plan_execute_batched(plan, states, thetas)
        for b in range(Bsz):
            out = np.empty(1 << n, dtype=np.complex64)
            Q.qs_state_copy_to_host(states[b], out)
            assert np.abs(out - ref(n, gates, thetas[b])).max() <= 2e-5, b
    finally:
        for s in states:
            Q.qs_state_free(s)
        Q.qs_plan_free(plan)


@pytest.mark.parametrize("pipe", [0, 1])
def test_batched_tensor_core_more_tiles_than_sms(pipe):
    """77 states of 14 qubits: 154 tensor-core tiles over 152 CTAs, so the
    contiguous per-CTA tile ranges (two tiles each) leave trailing CTAs with
    nothing to do; blocks rebuilt per state from theta (per-state W images).
    Sampled rows against the oracle, complex64 bar 2e-5."""
    n, Bsz, nterms = 14, 77, 10
    gates, _ = W.ucc(n, nterms, seed=8)
    thetas = W.thetas_normal(nterms, 9, sigma=0.3, batch=Bsz)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4,
                                                            fuse_parametric=1, tc_pipeline=pipe))
    states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
    try:
        assert any(op["type"] == 3 for op in Q.qs_plan_ops(plan))
        for s in states:
            Q.qs_state_set_basis(s, 0)
        Q.qs_plan_execute_batched(plan, states, thetas)
        for b in (0, 1, 38, 75, 76):
            out = np.empty(1 << n, dtype=np.complex64)
            Q.qs_state_copy_to_host(states[b], out)
            assert np.abs(out - ref(n, gates, thetas[b])).max() <= 2e-5
    finally:
        for s in states:
            Q.qs_state_free(s)
        Q.qs_plan_free(plan)


def test_batched_fixed_circuit_without_parameters():
    n, Bsz = 13, 3
    gates = W.random_layered(n, 5, seed=21)
    want = ref(n, gates)
    for opts in (Q.make_opts(fuse_k=2), Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2),
                 Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2, tc_pipeline=1)):
        plan = Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        states = [Q.qs_state_alloc(n, Q.QS_C64) for _ in range(Bsz)]
        try:
            Q.qs_plan_execute_batched(plan, states)
            for s in states:
                out = np.empty(1 << n, dtype=np.complex64)
                Q.qs_state_copy_to_host(s, out)
                assert np.abs(out - want).max() <= 2e-5
        finally:
            for s in states:
                Q.qs_state_free(s)
            Q.qs_plan_free(plan)


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_gathered_amplitudes_equal_the_full_copy(dtname):
    dt = DT[dtname]
    n = 13
    gates = W.random_layered(n, 4, seed=3)
    h = Q.qs_state_alloc(n, dt)
    try:
        Q.qs_apply_circuit(h, gates)
        full = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
        Q.qs_state_copy_to_host(h, full)
        idx = np.array([0, 1, 7, (1 << n) - 1, 4096, 17, 17], dtype=np.uint64)
        got = Q.qs_state_get_amplitudes(h, idx, dt)
        assert np.array_equal(got, full[idx.astype(np.int64)])
        assert len(Q.qs_state_get_amplitudes(h, [], dt)) == 0
        with pytest.raises(Q.QsError):
            Q.qs_state_get_amplitudes(h, [1 << n], dt)
    finally:
        Q.qs_state_free(h)


def test_invalid_sizes_give_errors_not_faults():
    h = Q.qs_state_alloc(4, Q.QS_C64)
    try:
        with pytest.raises(Q.QsError):
            Q.qs_state_set_basis(h, 1 << 4)
        with pytest.raises(Q.QsError):
            Q.qs_state_copy_to_host(h, np.empty(8, dtype=np.complex64))
        with pytest.raises(Q.QsError):
            Q.qs_apply_circuit(h, [W.Gate("h", (4,))])
        with pytest.raises(Q.QsError):
            Q.qs_expval_pauli_sum(h, [1.0], [1 << 4], [0])
        with pytest.raises(Q.QsError):
            Q.qs_apply_circuit(h, [W.Gate("rx", (0,), param_index=3)], np.zeros(2))
    finally:
        Q.qs_state_free(h)
    with pytest.raises(Q.QsError) as e:
        Q.qs_state_alloc(40, Q.QS_C128)     # 16 TiB
    assert e.value.status == Q.QS_ERR_OOM


def test_state_diff_mixed_precision():
    n = 12
    psi = W.random_state(n, 9)
    a = Q.qs_state_alloc(n, Q.QS_C64)
    b = Q.qs_state_alloc(n, Q.QS_C128)
    try:
        Q.qs_state_copy_from_host(a, psi.astype(np.complex64))
        Q.qs_state_copy_from_host(b, psi)
        m, l2 = Q.qs_state_diff(a, b)
        d = psi.astype(np.complex64).astype(complex) - psi
        assert abs(m - np.abs(d).max()) < 1e-15 and abs(l2 - np.linalg.norm(d)) < 1e-12
    finally:
        Q.qs_state_free(a)
        Q.qs_state_free(b)


def test_autotuner_picks_a_valid_plan_and_caches_it():
    n = 14
    gates = W.random_layered(n, 6, seed=30)
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        best, ms = Q.qs_plan_autotune(h, gates)
        assert ms > 0
        best2, ms2 = Q.qs_plan_autotune(h, gates)      # cached: same answer
        assert Q.opts_dict(best) == Q.opts_dict(best2) and ms2 == ms
        Q.qs_state_set_basis(h, 0)
        Q.qs_apply_circuit(h, gates, None, best)
        out = np.empty(1 << n, dtype=np.complex64)
        Q.qs_state_copy_to_host(h, out)
        assert np.abs(out - ref(n, gates)).max() <= 2e-5
    finally:
        Q.qs_state_free(h)


def test_launch_counter_moves():
    before = Q.qs_launch_count()
    run(8, Q.QS_C64, W.random_layered(8, 2, 0))
    assert Q.qs_launch_count() > before


def _phase_workload(maker, n):
    if maker == "qaoa":
        return W.qaoa(n, 3, W.random_regular_graph(n, 3, seed=n))
    return W.phase_run_circuit(n, 3, 30, seed=n)


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("maker,n", [("qaoa", 16), ("zoo", 15), ("qaoa", 12), ("zoo", 13), ("zoo", 18)])
def test_phase_pass_matches_oracle(dtname, maker, n):
    """Diagonal phase runs (QAOA cost layers; Z-string exponentials, one-control
    phases and SWAP sandwiches) as one sweep each, from a random state, element
    by element against the oracle. n = 12 is a single 4096-amplitude chunk;
    n = 18 spans more chunks than the grid has warps."""
    dt = DT[dtname]
    gates, p = _phase_workload(maker, n)
    theta = W.thetas_uniform(max(p, 1), 7)
    psi0 = W.random_state(n, 8)
    want = ref(n, gates, theta, psi0=psi0)
    modes = [Q.make_opts(), Q.make_opts(fuse_k=2, phase_min_gates=4)]
    if dt == Q.QS_C64 and n >= 13:
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1))
    if dt == Q.QS_C128:   # phase and tile passes in FP64 (FP32 pairs are the default)
        modes.append(Q.make_opts(c128_pairs=2))
    for opts in modes:
        plan = Q.qs_plan_create(n, dt, gates, opts)
        try:
            assert sum(op["type"] == 4 for op in Q.qs_plan_ops(plan)) >= 3
        finally:
            Q.qs_plan_free(plan)
        got = run(n, dt, gates, theta, psi0=psi0, opts=opts)
        assert np.abs(got - want).max() <= TOL[dt], (opts, np.abs(got - want).max())


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_phase_pass_batched_rows_use_their_own_parameters(dtname):
    """A QAOA plan executed for several parameter rows in one CUDA graph: the
    phase pass reads each row's angles; every row's state and <C> against the
    oracle, on capture and on replay with the rows reversed."""
    dt = DT[dtname]
    n, Bsz = 14, 5
    edges = W.random_regular_graph(n, 3, seed=3)
    gates, p = W.qaoa(n, 2, edges)
    H = W.maxcut_hamiltonian(edges)
    thetas = np.stack([W.thetas_uniform(p, 20 + b) for b in range(Bsz)])
    modes = [Q.make_opts(), Q.make_opts(fuse_k=4, fuse_parametric=1)]
    if dt == Q.QS_C64:
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1))
    else:   # phase and tile passes in FP64 (FP32 pairs are the default), per-row angles
        modes.append(Q.make_opts(fuse_k=2, fuse_parametric=1, c128_pairs=2))
    for opts in modes:
        plan = Q.qs_plan_create(n, dt, gates, opts)
        states = [Q.qs_state_alloc(n, dt) for _ in range(Bsz)]
        try:
            for rep in range(2):
                for s in states:
                    Q.qs_state_set_basis(s, 0)
                th = thetas if rep == 0 else thetas[::-1].copy()
                ex = Q.qs_plan_execute_batched(plan, states, th, H)
                for b in range(Bsz):
                    psi = O.apply_circuit(O.basis(n, 0), n, gates, th[b])
                    out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
                    Q.qs_state_copy_to_host(states[b], out)
                    assert np.abs(out - psi).max() <= TOL[dt]
                    assert abs(ex[b] - O.expval(psi, n, *H).real) <= TOL[dt] * np.abs(H[0]).sum() * 10
        finally:
            for s in states:
                Q.qs_state_free(s)
            Q.qs_plan_free(plan)


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("maker,n", [("hea", 12), ("qaoa", 14), ("layered", 11), ("mix", 7), ("hea", 5)])
def test_smgp_staggered_groups_match_oracle(dtname, maker, n):
    """Staggered multi-gate plans (groups of 8, 4 and 2 one-target gates, one
    two-dimensional launch per time step) element by element against the
    oracle, from a random state; every one-target form inside groups."""
    dt = DT[dtname]
    theta = None
    if maker == "hea":
        gates, p = W.hea_staggered(n, 3)
        theta = W.thetas_uniform(p, 5)
    elif maker == "qaoa":
        gates, p = W.qaoa(n, 2, W.random_regular_graph(n, 3, seed=2))
        theta = W.thetas_uniform(p, 6)
    elif maker == "layered":
        gates = W.random_layered(n, 6, seed=4)
    else:
        kinds = ("h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "p")
        rng = np.random.default_rng(9)
        gates = [W.Gate(kinds[int(rng.integers(0, len(kinds)))], (q,), angle=float(rng.uniform(-3, 3)))
                 for _ in range(4) for q in rng.permutation(n)]
    psi0 = W.random_state(n, 10)
    plan = Q.qs_plan_create(n, dt, gates, Q.make_opts(mode=Q.QS_MODE_SMGP))
    try:
        info = Q.qs_plan_info_get(plan)
        assert info["launches"] == len(gates)   # S launches per group of S gates
    finally:
        Q.qs_plan_free(plan)
    got = run(n, dt, gates, theta, psi0=psi0, opts=Q.make_opts(mode=Q.QS_MODE_SMGP))
    want = ref(n, gates, theta, psi0=psi0)
    assert np.abs(got - want).max() <= TOL[dt]


PAIRS = [Q.make_opts(fuse_k=1, c128_pairs=1), Q.make_opts(fuse_k=3, c128_pairs=1),
         Q.make_opts(fuse_k=5, tile_qubits=11, low_qubits=3, c128_pairs=1),
         Q.make_opts(fuse_k=2, tile_qubits=6, low_qubits=2, c128_pairs=1),
         Q.make_opts(paper_mode=1, c128_pairs=1)]


@pytest.mark.parametrize("oi", range(len(PAIRS)))
def test_c128_fp32_pair_tile_passes_match_oracle(oi):
    """complex128 tile passes computed in FP32 pairs (every gate kind and form,
    dense blocks k = 1..5, diagonal blocks) hold the complex128 bar against the
    oracle, and sit within 1e-13 of the FP64 tile passes."""
    n = 9
    gates = W.random_gate_mix(n, 120, seed=30 + oi) + W.random_layered(n, 3, seed=oi)
    psi0 = W.random_state(n, 4)
    want = ref(n, gates, psi0=psi0)
    got = run(n, Q.QS_C128, gates, psi0=psi0, opts=PAIRS[oi])
    assert np.abs(got - want).max() <= 1e-12
    fp64 = run(n, Q.QS_C128, gates, psi0=psi0, opts=Q.make_opts(fuse_k=3))
    assert np.abs(got - fp64).max() <= 1e-13


def test_c128_fp32_pairs_many_tiles_and_parameters():
    """n = 18 random layers over many tiles, and a parametric HEA (device-resolved
    angles, blocks rebuilt from theta) in FP32 pairs, against the oracle."""
    n = 18
    gates = W.random_layered(n, 6, seed=4)
    got = run(n, Q.QS_C128, gates, opts=Q.make_opts(fuse_k=4, c128_pairs=1))
    assert np.abs(got - ref(n, gates)).max() <= 1e-12
    n = 12
    gates, p = W.hea_staggered(n, 3)
    theta = W.thetas_uniform(p, 3)
    for opts in (Q.make_opts(c128_pairs=1), Q.make_opts(fuse_k=3, fuse_parametric=1, c128_pairs=1)):
        got = run(n, Q.QS_C128, gates, theta, opts=opts)
        assert np.abs(got - ref(n, gates, theta)).max() <= 1e-12


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("maker", ["layered", "qaoa", "mix"])
def test_stream_apply_host_resident_state(dtname, maker):
    """A state held in host memory and streamed through three device buffers
    (Section 3.2's batches, high qubits = batch index) equals the oracle, with
    per-gate, fused and (complex64, 13-qubit buffers) tensor-core sub-plans,
    from pageable numpy memory and from pinned torch memory."""
    import torch
    dt = DT[dtname]
    n, theta = 16, None
    if maker == "layered":
        gates = W.random_layered(n, 5, seed=3)
    elif maker == "qaoa":
        gates, p = W.qaoa(n, 2, W.random_regular_graph(n, 3, seed=4))
        theta = W.thetas_uniform(p, 2)
    else:
        gates = [g for g in W.random_gate_mix(n, 80, seed=5) if sum(q >= 10 for q in g.qubits) <= 2]
    psi0 = W.random_state(n, 6)
    want = ref(n, gates, theta, psi0=psi0)
    cases = [(None, 10, 2), (Q.make_opts(), 10, 2), (Q.make_opts(fuse_k=3), 11, 3)]
    if dt == Q.QS_C64:
        cases.append((Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2), 11, 2))
    for opts, l, h in cases:
        host = np.array(psi0, dtype=Q.NP_DTYPE[dt], copy=True)   # streamed in place
        info = Q.qs_stream_apply(host, n, dt, gates, theta, opts, batch_qubits=l, pass_qubits=h)
        assert info["passes"] == len(Q.qs_stream_plan(n, gates, l, h)) >= 2
        assert np.abs(host - want).max() <= TOL[dt], (opts, l, h)
    pinned = torch.from_numpy(np.array(psi0, dtype=Q.NP_DTYPE[dt], copy=True)).pin_memory()
    Q.qs_stream_apply(pinned, n, dt, gates, theta, Q.make_opts(), batch_qubits=10, pass_qubits=2)
    assert np.abs(pinned.numpy() - want).max() <= TOL[dt]


@pytest.mark.parametrize("dtname", ["c128", "c64"])
@pytest.mark.parametrize("nwork", [1, 2, 3])
def test_execute_host_pipeline_matches_oracle(dtname, nwork):
    """qs_plan_execute_host: five different host-resident input states through
    1-3 device work states (copies in and out overlapped with the circuit);
    every output and its norm against the oracle, including a parametric
    circuit resolved once for all inputs and a host_out of NULL (norms only)."""
    import torch
    dt = DT[dtname]
    n = 14
    gates, p = W.hea_staggered(n, 2)
    theta = W.thetas_uniform(p, 4)
    ins = [np.array(W.random_state(n, 40 + i), dtype=Q.NP_DTYPE[dt]) for i in range(5)]
    outs = [torch.empty(1 << n, dtype=torch.complex128 if dt == Q.QS_C128 else torch.complex64).pin_memory()
            for _ in range(5)]
    opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2, fuse_parametric=1) if dt == Q.QS_C64 else Q.make_opts()
    plan = Q.qs_plan_create(n, dt, gates, opts)
    work = [Q.qs_state_alloc(n, dt) for _ in range(nwork)]
    try:
        norms = Q.qs_plan_execute_host(plan, work, ins, outs, theta)
        for i in range(5):
            want = ref(n, gates, theta, psi0=ins[i].astype(np.complex128))
            assert np.abs(outs[i].numpy() - want).max() <= TOL[dt]
            assert abs(norms[i] - 1) <= 10 * TOL[dt]
        norms2 = Q.qs_plan_execute_host(plan, work, ins[:2], None, theta)
        assert np.abs(norms2 - norms[:2]).max() <= 1e-12
    finally:
        for w in work:
            Q.qs_state_free(w)
        Q.qs_plan_free(plan)


def test_stream_and_pipeline_edge_cases():
    """Streaming with every batch alone (pass_qubits 0: only gates below the batch
    qubits), with one batch holding the whole state (batch_qubits = n), and the
    host pipeline with no inputs."""
    n = 13
    dt = Q.QS_C128
    psi0 = W.random_state(n, 12)
    low_gates = [g for g in W.random_layered(n, 4, seed=6) if max(g.qubits) < 9]
    host = np.array(psi0, copy=True)
    info = Q.qs_stream_apply(host, n, dt, low_gates, None, Q.make_opts(), batch_qubits=9, pass_qubits=0)
    assert info["passes"] == 1 and info["groups"] == 16
    assert np.abs(host - ref(n, low_gates, psi0=psi0)).max() <= TOL[dt]
    gates = W.random_layered(n, 4, seed=7)
    host = np.array(psi0, copy=True)
    info = Q.qs_stream_apply(host, n, dt, gates, None, None, batch_qubits=n, pass_qubits=0)
    assert info["passes"] == 1 and info["groups"] == 1
    assert np.abs(host - ref(n, gates, psi0=psi0)).max() <= TOL[dt]
    plan = Q.qs_plan_create(n, dt, gates, Q.make_opts())
    w = Q.qs_state_alloc(n, dt)
    try:
        assert len(Q.qs_plan_execute_host(plan, [w], [], [])) == 0
    finally:
        Q.qs_state_free(w)
        Q.qs_plan_free(plan)


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_batched_l2_waves_ragged(dtname):
    """Batched execution in L2-sized waves (batch_l2_waves: two 32 MiB states per
    wave, the last wave holding one): every row's state and <H> equal the
    default pass-by-pass schedule and the oracle, for CUDA-core plans with parametric blocks rebuilt per row
    and (complex64) tensor-core plans with per-row W images."""
    dt = DT[dtname]
    n = 22 if dt == Q.QS_C64 else 21
    Bsz = 5
    gates, _ = W.ucc(n, 10, seed=3, wmin=2, wmax=5)
    th = W.thetas_normal(10, 4, sigma=0.3, batch=Bsz)
    H = W.random_pauli_sum(n, 12, seed=5)
    modes = [Q.make_opts(fuse_k=4, fuse_parametric=1)]
    if dt == Q.QS_C64:
        modes.append(Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4, fuse_parametric=1))
    want2 = O.apply_circuit(O.basis(n, 0), n, gates, th[2])
    want_e = [O.expval(O.apply_circuit(O.basis(n, 0), n, gates, th[b]), n, *H).real for b in range(Bsz)]
    for base in modes:
        results = []
        for waves in (1, 0):
            o = Q.make_opts(mode=base.mode, fuse_k=base.fuse_k, fuse_parametric=1, tc_min_gates=base.reserved[0],
                            batch_l2_waves=waves)
            plan = Q.qs_plan_create(n, dt, gates, o)
            states = [Q.qs_state_alloc(n, dt) for _ in range(Bsz)]
            try:
                for s in states:
                    Q.qs_state_set_basis(s, 0)
                ex = Q.qs_plan_execute_batched(plan, states, th, H)
                out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
                Q.qs_state_copy_to_host(states[2], out)
                results.append((ex, out))
            finally:
                for s in states:
                    Q.qs_state_free(s)
                Q.qs_plan_free(plan)
        (ex0, out0), (ex1, out1) = results
        assert np.abs(out0 - want2).max() <= TOL[dt]
        assert np.abs(out0 - out1).max() <= TOL[dt]
        for b in range(Bsz):
            assert abs(ex0[b] - want_e[b]) <= TOL[dt] * np.abs(H[0]).sum() * 10
            assert abs(ex0[b] - ex1[b]) <= TOL[dt] * np.abs(H[0]).sum() * 10


@pytest.mark.parametrize("maker", ["mix", "hea"])
def test_adjoint_gradient_c128_fp32_pairs_and_options(maker):
    """qs_adjoint_grad_opts: complex128 with the forward tile passes and the
    reverse sweep in FP32 pairs, against the oracle at the complex128 bar and
    within 1e-12 of the FP64 sweep; complex64 with a tensor-core forward plan."""
    n = 15
    if maker == "mix":
        gates, p = _parametrized_gate_mix(n, 140, seed=31)
        theta = W.thetas_uniform(p, 32)
    else:
        gates, p = W.hea(n, 4)
        theta = W.thetas_uniform(p, 33)
    H = W.random_pauli_sum(n, 25, seed=34)
    scale = np.abs(H[0]).sum()
    e_ref, g_ref = O.adjoint_grad(O.basis(n, 0), n, gates, theta, *H)
    h = Q.qs_state_alloc(n, Q.QS_C128)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, theta, *H, opts=Q.make_opts(c128_pairs=1))
        e64, g64 = Q.qs_adjoint_grad(h, gates, theta, *H, opts=Q.make_opts(c128_pairs=2))
    finally:
        Q.qs_state_free(h)
    assert abs(e - e_ref) <= 1e-12 * scale * 10
    assert np.abs(g - g_ref).max() <= 1e-12 * scale * 10
    assert np.abs(g - g64).max() <= 1e-12 * scale
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        e, g = Q.qs_adjoint_grad(h, gates, theta, *H, opts=Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=2,
                                                                         fuse_parametric=1))
    finally:
        Q.qs_state_free(h)
    assert np.abs(g - g_ref).max() <= 2e-5 * scale * 10


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_phase_pass_complete_graph_many_terms(dtname):
    """QAOA on the complete graph of 14 qubits: 91 ZZ terms in one phase run
    (66 inside the 12 low bits, 24 with one low bit, 1 above), so the per-bit
    factor lists hold several terms each; against the oracle."""
    dt = DT[dtname]
    n = 14
    edges = [(u, v) for u in range(n) for v in range(u + 1, n)]
    gates, p = W.qaoa(n, 2, edges)
    theta = np.array([0.23, -0.41, 0.17, 0.62])
    plan = Q.qs_plan_create(n, dt, gates, Q.make_opts())
    try:
        runs = [op for op in Q.qs_plan_ops(plan) if op["type"] == 4]
        assert len(runs) == 2 and len(runs[0]["terms"]) >= 91
    finally:
        Q.qs_plan_free(plan)
    got = run(n, dt, gates, theta, opts=Q.make_opts())
    assert np.abs(got - ref(n, gates, theta)).max() <= TOL[dt]


def test_torch_autograd_expval_with_options():
    """Q.expval through torch.autograd: the value and theta.grad equal the
    oracle's adjoint gradient, with the default plan (complex128 CUDA-core
    passes in FP32 pairs) and with FP64 passes asked for in the plan options."""
    import torch
    n = 10
    gates, p = W.hea(n, 3)
    th0 = W.thetas_uniform(p, 41)
    H = W.random_pauli_sum(n, 12, seed=42)
    e_ref, g_ref = O.adjoint_grad(O.basis(n, 0), n, gates, th0, *H)
    scale = np.abs(H[0]).sum()
    psi0 = Q.State(n, "c128")
    try:
        for opts in (None, Q.make_opts(c128_pairs=2)):
            theta = torch.tensor(th0, requires_grad=True)
            e = Q.expval(theta, psi0, gates, H, opts)
            e.backward()
            assert abs(float(e.detach()) - e_ref) <= 1e-12 * scale * 10
            assert np.abs(theta.grad.numpy() - g_ref).max() <= 1e-12 * scale * 10
    finally:
        psi0.free()


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_two_states_on_two_streams(dtname):
    """Copy, inner product and Pauli apply between states on different non-blocking
    streams: the circuit queued on the source's stream (no host wait) must be
    complete when the other stream reads it."""
    import torch
    dt = DT[dtname]
    n = 18
    gates = W.random_layered(n, 30, seed=3)
    theta = None
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = Q.qs_state_alloc(n, dt, C_stream(sa))
    b = Q.qs_state_alloc(n, dt, C_stream(sb))
    c = Q.qs_state_alloc(n, dt, C_stream(sb))
    plan = Q.qs_plan_create(n, dt, gates, Q.make_opts(mode=Q.QS_MODE_PER_GATE))
    try:
        want = ref(n, gates, theta)
        Q.qs_plan_execute(plan, a, theta)          # queued on stream a only
        Q.qs_state_copy(b, a)                      # ordered on stream b
        out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
        Q.qs_state_copy_to_host(b, out)
        assert np.abs(out - want).max() <= TOL[dt]
        Q.qs_state_set_basis(a, 0)
        Q.qs_plan_execute(plan, a, theta)          # a again holds C|0>, queued on stream a
        ip = Q.qs_inner(b, a)                      # runs on stream b
        assert abs(ip - 1.0) <= (1e-10 if dt == Q.QS_C128 else 1e-4)
        coeff, xm, zm = np.array([1.0]), np.array([1], dtype=np.uint64), np.array([0], dtype=np.uint64)
        Q.qs_state_set_basis(a, 0)
        Q.qs_plan_execute(plan, a, theta)
        Q.qs_apply_pauli_sum(a, coeff, xm, zm, c)  # output c on stream b, written on stream a
        Q.qs_state_copy_to_host(c, out)
        assert np.abs(out - O.apply_pauli_sum(want, n, coeff, xm, zm)).max() <= TOL[dt]
    finally:
        Q.qs_plan_free(plan)
        for h in (a, b, c):
            Q.qs_state_free(h)


@pytest.mark.parametrize("dtname", ["c128", "c64"])
def test_one_plan_executed_on_two_streams(dtname):
    """One parametric plan run back to back on states with different streams and
    different parameters: the second execution rewrites the plan's gate table and
    theta rows only after the first has used them."""
    import torch
    dt = DT[dtname]
    n = 17
    gates, p = W.hea(n, 6)
    t1, t2 = W.thetas_uniform(p, 1), W.thetas_uniform(p, 2)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = Q.qs_state_alloc(n, dt, C_stream(sa))
    b = Q.qs_state_alloc(n, dt, C_stream(sb))
    plan = Q.qs_plan_create(n, dt, gates, Q.make_opts(fuse_k=2))
    try:
        Q.qs_plan_execute(plan, a, t1)
        Q.qs_plan_execute(plan, b, t2)
        for h, th in ((a, t1), (b, t2)):
            out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
            Q.qs_state_copy_to_host(h, out)
            assert np.abs(out - ref(n, gates, th)).max() <= TOL[dt]
    finally:
        Q.qs_plan_free(plan)
        Q.qs_state_free(a)
        Q.qs_state_free(b)


@pytest.mark.parametrize("dtname,n,opts", [("c128", 11, None), ("c64", 11, None),
                                            ("c128", 11, Q.make_opts(fuse_k=2)),
                                            ("c64", 13, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4,
                                                                    fuse_parametric=1))])
def test_one_shot_batched_apply(dtname, n, opts):
    """qs_apply_circuit_batched: plan, B states each with its own parameter row,
    free; every state equals the oracle with that row."""
    dt = DT[dtname]
    gates, p = W.hea(n, 3)
    B = 3
    theta = np.stack([W.thetas_uniform(p, 10 + b) for b in range(B)])
    hs = [Q.qs_state_alloc(n, dt) for _ in range(B)]
    try:
        for b, h in enumerate(hs):
            Q.qs_state_set_basis(h, b)
        Q.qs_apply_circuit_batched(hs, gates, theta, opts)
        for b, h in enumerate(hs):
            out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
            Q.qs_state_copy_to_host(h, out)
            assert np.abs(out - ref(n, gates, theta[b], basis=b)).max() <= TOL[dt]
    finally:
        for h in hs:
            Q.qs_state_free(h)


def C_stream(s):
    import ctypes
    return ctypes.c_void_p(s.cuda_stream)


BULK = [dict(fuse_k=1, tile_qubits=10, low_qubits=1), dict(fuse_k=2, tile_qubits=12, low_qubits=4),
        dict(fuse_k=3, tile_qubits=11, low_qubits=2), dict(fuse_k=5, tile_qubits=12, low_qubits=3),
        dict(paper_mode=1, tile_qubits=9, low_qubits=2)]


@pytest.mark.parametrize("dtname", ["c64", "c128"])
@pytest.mark.parametrize("n", [9, 12, 17])
def test_bulk_staged_tile_passes_match_oracle(dtname, n):
    """Tile passes whose tiles are moved by bulk copies into two shared-memory
    buffers (tile_staging=2; complex128 in FP64, the tiles the bulk path
    takes): gate mixes with controls above and below their targets, every
    fusion width, runs of 16 bytes to 256 bytes, states of one tile up to
    thousands of tiles per pass, against the oracle."""
    dt = DT[dtname]
    gates = W.random_gate_mix(n, 80, seed=n + 5) + W.random_layered(n, 4, seed=n)
    psi0 = W.random_state(n, n)
    want = ref(n, gates, psi0=psi0)
    for kw in BULK:
        kw = dict(kw, tile_qubits=min(kw["tile_qubits"], n))
        opts = Q.make_opts(tile_staging=2, c128_pairs=2, **kw)
        plan = Q.qs_plan_create(n, dt, gates, opts)
        try:
            info = Q.qs_plan_info_get(plan)
            assert info["bulk_tile_passes"] == info["passes"] > 0, kw
        finally:
            Q.qs_plan_free(plan)
        got = run(n, dt, gates, psi0=psi0, opts=opts)
        assert np.abs(got - want).max() <= TOL[dt], (kw, np.abs(got - want).max())


@pytest.mark.parametrize("dtname", ["c64", "c128"])
def test_bulk_staged_tile_passes_batched_with_parameters(dtname):
    """Batched execution (one launch per pass over all states, parametric
    blocks rebuilt per row) with bulk-staged tiles: every row against the
    oracle after a graph capture and a replay."""
    dt = DT[dtname]
    n, Bsz = 13, 6
    gates, p = W.hea(n, 3)
    thetas = np.stack([W.thetas_uniform(p, 60 + b) for b in range(Bsz)])
    opts = Q.make_opts(fuse_k=3, fuse_parametric=1, tile_staging=2, c128_pairs=2)
    plan = Q.qs_plan_create(n, dt, gates, opts)
    states = [Q.qs_state_alloc(n, dt) for _ in range(Bsz)]
    try:
        assert Q.qs_plan_info_get(plan)["bulk_tile_passes"] > 0
        for _ in range(2):
            for s in states:
                Q.qs_state_set_basis(s, 0)
            Q.qs_plan_execute_batched(plan, states, thetas)
        for b in range(Bsz):
            out = np.empty(1 << n, dtype=Q.NP_DTYPE[dt])
            Q.qs_state_copy_to_host(states[b], out)
            assert np.abs(out - ref(n, gates, thetas[b])).max() <= TOL[dt], b
    finally:
        for s in states:
            Q.qs_state_free(s)
        Q.qs_plan_free(plan)


def test_bulk_staged_tile_pass_wait_timeout_returns_error_and_recovers():
    """Failure detection for the bulk-staged tile pass: with a wait limit of 2
    immediate polls the first wait for a tile runs out, the CTAs let their
    copies land and return, and the execution reports QS_ERR_TIMEOUT; with the
    default limit the same plan then matches the oracle."""
    n = 16
    gates = W.random_layered(n, 4, seed=8)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(fuse_k=2, tile_staging=2))
    h = Q.qs_state_alloc(n, Q.QS_C64)
    try:
        assert Q.qs_plan_info_get(plan)["bulk_tile_passes"] > 0
        Q.qs_plan_set_wait_limit(plan, 2)
        Q.qs_state_set_basis(h, 0)
        with pytest.raises(Q.QsError) as e:
            Q.qs_plan_execute(plan, h)
        assert e.value.status == Q.QS_ERR_TIMEOUT
        Q.qs_plan_set_wait_limit(plan, 0)
        Q.qs_state_set_basis(h, 0)
        Q.qs_plan_execute(plan, h)
        out = np.empty(1 << n, dtype=np.complex64)
        Q.qs_state_copy_to_host(h, out)
    finally:
        Q.qs_state_free(h)
        Q.qs_plan_free(plan)
    assert np.abs(out - ref(n, gates)).max() <= 2e-5


@pytest.mark.parametrize("dtname,fuse_k", [("c64", 4), ("c64", 5), ("c128", 4)])
def test_tensor_core_narrower_contraction_widths(dtname, fuse_k):
    """Tensor-core plans whose contraction is narrower than the pass (4 or 5
    qubits in complex64, 4 in complex128; blocks padded with qubits they act
    on as the identity): layered random circuits over several tiles per CTA
    against the oracle, complex64 bar 2e-5, complex128 1e-12."""
    dt = DT[dtname]
    for n, depth in ((14, 8), (22, 6)):
        gates = W.random_layered(n, depth, seed=n + fuse_k)
        opts = Q.make_opts(mode=Q.QS_MODE_TENSOR, fuse_k=fuse_k, tc_min_gates=2 if dt == Q.QS_C64 else 0)
        plan = Q.qs_plan_create(n, dt, gates, opts)
        try:
            assert any(op["type"] == 3 for op in Q.qs_plan_ops(plan))
        finally:
            Q.qs_plan_free(plan)
        got = run(n, dt, gates, opts=opts)
        assert np.abs(got - ref(n, gates)).max() <= TOL[dt], (n, np.abs(got - ref(n, gates)).max())
