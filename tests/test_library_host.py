"""Host-side checks of the CUDA library: it builds, loads, exports every entry
point declared in include/qsim_gb300.h, validates arguments, refuses to run
without a GPU (no CPU fallback), and its planner (gate DAG + contraction +
tile passes, all host code) produces op sequences whose product equals the
oracle's brute-force unitary.
"""
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "qsim_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound():
    L = Q.lib()
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
        assert name in Q.exported_symbols(), name
    assert "sm_103a" in Q.qs_version()


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """The boundary is a C ABI: include/qsim_gb300.h compiles as strict C99
    (no C++ types in any signature), and a C program links against the library
    and calls an entry point that needs no device."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_abi.c"
    src.write_text('#include <stdio.h>\n#include "qsim_gb300.h"\n'
                   "int main(void) { qs_plan_opts o = {0}; qs_stream_info si = {0}; (void)o; (void)si;\n"
                   '  printf("%s\\n", qs_version()); return 0; }\n')
    lib = Q.lib()._name
    exe = tmp_path / "use_abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), lib, "-o", str(exe), "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    assert "sm_103a" in out


def test_no_gpu_means_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(Q.QsError) as e:
        Q.qs_state_alloc(4, Q.QS_C64)
    assert e.value.status == Q.QS_ERR_CUDA


@pytest.mark.parametrize("bad", [
    [W.Gate("h", (5,))],                         # qubit >= n
    [W.Gate("x", (1,), controls=(1,))],          # repeated qubit
    [W.Gate("swap", (0,))],                      # wrong target count
    [W.Gate("x", (0,), controls=(1, 2, 3))],     # too many controls
])
def test_invalid_gates_are_rejected_before_device_work(bad):
    with pytest.raises(Q.QsError) as e:
        Q.qs_plan_create(4, Q.QS_C64, bad, Q.make_opts())
    assert e.value.status == Q.QS_ERR_ARG


def test_theta_bounds_and_options_are_validated():
    with pytest.raises(Q.QsError):
        Q.qs_plan_create(10, Q.QS_C128, W.qft(10), Q.make_opts(fuse_k=6))   # CUDA-core blocks: k <= 5
    with pytest.raises(Q.QsError):
        Q.qs_plan_create(10, Q.QS_C64, W.qft(10), Q.make_opts(tile_qubits=15))
    for pairs in (-1, 3):   # complex128 arithmetic: 0 / 1 FP32 pairs (default), 2 FP64
        with pytest.raises(Q.QsError):
            Q.qs_plan_create(10, Q.QS_C128, W.qft(10), Q.make_opts(c128_pairs=pairs))
    for pairs in (0, 1, 2):
        Q.qs_plan_free(Q.qs_plan_create(10, Q.QS_C128, W.qft(10), Q.make_opts(c128_pairs=pairs)))


def test_gate_count_limit_is_checked_before_the_list_is_read():
    """A gate count above 2^30 (the planner's 32-bit gate indices) is an argument
    error raised before any gate is read: the one-gate array passed here is never
    read past its end."""
    import ctypes
    one = Q.pack_gates([W.Gate("h", (0,))])
    h = ctypes.c_void_p()
    for create in ("plan", "stream"):
        if create == "plan":
            st = Q.lib().qs_plan_create(4, Q.QS_C64, one, (1 << 30) + 1, None, ctypes.byref(h))
        else:
            st = Q.lib().qs_stream_plan(4, one, (1 << 30) + 1, 2, 1, None, None, None, 0, None)
        assert st == Q.QS_ERR_ARG
        assert "too many gates" in Q.lib().qs_last_error().decode()


# ------------------------------------------------------------- planner algebra

def apply_block(psi, n, qubits, M):
    """Applies a 2^k x 2^k matrix over `qubits` (local bit j = qubits[j])."""
    k = len(qubits)
    others = [q for q in range(n) if q not in qubits]
    base = np.zeros(1 << (n - k), dtype=np.int64)
    for j, q in enumerate(others):
        base |= ((np.arange(1 << (n - k)) >> j) & 1) << q
    offs = np.zeros(1 << k, dtype=np.int64)
    for j, q in enumerate(qubits):
        offs |= ((np.arange(1 << k) >> j) & 1) << q
    idx = base[:, None] | offs[None, :]
    out = psi.copy()
    out[idx] = psi[idx] @ M.T
    return out


def plan_unitary(n, gates, plan, theta=None):
    ops = Q.qs_plan_ops(plan)
    U = np.eye(1 << n, dtype=complex)
    for op in ops:
        if op["type"] == 0:
            G = O.unitary(n, [gates[op["gate"]]], theta)
        elif op["type"] in (1, 3):
            G = np.stack([apply_block(c, n, op["qubits"], op["matrix"]) for c in np.eye(1 << n, dtype=complex)],
                         axis=1)
        else:
            G = np.stack([apply_block(c, n, op["qubits"], np.diag(op["matrix"])) for c in np.eye(1 << n, dtype=complex)],
                         axis=1)
        U = G @ U
    return U, ops


@pytest.mark.parametrize("n,k,m,L,dt", [(6, 2, 4, 1, Q.QS_C128), (7, 3, 5, 2, Q.QS_C64), (7, 4, 6, 1, Q.QS_C64),
                                         (5, 5, 5, 1, Q.QS_C64), (3, 2, 3, 3, Q.QS_C128)])
def test_fused_plan_equals_brute_force(n, k, m, L, dt):
    for seed in range(3):
        gates = W.random_gate_mix(n, 50, seed=seed) + W.random_layered(n, 2, seed)
        plan = Q.qs_plan_create(n, dt, gates, Q.make_opts(fuse_k=k, tile_qubits=m, low_qubits=L))
        try:
            U, ops = plan_unitary(n, gates, plan)
            assert np.abs(U - O.unitary(n, gates)).max() < 1e-12
            used = sorted(op.get("gate", -1) for op in ops if op["type"] == 0)
            assert len(set(used)) == len(used)
            for op in ops:   # a block starts from a gate of up to 4 qubits, then grows to k
                assert len(op["qubits"]) <= (4 if op["type"] == 0 else max(k, 4))
            for ps in Q.qs_plan_passes(plan):
                assert min(m, n) <= len(ps["tile"]) <= 14   # wider only when one op needs it
                assert set(range(min(L, n))) <= set(ps["tile"])
                b, e = ps["ops"]
                for op in ops[b:e]:
                    assert set(op["qubits"]) <= set(ps["tile"])
        finally:
            Q.qs_plan_free(plan)


def test_parametric_gates_stay_separate_unless_asked():
    n = 5
    gates, p = W.hea(n, 2)
    theta = W.thetas_uniform(p, 0)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(fuse_k=3, tile_qubits=5, low_qubits=1))
    ops = Q.qs_plan_ops(plan)
    pg = {op["gate"] for op in ops if op["type"] == 0}
    assert all(i in pg for i, g in enumerate(gates) if g.param_index >= 0)
    U, _ = plan_unitary(n, gates, plan, theta)
    assert np.abs(U - O.unitary(n, gates, theta)).max() < 1e-12
    Q.qs_plan_free(plan)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(fuse_k=3, tile_qubits=5, low_qubits=1,
                                                             fuse_parametric=1))
    assert any(op["type"] != 0 for op in Q.qs_plan_ops(plan))
    Q.qs_plan_free(plan)


def test_paper_mode_compression_on_hea():
    """Section 3.4 merges only (k = 2): 1q (x) 1q, same-qubit products, same-(c, t) CU.
    The paper's HEA (RX, RY, RZ layers + CNOTs) compresses by tens of percent (Fig. 16)."""
    n = 12
    gates = []
    for layer in range(5):
        for kind in ("rx", "ry", "rz"):
            for q in range(n):
                gates.append(W.Gate(kind, (q,), angle=0.1 * (q + layer)))
        for q in range(layer % 2, n - 1, 2):
            gates.append(W.Gate("x", (q + 1,), controls=(q,)))
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(paper_mode=1, tile_qubits=10, low_qubits=4))
    info = Q.qs_plan_info_get(plan)
    ratio = (info["gates"] - info["blocks"]) / info["gates"]
    assert 0.3 < ratio < 0.95
    Q.qs_plan_free(plan)
    # the same merges on the circuit's first six qubits reproduce its unitary
    small = [g for g in gates if max(g.qubits) < 6]
    plan = Q.qs_plan_create(6, Q.QS_C128, small, Q.make_opts(paper_mode=1, tile_qubits=6, low_qubits=1))
    try:
        U, _ = plan_unitary(6, small, plan)
        assert np.abs(U - O.unitary(6, small)).max() < 1e-12
    finally:
        Q.qs_plan_free(plan)


def phase_diagonal(n, terms, theta):
    """prod_j exp(i alpha_j (-1)^popcount(mask_j & x)) over all x."""
    x = np.arange(1 << n, dtype=np.int64)
    ang = np.zeros(1 << n)
    for mask, pidx, a0, coef in terms:
        a = a0 + (coef * theta[pidx] if pidx >= 0 else 0.0)
        par = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            if (mask >> q) & 1:
                par ^= (x >> q) & 1
        ang += a * (1 - 2 * par)
    return np.exp(1j * ang)


def apply_plan_ops(psi, n, gates, plan, theta):
    cur = psi.copy()
    for op in Q.qs_plan_ops(plan):
        if op["type"] == 0:
            cur = O.apply_circuit(cur, n, [gates[op["gate"]]], theta)
        elif op["type"] == 2:
            cur = apply_block(cur, n, op["qubits"], np.diag(op["matrix"]))
        elif op["type"] == 4:
            cur = cur * phase_diagonal(n, op["terms"], theta)
        else:
            cur = apply_block(cur, n, op["qubits"], op["matrix"])
    return cur


@pytest.mark.parametrize("maker", ["qaoa", "zoo"])
def test_phase_runs_equal_their_gates(maker):
    """Runs of CNOTs, SWAPs and diagonal gates whose basis permutation is the
    identity become one diagonal phase op; its phase polynomial applied with
    numpy, with the other ops, reproduces the oracle's gate-by-gate state for
    random parameters. n = 14 > 12 puts masks on both sides of the kernel's
    lo / hi split (every term class occurs in the zoo)."""
    n = 14
    if maker == "qaoa":
        gates, p = W.qaoa(n, 3, W.random_regular_graph(n, 3, seed=1))
    else:
        gates, p = W.phase_run_circuit(n, 3, 30, seed=2)
    theta = W.thetas_uniform(max(p, 1), 3)
    psi = W.random_state(n, 4)
    want = O.apply_circuit(psi, n, gates, theta)
    for opts in (Q.make_opts(), Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=4),
                 Q.make_opts(phase_min_gates=4)):
        plan = Q.qs_plan_create(n, Q.QS_C128, gates, opts) if opts.mode != Q.QS_MODE_TENSOR else \
            Q.qs_plan_create(n, Q.QS_C64, gates, opts)
        try:
            ops = Q.qs_plan_ops(plan)
            runs = [op for op in ops if op["type"] == 4]
            assert len(runs) >= 3
            assert np.abs(apply_plan_ops(psi, n, gates, plan, theta) - want).max() < 1e-12
            if maker == "zoo":
                low = (1 << 12) - 1
                classes = {("low" if m & ~low == 0 else "mixed") if bin(m & low).count("1") >= 2 else
                           ("lin" if m & low else "high") for op in runs for m, *_ in op["terms"]}
                assert {"low", "lin", "high", "mixed"} <= classes, classes
        finally:
            Q.qs_plan_free(plan)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(phase_min_gates=-1))
    assert not any(op["type"] == 4 for op in Q.qs_plan_ops(plan))
    Q.qs_plan_free(plan)


def test_smgp_groups_and_launch_accounting():
    """Staggered multi-gate plans (Section 3.3): runs of uncontrolled one-target
    gates on distinct qubits become groups of S = 8, 4 or 2 (S targets plus
    lg S segment qubits must fit the register); each group costs S launches,
    the other gates one each."""
    n = 12
    gates = [W.Gate("h", (q,)) for q in range(n)] + [W.Gate("x", (1,), (0,))] + \
        [W.Gate("rz", (q,), angle=0.1) for q in (3, 4, 3)]
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_SMGP))
    info = Q.qs_plan_info_get(plan)
    # 12 H -> groups of 8 and 4; CNOT single; RZ(3), RZ(4) -> group of 2; RZ(3) single
    assert info["launches"] == 8 + 4 + 1 + 2 + 1
    assert len(Q.qs_plan_ops(plan)) == len(gates)     # introspection as a per-gate plan
    Q.qs_plan_free(plan)
    small = Q.qs_plan_create(5, Q.QS_C64, [W.Gate("h", (q,)) for q in range(5)], Q.make_opts(mode=Q.QS_MODE_SMGP))
    assert Q.qs_plan_info_get(small)["launches"] == 2 + 2 + 1    # S + lg S <= 5 caps groups at 2
    Q.qs_plan_free(small)


@pytest.mark.parametrize("l,h", [(8, 2), (9, 1), (6, 3)])
def test_stream_passes_reorder_only_commuting_gates(l, h):
    """Host-resident execution (Section 3.2): streamed passes come from the
    tile-pass scheduler with the l low qubits always present and at most h
    batch-index qubits per pass. Every gate appears once; applying the passes'
    gates in their order reproduces the circuit (oracle, n = 11); random layers
    at depth 6 need several passes, and a gate needing more than h batch qubits
    is an argument error."""
    n = 11
    gates = W.random_layered(n, 6, seed=l) + W.random_gate_mix(n, 40, seed=h)
    gates = [g for g in gates if sum(q >= l for q in g.qubits) <= h]
    passes = Q.qs_stream_plan(n, gates, l, h)
    order = [g for _, gs in passes for g in gs]
    assert sorted(order) == list(range(len(gates)))
    assert all(bin(m).count("1") <= h and m & ((1 << l) - 1) == 0 for m, _ in passes)
    psi = W.random_state(n, 5)
    want = O.apply_circuit(psi, n, gates)
    got = O.apply_circuit(psi, n, [gates[i] for i in order])
    assert np.abs(got - want).max() < 1e-12
    assert len(passes) > 1
    with pytest.raises(Q.QsError):
        Q.qs_stream_plan(n, [W.Gate("x", (10,), (8, 9))], 8, 2)
    assert len(Q.qs_stream_plan(n, gates, l, n - l)) == 1
    assert len(Q.qs_stream_plan(n, gates, n, 0)) == 1          # one batch: the whole state
    with pytest.raises(Q.QsError):
        Q.qs_stream_plan(n, gates, 0, 2)                       # batches of at least one qubit


def test_per_gate_sweep_accounting():
    n = 8
    gates = [W.Gate("h", (0,)), W.Gate("x", (1,), controls=(0,)), W.Gate("z", (2,), controls=(1,)),
             W.Gate("rz", (3,), angle=0.3), W.Gate("swap", (4, 5)), W.Gate("p", (6,), angle=0.2)]
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, None)
    info = Q.qs_plan_info_get(plan)
    # dense 1 + CNOT 1/2 + CZ 1/4 + RZ 1 + SWAP 1/2 + P 1/2
    assert abs(info["per_gate_sweeps"] - (1 + 0.5 + 0.25 + 1 + 0.5 + 0.5)) < 1e-12
    assert info["launches"] == len(gates)
    Q.qs_plan_free(plan)


def _padded_qubits(U, k):
    """Local bits on which a 2^k x 2^k block acts as the identity."""
    out = []
    for b in range(k):
        M = U.reshape([2] * (2 * k))
        # axes: row bits k-1..0 then column bits k-1..0 (bit b of an index is axis k-1-b)
        r, c = k - 1 - b, 2 * k - 1 - b
        sub = np.moveaxis(M, (r, c), (0, 1))
        if np.allclose(sub[0, 1], 0) and np.allclose(sub[1, 0], 0) and np.allclose(sub[0, 0], sub[1, 1]):
            out.append(b)
    return out


@pytest.mark.parametrize("fuse_k", [0, 4, 5])
def test_tensor_mode_plan_matches_oracle_on_a_state(fuse_k):
    """Tensor-core plans (blocks of the 6-, 5- or 4-qubit contraction padded to
    6 qubits, tile passes in between) reproduce the circuit: ops applied with
    numpy to a random state equal the oracle's gate-by-gate result; with a
    narrower contraction the blocks act as the identity on their padding."""
    n = 14
    gates = W.random_layered(n, 8, seed=3)
    plan = Q.qs_plan_create(n, Q.QS_C64, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, fuse_k=fuse_k))
    try:
        ops = Q.qs_plan_ops(plan)
        assert any(op["type"] == 3 for op in ops)
        psi = W.random_state(n, 1)
        cur = psi.copy()
        for op in ops:
            if op["type"] == 0:
                cur = O.apply_circuit(cur, n, [gates[op["gate"]]])
            elif op["type"] == 2:
                cur = apply_block(cur, n, op["qubits"], np.diag(op["matrix"]))
            else:
                if op["type"] == 3:
                    assert len(op["qubits"]) == 6
                    if fuse_k:
                        assert len(_padded_qubits(np.asarray(op["matrix"]).reshape(64, 64), 6)) >= 6 - fuse_k
                cur = apply_block(cur, n, op["qubits"], op["matrix"])
        assert np.abs(cur - O.apply_circuit(psi, n, gates)).max() < 1e-12
        for ps in Q.qs_plan_passes(plan):
            b, e = ps["ops"]
            if any(op["type"] == 3 for op in ops[b:e]):
                assert e - b == 1 and len(ps["tile"]) == 13
    finally:
        Q.qs_plan_free(plan)


@pytest.mark.parametrize("tc_min,fuse_k", [(0, 0), (2, 0), (5, 0), (0, 4)])
def test_complex128_tensor_plan_matches_oracle_on_a_state(tc_min, fuse_k):
    """Complex128 tensor-core plans: 5-qubit (or, with fuse_k = 4, 4-qubit)
    contraction, blocks of >= tc_min gates (0: every block) padded to 5 qubits
    on 12-qubit tiles, the rest as CUDA-core ops; applied with numpy they
    reproduce the oracle's state. The complex64 precision options are refused."""
    n = 13
    gates = W.random_layered(n, 6, seed=4)
    plan = Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_min_gates=tc_min,
                                                             fuse_k=fuse_k))
    try:
        ops = Q.qs_plan_ops(plan)
        tc = [op for op in ops if op["type"] == 3]
        assert tc
        if tc_min == 0:
            assert all(op["type"] in (3, 4) for op in ops)
        psi = W.random_state(n, 2)
        cur = psi.copy()
        for op in ops:
            if op["type"] == 0:
                cur = O.apply_circuit(cur, n, [gates[op["gate"]]])
            elif op["type"] == 2:
                cur = apply_block(cur, n, op["qubits"], np.diag(op["matrix"]))
            else:
                if op["type"] == 3:
                    assert len(op["qubits"]) == 5
                    if fuse_k:
                        assert len(_padded_qubits(np.asarray(op["matrix"]).reshape(32, 32), 5)) >= 5 - fuse_k
                cur = apply_block(cur, n, op["qubits"], op["matrix"])
        assert np.abs(cur - O.apply_circuit(psi, n, gates)).max() < 1e-12
        for ps in Q.qs_plan_passes(plan):
            b, e = ps["ops"]
            if any(op["type"] == 3 for op in ops[b:e]):
                assert e - b == 1 and len(ps["tile"]) == 12
    finally:
        Q.qs_plan_free(plan)
    with pytest.raises(Q.QsError) as e:
        Q.qs_plan_create(n, Q.QS_C128, gates, Q.make_opts(mode=Q.QS_MODE_TENSOR, tc_precision=4))
    assert e.value.status == Q.QS_ERR_ARG


def test_planner_fuzz_ops_reproduce_the_circuit():
    """Seeded sweep over circuits (random mixes with controls, layers, QFT, QAOA,
    diagonal runs, HEA with parameters) and plan options (contraction width,
    tile width, low qubits, paper mode, phase runs on or off, SMGP): in every
    plan each gate is applied exactly once and the ops applied with numpy, in
    plan order, reproduce the oracle's gate-by-gate state."""
    rng = np.random.default_rng(2509)
    seen = set()
    for case in range(48):
        kind = ("mix", "layered", "qft", "qaoa", "phase", "hea")[case % 6]
        # phase runs need a 4096-amplitude chunk (n >= 12)
        n = 12 + case % 2 if kind in ("qaoa", "phase") else int(rng.integers(3, 10))
        theta = None
        if kind == "mix":
            gates = W.random_gate_mix(n, 40, seed=case)
        elif kind == "layered":
            gates = W.random_layered(n, 4, seed=case, entangler=("cnot", "cz")[case % 2])
        elif kind == "qft":
            gates = W.qft(n)
        elif kind == "qaoa":
            gates, p = W.qaoa(n, 2, [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.4])
            theta = W.thetas_uniform(max(p, 1), case)
        elif kind == "phase":
            gates, p = W.phase_run_circuit(n, 2, 12, seed=case, max_weight=min(4, n))
            theta = W.thetas_uniform(max(p, 1), case)
        else:
            gates, p = W.hea(n, 2)
            theta = W.thetas_uniform(p, case)
        L = int(rng.integers(1, min(3, n - 1) + 1))
        k = int(rng.integers(1, min(5, n - L) + 1))
        m = int(rng.integers(L + k, n + 1))          # a tile holds the low qubits plus a block
        pick = (case // 6) % 4                    # every circuit kind meets every option set
        dt = (Q.QS_C64, Q.QS_C128)[case % 2]       # the cost rule differs: more dense blocks in complex64
        if pick == 0:
            opts = Q.make_opts(fuse_k=k, tile_qubits=m, low_qubits=L, phase_min_gates=4)
        elif pick == 1:
            opts = Q.make_opts(fuse_k=k, tile_qubits=m, low_qubits=L, phase_min_gates=-1)
        elif pick == 2:
            opts = Q.make_opts(paper_mode=1, fuse_k=k, tile_qubits=m, low_qubits=L)
        else:
            opts = Q.make_opts(mode=Q.QS_MODE_SMGP)
        plan = Q.qs_plan_create(n, dt, gates, opts)
        try:
            ops = Q.qs_plan_ops(plan)
            seen.update(op["type"] for op in ops)
            per_gate = [op["gate"] for op in ops if op["type"] == 0]
            assert len(per_gate) == len(set(per_gate)), (case, kind)
            psi = W.random_state(n, case)
            got = apply_plan_ops(psi, n, gates, plan, theta)
            want = O.apply_circuit(psi, n, gates, theta)
            assert np.abs(got - want).max() < 1e-12, (case, kind, n, pick)
        finally:
            Q.qs_plan_free(plan)
    assert seen == {0, 1, 2, 4}, seen     # per-gate, dense block, diagonal block, phase run


def test_tuning_cache_put_lookup_save_load(tmp_path):
    """The autotuner's cache across processes: an entry put for a circuit is
    found again, survives a save / clear / load round trip with its options and
    time, ignores fields a gate's kind does not use, and a malformed file is
    refused without touching the cache."""
    import dataclasses
    n = 12
    gates, p = W.hea(n, 2)
    Q.qs_tune_cache_clear()
    assert Q.qs_tune_cache_lookup(n, Q.QS_C64, gates) is None
    opts = Q.make_opts(fuse_k=3, tile_qubits=11, low_qubits=4, phase_min_gates=-1)
    Q.qs_tune_cache_put(n, Q.QS_C64, gates, opts, 1.25)
    hit = Q.qs_tune_cache_lookup(n, Q.QS_C64, gates)
    assert hit is not None and Q.opts_dict(hit[0]) == Q.opts_dict(opts) and hit[1] == 1.25
    assert Q.qs_tune_cache_lookup(n, Q.QS_C128, gates) is None              # the dtype is part of the key
    assert Q.qs_tune_cache_lookup(n, Q.QS_C64, gates[:-1]) is None          # and the gate list
    moved = [dataclasses.replace(gates[0], angle=gates[0].angle + 0.5)] + gates[1:]
    assert Q.qs_tune_cache_lookup(n, Q.QS_C64, moved) is None               # and a rotation's angle
    # unused fields (a second target slot, the matrix of a non-matrix gate) do not change the key
    arr = Q.pack_gates(gates)
    for k in range(len(gates)):
        if arr[k].nq == 1:
            arr[k].q[1] = 7
        arr[k].ctrl[1] = 5 if arr[k].nctrl < 2 else arr[k].ctrl[1]
        if arr[k].nctrl == 0:
            arr[k].ctrl[0] = 4
        if arr[k].kind not in (Q.KIND["rx"], Q.KIND["ry"], Q.KIND["rz"], Q.KIND["p"]):
            arr[k].param, arr[k].param_index, arr[k].scale = 9.0, 3, 2.0
        arr[k].mat[0] = 3.0
    import ctypes
    found = ctypes.c_int()
    assert Q.lib().qs_tune_cache_lookup(n, Q.QS_C64, arr, len(gates), None, None, ctypes.byref(found)) == Q.QS_OK
    assert found.value == 1
    path = str(tmp_path / "tune.txt")
    assert Q.qs_tune_cache_save(path) == 1
    Q.qs_tune_cache_clear()
    assert Q.qs_tune_cache_lookup(n, Q.QS_C64, gates) is None
    assert Q.qs_tune_cache_load(path) == 1
    hit = Q.qs_tune_cache_lookup(n, Q.QS_C64, gates)
    assert hit is not None and Q.opts_dict(hit[0]) == Q.opts_dict(opts) and hit[1] == 1.25
    text = open(path).read().splitlines()
    assert text[0] == "qsgb300-tune 1" and len(text) == 2
    for bad in (["qsgb300-tune 1", text[1] + " 9"], ["qsgb300-tune 1", "12 0 1"], ["not a cache", text[1]],
                ["qsgb300-tune 1", text[1].replace("12 0 ", "99 0 ", 1)]):
        (tmp_path / "bad.txt").write_text("\n".join(bad) + "\n")
        Q.qs_tune_cache_clear()
        with pytest.raises(Q.QsError) as e:
            Q.qs_tune_cache_load(str(tmp_path / "bad.txt"))
        assert e.value.status == Q.QS_ERR_ARG
        assert Q.qs_tune_cache_lookup(n, Q.QS_C64, gates) is None
    with pytest.raises(Q.QsError):      # options that cannot plan the circuit are refused
        Q.qs_tune_cache_put(n, Q.QS_C64, gates, Q.make_opts(fuse_k=6), 1.0)
    Q.qs_tune_cache_clear()


def test_product_and_oracle_share_no_code():
    """The CUDA library and its binding never import, include or link the oracle,
    and the oracle uses nothing of the library: only the seeded input generators
    (workloads.py, no simulator arithmetic) serve both sides."""
    import glob
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2509_04955_gb300")
    product = glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*"))
    for f in product:
        if f.endswith("workloads.py") or os.path.isdir(f) or f.endswith((".o", ".so")):
            continue
        text = open(f, errors="replace").read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
        assert not re.search(r'#include\s+[<"][^>"]*oracle', text), f
    for f in glob.glob(os.path.join(root, "oracle", "*")):
        if os.path.isdir(f) or f.endswith((".o", ".so")):
            continue
        text = open(f, errors="replace").read()
        assert "qsim_gb300" not in text and "csrc" not in text, f
        assert not re.search(r"^\s*(import|from)\s+paper_2509_04955_gb300(?!\.workloads)", text, re.M), f


def test_bulk_tile_staging_where_runs_and_buffers_allow():
    """tile_staging=2 stages tile passes by bulk copies when a run of
    2^low_qubits amplitudes is at least 16 bytes and two tiles fit in shared
    memory (low_qubits >= 1, so a complex64 run is at least 16 bytes and only
    the buffer size can rule a complex64 or FP64 tile out); FP32-pair tiles
    keep the vector path."""
    gates = W.random_layered(16, 6, seed=3)
    def bulk(dt, **kw):
        plan = Q.qs_plan_create(16, dt, gates, Q.make_opts(tile_staging=2, **kw))
        try:
            info = Q.qs_plan_info_get(plan)
            return info["bulk_tile_passes"], info["passes"]
        finally:
            Q.qs_plan_free(plan)
    b, n = bulk(Q.QS_C64, fuse_k=2, tile_qubits=12, low_qubits=4)
    assert b == n > 0
    b, n = bulk(Q.QS_C128, fuse_k=2, tile_qubits=11, low_qubits=3, c128_pairs=2)
    assert b == n > 0
    assert bulk(Q.QS_C128, fuse_k=2, tile_qubits=11, low_qubits=3)[0] == 0       # FP32 pairs
    b, n = bulk(Q.QS_C64, fuse_k=1, tile_qubits=10, low_qubits=1)               # 16-byte runs
    assert b == n > 0
    assert bulk(Q.QS_C128, fuse_k=2, tile_qubits=13, low_qubits=4, c128_pairs=2)[0] == 0   # 2 x 128 KiB
    plan = Q.qs_plan_create(16, Q.QS_C64, gates, Q.make_opts(fuse_k=2))
    assert Q.qs_plan_info_get(plan)["bulk_tile_passes"] == 0                    # default: vector path
    Q.qs_plan_free(plan)
    with pytest.raises(Q.QsError):
        Q.qs_plan_create(16, Q.QS_C64, gates, Q.make_opts(tile_staging=3))
