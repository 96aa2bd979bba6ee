"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine (scipy's matrix exponential, numpy's Kronecker product and inverse
FFT), a closed form (GHZ, QFT, single-Pauli values, Pauli-exponential), an
invariant (norm, circuit times inverse), the paper's printed index patterns
(Eq. 6, Eq. 7 fixtures under tests/golden/) or an independent method
(parameter shift and finite differences against the adjoint gradient).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2509_04955_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]])
Z = np.diag([1.0 + 0j, -1.0])
I2 = np.eye(2, dtype=complex)


def G(kind, targets, controls=(), angle=0.0, **kw):
    return W.Gate(kind, tuple(targets), tuple(controls), angle=angle, **kw)


# ---------------------------------------------------------------- gate matrices

@pytest.mark.parametrize("kind,P", [("rx", X), ("ry", Y), ("rz", Z)])
def test_rotations_are_matrix_exponentials(kind, P):
    for a in np.linspace(-3.0, 3.0, 7):
        ref = scipy.linalg.expm(-0.5j * a * P)
        assert np.allclose(O.gate_matrix(G(kind, (0,), angle=a)), ref, atol=1e-14)


def test_fixed_gate_identities():
    m = lambda k, a=0.0: O.gate_matrix(G(k, (0,), angle=a))
    assert np.allclose(m("h"), (X + Z) / math.sqrt(2), atol=1e-15)
    assert np.allclose(m("x"), X) and np.allclose(m("y"), Y) and np.allclose(m("z"), Z)
    assert np.allclose(m("s") @ m("s"), Z)
    assert np.allclose(m("t") @ m("t"), m("s"))
    assert np.allclose(m("s") @ m("sdg"), I2) and np.allclose(m("t") @ m("tdg"), I2)
    assert np.allclose(m("p", math.pi / 2), m("s"))
    assert np.allclose(m("p", 0.3), scipy.linalg.expm(1j * 0.3 * np.diag([0.0, 1.0])))


@pytest.mark.parametrize("kind,P", [("rx", X), ("ry", Y), ("rz", Z)])
def test_rotation_derivatives(kind, P):
    a = 0.731
    d = O.gate_dmatrix(G(kind, (0,), angle=a))
    assert np.allclose(d, -0.5j * P @ scipy.linalg.expm(-0.5j * a * P), atol=1e-14)
    d = O.gate_dmatrix(G("p", (0,), angle=a))
    assert np.allclose(d, np.diag([0, 1j * np.exp(1j * a)]), atol=1e-14)


# ---------------------------------------------------------------- qubit order

def test_qubit_order_on_basis_states():
    n = 4
    for q in range(n):
        out = O.apply_circuit(O.basis(n, 0), n, [G("x", (q,))])
        assert np.argmax(np.abs(out)) == 1 << q
    # CNOT control 1 target 3 on |0010> -> |1010>
    out = O.apply_circuit(O.basis(n, 0b0010), n, [G("x", (3,), (1,))])
    assert abs(out[0b1010] - 1) < 1e-15
    # control below and above the target
    out = O.apply_circuit(O.basis(n, 0b1000), n, [G("x", (0,), (3,))])
    assert abs(out[0b1001] - 1) < 1e-15
    out = O.apply_circuit(O.basis(n, 0b0001), n, [G("x", (3,), (0,))])
    assert abs(out[0b1001] - 1) < 1e-15
    # control clear: nothing happens
    out = O.apply_circuit(O.basis(n, 0b0100), n, [G("x", (0,), (1,))])
    assert abs(out[0b0100] - 1) < 1e-15
    out = O.apply_circuit(O.basis(n, 0b0010), n, [G("swap", (1, 2))])
    assert abs(out[0b0100] - 1) < 1e-15


def test_eq6_quad_order_fixture():
    """u2 on (t1, t2): local index = 2*bit(t2) + bit(t1) (Eq. 6, golden file)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "eq6_quad_order.txt"), dtype=int)
    n, t1, t2 = 5, 1, 3
    for r in range(4):
        M = np.zeros((4, 4), dtype=complex)
        M[r, 0] = 1.0           # maps local basis 0 to local basis r
        M[0, r] = 1.0
        for j in range(1, 4):
            if j != r:
                M[j, j] = 1.0
        out = O.apply_circuit(O.basis(n, 0), n, [G("u2", (t1, t2), matrix=tuple(M.reshape(-1)))])
        _, b2, b1 = rows[r]
        assert abs(out[(b2 << t2) | (b1 << t1)] - 1) < 1e-15


def test_eq7_kronecker_fixture():
    """Two one-qubit gates on t1 < t2: the circuit's unitary is M2 (x) M1 with
    the entry pattern printed in Eq. 7 (golden file)."""
    rng = np.random.default_rng(5)
    M1, M2 = W.random_unitary(2, rng), W.random_unitary(2, rng)
    U = O.unitary(2, [G("u1", (0,), matrix=tuple(M1.reshape(-1))),
                      G("u1", (1,), matrix=tuple(M2.reshape(-1)))])
    rows = np.loadtxt(os.path.join(GOLDEN, "eq7_kron_pattern.txt"), dtype=int)
    assert len(rows) == 16
    for r, c, a, b, cc, d in rows:
        assert abs(U[r, c] - M1[a, b] * M2[cc, d]) < 1e-15


# ---------------------------------------------------------------- brute force

def test_brute_force_matches_numpy_kron_for_single_gates():
    """Eq. 2 written with numpy's kron: qubit q sits n-q-1 factors from the left."""
    n = 3
    rng = np.random.default_rng(0)
    for q in range(n):
        U1 = W.random_unitary(2, rng)
        ref = np.kron(np.kron(np.eye(1 << (n - q - 1)), U1), np.eye(1 << q))
        got = O.unitary(n, [G("u1", (q,), matrix=tuple(U1.reshape(-1)))])
        assert np.allclose(got, ref, atol=1e-14)
    # controlled U: |0><0| (x) I + |1><1| (x) U, control 2 target 0
    U1 = W.random_unitary(2, rng)
    P0, P1 = np.diag([1.0, 0]), np.diag([0, 1.0])
    ref = np.kron(np.kron(P0, I2), I2) + np.kron(np.kron(P1, I2), U1)
    got = O.unitary(n, [G("u1", (0,), (2,), matrix=tuple(U1.reshape(-1)))])
    assert np.allclose(got, ref, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_per_gate_matches_brute_force(n):
    gates = W.random_gate_mix(n, 40, seed=100 + n)
    U = O.unitary(n, gates)
    for seed in range(2):
        psi = W.random_state(n, seed)
        assert np.abs(O.apply_circuit(psi, n, gates) - U @ psi).max() < 1e-13
    assert np.abs(U.conj().T @ U - np.eye(1 << n)).max() < 1e-12


def test_per_gate_matches_brute_force_n8_random_layers():
    n = 8
    gates = W.random_layered(n, 3, seed=3)
    psi = W.random_state(n, 9)
    assert np.abs(O.apply_circuit(psi, n, gates) - O.unitary(n, gates) @ psi).max() < 1e-13


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz(n):
    gates = [G("h", (0,))] + [G("x", (q,), (q - 1,)) for q in range(1, n)]
    out = O.apply_circuit(O.basis(n, 0), n, gates)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.abs(out - ref).max() < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6, 10])
def test_qft_closed_form(n):
    x = W.random_basis_index(n, 11 + n)
    out = O.apply_circuit(O.basis(n, x), n, W.qft(n))
    y = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.abs(out - ref).max() < 1e-13


def test_qft_is_scaled_inverse_fft():
    n = 8
    psi = W.random_state(n, 4)
    out = O.apply_circuit(psi, n, W.qft(n))
    assert np.abs(out - np.fft.ifft(psi) * math.sqrt(1 << n)).max() < 1e-13


@pytest.mark.parametrize("maker", ["random", "qft", "hea", "ucc", "mix"])
def test_circuit_times_inverse_is_identity_and_norm(maker):
    n = 9
    theta = None
    if maker == "random":
        gates = W.random_layered(n, 6, 1)
    elif maker == "qft":
        gates = W.qft(n)
    elif maker == "hea":
        gates, p = W.hea(n, 3)
        theta = W.thetas_uniform(p, 2)
    elif maker == "ucc":
        gates, _ = W.ucc(n, 12, 3)
        theta = W.thetas_normal(12, 4)
    else:
        gates = W.random_gate_mix(n, 60, 5)
    psi = W.random_state(n, 7)
    out = O.apply_circuit(psi, n, gates, theta)
    assert abs(O.norm2(out, n) - 1) < 1e-13
    back = O.apply_circuit(out, n, W.inverse_circuit(gates, theta))
    assert np.abs(back - psi).max() < 1e-13


def test_qaoa_circuit_equals_matrix_exponentials():
    """The QAOA gate list applied by the oracle equals the textbook unitary
    prod_l exp(-i beta_l B) exp(-i gamma_l C_ZZ) H^n |0>, with C_ZZ = sum_edges
    Z_u Z_v and B = sum_q X_q built as explicit 2^n x 2^n matrices."""
    n, layers = 6, 2
    edges = W.random_regular_graph(n, 3, seed=5)
    assert len(edges) == 9 and all(sum(1 for e in edges if q in e) == 3 for q in range(n))
    gates, p = W.qaoa(n, layers, edges)
    theta = np.array([0.37, -0.81, 1.13, 0.29])
    psi = O.apply_circuit(O.basis(n, 0), n, gates, theta)
    I2, X, Z = np.eye(2), np.array([[0, 1], [1, 0]]), np.diag([1.0, -1.0])

    def on(q, m):   # qubit q = bit q of the index: the rightmost Kronecker factor is qubit 0
        out = np.eye(1)
        for k in reversed(range(n)):
            out = np.kron(out, m if k == q else I2)
        return out
    czz = sum(on(u, Z) @ on(v, Z) for u, v in edges)
    bx = sum(on(q, X) for q in range(n))
    want = np.full(1 << n, 2 ** (-n / 2), dtype=complex)
    for layer in range(layers):
        want = scipy.linalg.expm(-1j * theta[2 * layer] * czz) @ want
        want = scipy.linalg.expm(-1j * theta[2 * layer + 1] * bx) @ want
    assert np.abs(psi - want).max() < 1e-12
    # MaxCut value of a basis state = number of cut edges
    H = W.maxcut_hamiltonian(edges)
    for x in (0, 5, 42, 63):
        cut = sum(((x >> u) & 1) != ((x >> v) & 1) for u, v in edges)
        assert abs(O.expval(O.basis(n, x), n, *H).real - cut) < 1e-12


def test_qaoa_p1_expected_cut_closed_form():
    """Depth-1 QAOA on random 3- and 4-regular graphs (some with triangles):
    the oracle's <C> equals the published p = 1 formula for every edge sum.
    This pins the formula the full-size GPU test relies on."""
    from closed_forms import qaoa_p1_maxcut
    triangles = 0
    for n, d, seed in ((8, 3, 0), (8, 3, 1), (10, 3, 4), (9, 4, 2), (10, 4, 5)):
        edges = W.random_regular_graph(n, d, seed)
        nb = [{v for e in edges for v in e if q in e and v != q} for q in range(n)]
        triangles += sum(len(nb[u] & nb[v]) for u, v in edges)
        gates, p = W.qaoa(n, 1, edges)
        H = W.maxcut_hamiltonian(edges)
        for th in ([0.37, -0.81], [1.1, 0.3], [-0.6, 1.4]):
            psi = O.apply_circuit(O.basis(n, 0), n, gates, np.array(th))
            assert abs(O.expval(psi, n, *H).real - qaoa_p1_maxcut(n, edges, *th)) < 1e-12
    assert triangles > 0


def test_pauli_exponential_closed_form():
    """exp(-i t P) psi = cos t psi - i sin t P psi for every letter mix."""
    n = 6
    rng = np.random.default_rng(1)
    for trial in range(8):
        w = int(rng.integers(1, n + 1))
        support = [int(q) for q in rng.choice(n, size=w, replace=False)]
        letters = "".join("XYZ"[int(rng.integers(0, 3))] for _ in range(w))
        t = float(rng.normal())
        gates = W.pauli_exponential(support, letters, 0)
        psi = W.random_state(n, trial)
        out = O.apply_circuit(psi, n, gates, np.array([t]))
        x, z = W.pauli_string_masks(n, support, letters)
        Ppsi = O.apply_pauli_sum(psi, n, [1.0], [x], [z])
        assert np.abs(out - (math.cos(t) * psi - 1j * math.sin(t) * Ppsi)).max() < 1e-13


# ---------------------------------------------------------------- Pauli sums

def pauli_matrix(n, x, z):
    letters = {(0, 0): I2, (1, 0): X, (1, 1): Y, (0, 1): Z}
    M = np.ones((1, 1), dtype=complex)
    for q in range(n - 1, -1, -1):
        M = np.kron(M, letters[((x >> q) & 1, (z >> q) & 1)])
    return M


def test_single_pauli_on_basis_states():
    n = 5
    for xb in [0, 3, 17, 31]:
        psi = O.basis(n, xb)
        for q in range(n):
            assert abs(O.expval(psi, n, [1.0], [0], [1 << q]) - (-1) ** ((xb >> q) & 1)) < 1e-15
            assert abs(O.expval(psi, n, [1.0], [1 << q], [0])) < 1e-15
            assert abs(O.expval(psi, n, [1.0], [1 << q], [1 << q])) < 1e-15
    assert abs(O.expval(O.basis(n, 0), n, np.ones(n), np.zeros(n, np.uint64),
                        [1 << q for q in range(n)]) - n) < 1e-14
    # Y eigenstate (|0> + i|1>)/sqrt2 has <Y> = +1
    psi = np.array([1, 1j]) / math.sqrt(2)
    assert abs(O.expval(psi, 1, [1.0], [1], [1]) - 1) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6])
def test_expval_and_apply_match_matrices(n):
    coeff, xm, zm = W.random_pauli_sum(n, 12, seed=n)
    H = sum(c * pauli_matrix(n, int(x), int(z)) for c, x, z in zip(coeff, xm, zm))
    assert np.abs(H - H.conj().T).max() < 1e-14
    psi = W.random_state(n, 3)
    e = O.expval(psi, n, coeff, xm, zm)
    assert abs(e - psi.conj() @ H @ psi) < 1e-13
    assert abs(e.imag) < 1e-13 * np.abs(coeff).sum()
    assert np.abs(O.apply_pauli_sum(psi, n, coeff, xm, zm) - H @ psi).max() < 1e-13


# ---------------------------------------------------------------- gradients

def test_single_rotation_gradient_closed_form():
    # <Z> after RY(t)|0> = cos t
    for t in [-2.0, 0.3, 1.1]:
        e, g = O.adjoint_grad(O.basis(1, 0), 1, [G("ry", (0,), param_index=0)], [t], [1.0], [0], [1])
        assert abs(e - math.cos(t)) < 1e-15 and abs(g[0] + math.sin(t)) < 1e-15


def _param_shift(psi0, n, gates, theta, H):
    """Two-term shift rule per parameter; the shift that suits each use is
    pi/2 / scale (rotation angle = scale * theta)."""
    scales = {}
    for g in gates:
        if g.param_index >= 0:
            scales.setdefault(g.param_index, set()).add(g.scale)
    grad = np.zeros(len(theta))
    for p in range(len(theta)):
        # every use of a parameter shifted separately (generalised product rule)
        uses = [k for k, g in enumerate(gates) if g.param_index == p]
        for k in uses:
            s = gates[k].scale
            for sign in (+1, -1):
                gg = list(gates)
                gg[k] = W.Gate(gates[k].kind, gates[k].targets, gates[k].controls,
                               angle=gates[k].angle + sign * math.pi / 2, param_index=p, scale=s)
                grad[p] += sign * 0.5 * s * O.expval_of_circuit(psi0, n, gg, theta, *H)
    return grad


def _finite_diff(psi0, n, gates, theta, H, h=1e-4):
    grad = np.zeros(len(theta))
    for p in range(len(theta)):
        tp, tm = np.array(theta, float), np.array(theta, float)
        tp[p] += h
        tm[p] -= h
        grad[p] = (O.expval_of_circuit(psi0, n, gates, tp, *H) - O.expval_of_circuit(psi0, n, gates, tm, *H)) / (2 * h)
    return grad


@pytest.mark.parametrize("maker", ["hea", "ucc"])
def test_adjoint_equals_parameter_shift_and_fd(maker):
    n = 5
    if maker == "hea":
        gates, p = W.hea(n, 2)
        theta = W.thetas_uniform(p, 3)
    else:
        gates, _ = W.ucc(n, 6, 8, wmin=2, wmax=4)
        p = 6
        theta = W.thetas_normal(p, 9, sigma=0.5)
    H = W.random_pauli_sum(n, 10, 12)
    psi0 = O.basis(n, 0)
    e, g = O.adjoint_grad(psi0, n, gates, theta, *H)
    assert abs(e - O.expval_of_circuit(psi0, n, gates, theta, *H)) < 1e-13
    ps = _param_shift(psi0, n, gates, theta, H)
    fd = _finite_diff(psi0, n, gates, theta, H)
    assert np.abs(g - ps).max() < 1e-12
    assert np.abs(g - fd).max() < 1e-7


def test_controlled_rotation_gradient_matches_fd():
    n = 3
    gates = [G("h", (0,)), G("h", (1,)), G("ry", (2,), (0,), param_index=0),
             G("p", (1,), (2,), param_index=1), G("rx", (0,), (1, 2), param_index=2, scale=-1.5)]
    theta = np.array([0.4, -1.2, 0.9])
    H = W.random_pauli_sum(n, 6, 1)
    e, g = O.adjoint_grad(O.basis(n, 0), n, gates, theta, *H)
    assert np.abs(g - _finite_diff(O.basis(n, 0), n, gates, theta, H)).max() < 1e-8


def test_oracle_thread_count_does_not_change_results():
    """The gate loops' optional threads (all-cores CPU baseline) update
    disjoint amplitudes: a circuit with controls, two-target gates and every
    kind gives bit-identical states on 1 thread and on all processors."""
    L = O.lib()
    n = 16
    gates = W.random_gate_mix(n, 120, seed=5)
    try:
        assert L.or_set_threads(1) == 1
        a = O.apply_circuit(O.basis(n, 3), n, gates)
        L.or_set_threads(0)
        b = O.apply_circuit(O.basis(n, 3), n, gates)
    finally:
        L.or_set_threads(1)
    assert np.array_equal(a, b)
