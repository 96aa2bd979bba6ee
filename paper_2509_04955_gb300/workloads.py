"""Seeded synthetic inputs: gate lists, Pauli sums, angles and basis indices.

This module is shared by the FP64 oracle tests, the CUDA-path tests and the
benchmark. It holds no arithmetic of the simulator itself: no gate matrix,
no state update, no fusion. A gate is a name plus qubit indices plus an angle
(or a reference into a parameter vector); each side of the comparison turns
that into numbers on its own.

Conventions (Section 2.1, Eq. 1-2): qubit q is bit q of the amplitude index,
so qubit 0 is the least significant bit.

Workload shapes follow the circuit classes of Section 4.1 (QFT, hardware-
efficient ansatz, plus the random-layer and UCC-style Pauli-exponential
circuits used by the benchmark):

* ``random_layered``: every layer applies one of H, RX, RY, RZ (chosen
  uniformly, angle uniform in [-pi, pi]) to every qubit, then an entangler
  (CNOT or CZ) on a random perfect matching of the qubits. The matching is a
  Fisher-Yates shuffle of 0..n-1 paired consecutively.
* ``qft``: for j = n-1 .. 0: H(j), then CP(pi / 2^(j-m)) with control m and
  target j for m = j-1 .. 0; finally SWAP(j, n-1-j) for j < n/2.
* ``hea``: per layer RY(theta) then RZ(theta) on every qubit, then CZ(q, q+1)
  for q = 0 .. n-2. Every rotation has its own parameter.
* ``ucc``: per term exp(-i theta_j P_j) built from a basis change (H for X,
  RX(+pi/2) for Y), a CNOT ladder onto the highest support qubit, RZ(2 theta_j)
  and the mirror image.
* ``random_pauli_sum``: letters uniform over I, X, Y, Z per qubit,
  coefficients N(0, 1); returned as (coeff, xmask, zmask) with Y = x and z set.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Names understood by both the oracle and the CUDA library.
ONE_TARGET_KINDS = ("h", "x", "y", "z", "s", "sdg", "t", "tdg",
                    "rx", "ry", "rz", "p", "u1")
TWO_TARGET_KINDS = ("swap", "u2")
PARAMETRIC_KINDS = ("rx", "ry", "rz", "p")
SELF_INVERSE = ("h", "x", "y", "z", "swap")
INVERSE_NAME = {"s": "sdg", "sdg": "s", "t": "tdg", "tdg": "t"}


@dataclass(frozen=True)
class Gate:
    """One gate of a circuit.

    ``targets``: 1 qubit for ONE_TARGET_KINDS, 2 for TWO_TARGET_KINDS.
    ``controls``: up to 2 control qubits (the gate acts when all are 1).
    ``angle``: fixed angle for parametric kinds.
    ``param_index``/``scale``: when ``param_index >= 0`` the angle is
    ``angle + scale * theta[param_index]``.
    ``matrix``: for u1 (2x2) / u2 (4x4) a row-major complex matrix; for u2 the
    local index bit 0 belongs to ``targets[0]`` and bit 1 to ``targets[1]``.
    """
    kind: str
    targets: tuple
    controls: tuple = ()
    angle: float = 0.0
    param_index: int = -1
    scale: float = 1.0
    matrix: tuple | None = field(default=None, compare=False)

    @property
    def qubits(self) -> tuple:
        return tuple(self.targets) + tuple(self.controls)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_matching(n: int, rng: np.random.Generator) -> list[tuple[int, int]]:
    """Random perfect matching of 0..n-1 (odd n leaves one qubit out)."""
    perm = list(range(n))
    for i in range(n - 1, 0, -1):           # Fisher-Yates
        j = int(rng.integers(0, i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return [(perm[2 * i], perm[2 * i + 1]) for i in range(n // 2)]


def random_layered(n: int, depth: int, seed: int, entangler: str = "cnot") -> list[Gate]:
    rng = _rng(seed)
    gates: list[Gate] = []
    for _ in range(depth):
        for q in range(n):
            kind = ("h", "rx", "ry", "rz")[int(rng.integers(0, 4))]
            angle = float(rng.uniform(-math.pi, math.pi))
            if kind == "h":
                gates.append(Gate("h", (q,)))
            else:
                gates.append(Gate(kind, (q,), angle=angle))
        for a, b in random_matching(n, rng):
            if entangler == "cnot":
                gates.append(Gate("x", (b,), controls=(a,)))
            elif entangler == "cz":
                gates.append(Gate("z", (b,), controls=(a,)))
            else:
                raise ValueError(entangler)
    return gates


def qft(n: int, swaps: bool = True) -> list[Gate]:
    gates: list[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("h", (j,)))
        for m in range(j - 1, -1, -1):
            gates.append(Gate("p", (j,), controls=(m,), angle=math.pi / (1 << (j - m))))
    if swaps:
        for j in range(n // 2):
            gates.append(Gate("swap", (j, n - 1 - j)))
    return gates


def hea(n: int, layers: int) -> tuple[list[Gate], int]:
    """Hardware-efficient ansatz; returns (gates, number of parameters)."""
    gates: list[Gate] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("ry", (q,), param_index=p)); p += 1
        for q in range(n):
            gates.append(Gate("rz", (q,), param_index=p)); p += 1
        for q in range(n - 1):
            gates.append(Gate("z", (q + 1,), controls=(q,)))
    return gates, p


def pauli_exponential(support: list[int], letters: str, param_index: int) -> list[Gate]:
    """Gates for exp(-i theta P) with P = prod letters[j] on support[j]."""
    order = sorted(range(len(support)), key=lambda j: support[j])
    sup = [support[j] for j in order]
    let = [letters[j] for j in order]
    pre: list[Gate] = []
    post: list[Gate] = []
    for q, l in zip(sup, let):
        if l == "X":
            pre.append(Gate("h", (q,))); post.append(Gate("h", (q,)))
        elif l == "Y":
            pre.append(Gate("rx", (q,), angle=math.pi / 2))
            post.append(Gate("rx", (q,), angle=-math.pi / 2))
    ladder = [Gate("x", (sup[i + 1],), controls=(sup[i],)) for i in range(len(sup) - 1)]
    core = [Gate("rz", (sup[-1],), param_index=param_index, scale=2.0)]
    return pre + ladder + core + ladder[::-1] + post


def ucc(n: int, nterms: int, seed: int, wmin: int = 2, wmax: int = 8) -> tuple[list[Gate], list[tuple[list[int], str]]]:
    """UCC-style circuit: returns (gates, [(support, letters)] per term)."""
    rng = _rng(seed)
    gates: list[Gate] = []
    terms = []
    for j in range(nterms):
        w = int(rng.integers(wmin, min(wmax, n) + 1))
        support = [int(x) for x in rng.choice(n, size=w, replace=False)]
        letters = "".join("XYZ"[int(rng.integers(0, 3))] for _ in range(w))
        terms.append((support, letters))
        gates.extend(pauli_exponential(support, letters, j))
    return gates, terms


def random_pauli_sum(n: int, nterms: int, seed: int):
    """Returns (coeff[float64], xmask[uint64], zmask[uint64])."""
    rng = _rng(seed)
    coeff = rng.standard_normal(nterms)
    xm = np.zeros(nterms, dtype=np.uint64)
    zm = np.zeros(nterms, dtype=np.uint64)
    for j in range(nterms):
        x = z = 0
        for q in range(n):
            letter = int(rng.integers(0, 4))    # 0=I 1=X 2=Y 3=Z
            if letter in (1, 2):
                x |= 1 << q
            if letter in (2, 3):
                z |= 1 << q
        xm[j] = x
        zm[j] = z
    return coeff, xm, zm


def pauli_string_masks(n: int, support: list[int], letters: str) -> tuple[int, int]:
    x = z = 0
    for q, l in zip(support, letters):
        if l in "XY":
            x |= 1 << q
        if l in "YZ":
            z |= 1 << q
    return x, z


def hea_staggered(n: int, layers: int) -> tuple[list[Gate], int]:
    """The VQE-HEA circuit class of Section 4.1: per layer RX, RY, RZ on every
    qubit (one parameter each), then CNOT(q -> q + 1) for q = layer mod 2,
    layer mod 2 + 2, ... (staggered). Returns (gates, number of parameters)."""
    gates: list[Gate] = []
    k = 0
    for layer in range(layers):
        for kind in ("rx", "ry", "rz"):
            for q in range(n):
                gates.append(Gate(kind, (q,), param_index=k))
                k += 1
        for q in range(layer % 2, n - 1, 2):
            gates.append(Gate("x", (q + 1,), (q,)))
    return gates, k


def random_regular_graph(n: int, degree: int, seed: int) -> list[tuple[int, int]]:
    """Edges (u < v) of a random simple d-regular graph on n vertices: the
    configuration model (n*d stubs paired at random), redrawn until the pairing
    has no loop and no repeated edge."""
    if (n * degree) % 2 or degree >= n:
        raise ValueError("no simple d-regular graph with these sizes")
    rng = _rng(seed)
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), degree)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = {(int(min(a, b)), int(max(a, b))) for a, b in pairs}
        if len(edges) == len(pairs) and all(a != b for a, b in edges):
            return sorted(edges)
    raise RuntimeError("no simple pairing found")


def qaoa(n: int, layers: int, edges) -> tuple[list[Gate], int]:
    """QAOA circuit for MaxCut: H on every qubit, then per layer l the cost
    unitary prod_edges exp(-i gamma_l Z_u Z_v) (CNOT(u -> v), RZ_v(2 gamma_l),
    CNOT(u -> v)) and the mixer prod_q exp(-i beta_l X_q) = RX_q(2 beta_l).
    Parameters: theta[2 l] = gamma_l, theta[2 l + 1] = beta_l."""
    gates = [Gate("h", (q,)) for q in range(n)]
    for layer in range(layers):
        for u, v in edges:
            gates.append(Gate("x", (v,), (u,)))
            gates.append(Gate("rz", (v,), param_index=2 * layer, scale=2.0))
            gates.append(Gate("x", (v,), (u,)))
        for q in range(n):
            gates.append(Gate("rx", (q,), param_index=2 * layer + 1, scale=2.0))
    return gates, 2 * layers


def phase_run_circuit(n: int, layers: int, per_layer: int, seed: int, max_weight: int = 4):
    """Layers of H on every qubit, each followed by a stretch of gates that is
    diagonal as a whole: Z-string exponentials (a CNOT ladder, RZ, the ladder
    undone; weight 2..max_weight), one-control phase gates (CP, CRZ, CZ, CS,
    CT), one-qubit diagonal gates (Z, S, T, Sdg, Tdg, RZ, P) and SWAP
    sandwiches (SWAP, a diagonal gate on one of the two qubits, SWAP). Angles
    are parametric (one parameter each) or fixed uniform in [-pi, pi].
    Returns (gates, number of parameters)."""
    rng = _rng(seed)
    gates: list[Gate] = []
    npar = 0

    def angle_gate(kind, q, controls=()):
        nonlocal npar
        if rng.integers(0, 2):
            npar += 1
            return Gate(kind, (q,), controls, param_index=npar - 1, scale=float(rng.choice([1.0, -2.0, 0.5])))
        return Gate(kind, (q,), controls, angle=float(rng.uniform(-math.pi, math.pi)))

    for _ in range(layers):
        gates += [Gate("h", (q,)) for q in range(n)]
        for _ in range(per_layer):
            c = int(rng.integers(0, 4))
            if c == 0:
                sup = [int(q) for q in rng.choice(n, int(rng.integers(2, max_weight + 1)), replace=False)]
                ladder = [Gate("x", (sup[i + 1],), (sup[i],)) for i in range(len(sup) - 1)]
                gates += ladder + [angle_gate("rz", sup[-1])] + ladder[::-1]
            elif c == 1:
                a, b = (int(q) for q in rng.choice(n, 2, replace=False))
                kind = ("p", "rz", "z", "s", "t")[int(rng.integers(0, 5))]
                gates.append(angle_gate(kind, b, (a,)) if kind in ("p", "rz") else Gate(kind, (b,), (a,)))
            elif c == 2:
                q = int(rng.integers(0, n))
                kind = ("z", "s", "t", "sdg", "tdg", "rz", "p")[int(rng.integers(0, 7))]
                gates.append(angle_gate(kind, q) if kind in ("rz", "p") else Gate(kind, (q,)))
            else:
                a, b = (int(q) for q in rng.choice(n, 2, replace=False))
                gates += [Gate("swap", (a, b)), angle_gate("p", a), Gate("swap", (a, b))]
    return gates, npar


def maxcut_hamiltonian(edges):
    """C = sum_edges (1 - Z_u Z_v) / 2 as (coeff, xmask, zmask): the number of
    cut edges of a computational basis state."""
    coeff = [0.5 * len(edges)] + [-0.5] * len(edges)
    xm = [0] * (len(edges) + 1)
    zm = [0] + [(1 << u) | (1 << v) for u, v in edges]
    return np.array(coeff), np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64)


def random_basis_index(n: int, seed: int) -> int:
    return int(_rng(seed).integers(0, 1 << n)) if n < 63 else int(_rng(seed).integers(0, 1 << 62))


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex128 vector with Gaussian entries."""
    rng = _rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def random_unitary(dim: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-like unitary from the QR decomposition of a complex Gaussian matrix."""
    z = rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def thetas_uniform(p: int, seed: int) -> np.ndarray:
    return _rng(seed).uniform(-math.pi, math.pi, size=p)


def thetas_normal(p: int, seed: int, sigma: float = 0.1, batch: int | None = None) -> np.ndarray:
    shape = (p,) if batch is None else (batch, p)
    return _rng(seed).normal(0.0, sigma, size=shape)


def random_gate_mix(n: int, ngates: int, seed: int, max_controls: int = 2) -> list[Gate]:
    """Every gate kind on random qubits, controls above and below the target."""
    rng = _rng(seed)
    gates: list[Gate] = []
    kinds = ONE_TARGET_KINDS + TWO_TARGET_KINDS
    for _ in range(ngates):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        nt = 2 if kind in TWO_TARGET_KINDS else 1
        if n < nt:
            continue
        nc = int(rng.integers(0, min(max_controls, n - nt) + 1))
        qs = [int(x) for x in rng.choice(n, size=nt + nc, replace=False)]
        targets, controls = tuple(qs[:nt]), tuple(qs[nt:])
        angle = float(rng.uniform(-math.pi, math.pi))
        matrix = None
        if kind == "u1":
            matrix = tuple(random_unitary(2, rng).reshape(-1))
        elif kind == "u2":
            matrix = tuple(random_unitary(4, rng).reshape(-1))
        gates.append(Gate(kind, targets, controls, angle=angle if kind in PARAMETRIC_KINDS else 0.0,
                          matrix=matrix))
    return gates


def block_circuit(qubit_sets, gates_per_block: int, seed: int) -> list[Gate]:
    """For each qubit set in turn, a chain of random dense two-qubit (u2)
    gates on random pairs inside the set: a contraction to blocks of
    len(set) qubits sees one block per set, on exactly those qubits."""
    rng = _rng(seed)
    gates: list[Gate] = []
    for qs in qubit_sets:
        qs = [int(q) for q in qs]
        for _ in range(gates_per_block):
            a, b = (int(x) for x in rng.choice(len(qs), size=2, replace=False))
            gates.append(Gate("u2", (qs[a], qs[b]), matrix=tuple(random_unitary(4, rng).reshape(-1))))
    return gates


def inverse_circuit(gates: list[Gate], theta=None) -> list[Gate]:
    """The circuit whose product is the inverse: reversed order, each gate inverted.

    Parametric angles are resolved against ``theta`` and negated; custom
    matrices are conjugate-transposed (input bookkeeping, not simulation)."""
    out: list[Gate] = []
    for g in reversed(gates):
        if g.kind in SELF_INVERSE:
            out.append(g)
        elif g.kind in INVERSE_NAME:
            out.append(Gate(INVERSE_NAME[g.kind], g.targets, g.controls))
        elif g.kind in PARAMETRIC_KINDS:
            a = g.angle + (g.scale * float(theta[g.param_index]) if g.param_index >= 0 else 0.0)
            out.append(Gate(g.kind, g.targets, g.controls, angle=-a))
        elif g.kind in ("u1", "u2"):
            d = 2 if g.kind == "u1" else 4
            m = np.array(g.matrix).reshape(d, d).conj().T
            out.append(Gate(g.kind, g.targets, g.controls, matrix=tuple(m.reshape(-1))))
        else:
            raise ValueError(g.kind)
    return out


def gate_counts(gates: list[Gate]) -> dict:
    out: dict = {}
    for g in gates:
        key = ("c" * len(g.controls)) + g.kind
        out[key] = out.get(key, 0) + 1
    return out
