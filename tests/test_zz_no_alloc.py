"""The allocation-free expectation entry point (qs_expval_pauli_sum_noalloc),
for callers that cannot allocate device memory while they evaluate an
observable. It must give the same value as qs_expval_pauli_sum on the same
state, call after call, although every call reuses one array compiled into
the library, and it must make no device allocation. This file is collected
last so that a run stopping at its first failure has already run every other
test; it also passes on its own in a fresh process (the first call loads the
library's device code in the current context).
"""
import numpy as np
import pytest

import oracle as O
import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {Q.QS_C128: 1e-12, Q.QS_C64: 2e-5}


def shared_x_sum(n: int, seed: int):
    """20 strings on one non-zero x mask (three launches of at most 8 strings)
    and 12 diagonal strings (x = 0), shuffled so that the entry point's sort
    has to regroup them."""
    rng = np.random.default_rng(seed)
    x = int(rng.integers(1, 1 << n))
    xs = [x] * 20 + [0] * 12
    zs = [int(rng.integers(0, 1 << n)) for _ in xs]
    c = rng.standard_normal(len(xs))
    perm = rng.permutation(len(xs))
    return (c[perm], np.array(xs, dtype=np.uint64)[perm], np.array(zs, dtype=np.uint64)[perm])


@pytest.mark.parametrize("dt", [Q.QS_C128, Q.QS_C64])
def test_noalloc_expval_matches_allocating_entry_point_twice(dt):
    B.build()
    n = 14
    gates = W.random_layered(n, 3, seed=11)
    h = Q.qs_state_alloc(n, dt)
    try:
        Q.qs_apply_circuit(h, gates, None, Q.make_opts(fuse_k=3))
        _, _, ptr = Q.qs_state_info(h)
        H1 = W.random_pauli_sum(n, 300, seed=21)
        c2, x2, z2 = W.random_pauli_sum(n, 40, seed=22)
        # second Hamiltonian: fewer terms, diagonal strings and a shared x mask
        H2 = (np.concatenate([c2, [0.5, -1.5, 0.25]]),
              np.concatenate([x2, np.array([0, 0, x2[3]], dtype=np.uint64)]),
              np.concatenate([z2, np.array([3, 12, 7], dtype=np.uint64)]))
        H3 = shared_x_sum(n, seed=24)
        psi = O.apply_circuit(O.basis(n, 0), n, gates)
        Q.qs_expval_pauli_sum_noalloc(ptr, n, dt, None, *H1)   # first call in this context
        for H in (H1, H2, H3, H1):   # calls in a row on the shared array
            want = Q.qs_expval_pauli_sum(h, *H)
            a0 = Q.qs_device_alloc_count()
            got = Q.qs_expval_pauli_sum_noalloc(ptr, n, dt, None, *H)
            assert Q.qs_device_alloc_count() == a0, "the no-alloc entry point allocated device memory"
            bar = TOL[dt] * float(np.abs(H[0]).sum())
            assert abs(got - want) <= bar
            assert abs(got - O.expval(psi, n, *H).real) <= bar
        too_many = W.random_pauli_sum(n, 1025, seed=23)
        with pytest.raises(Q.QsError) as e:
            Q.qs_expval_pauli_sum_noalloc(ptr, n, dt, None, *too_many)
        assert e.value.status == Q.QS_ERR_ARG
    finally:
        Q.qs_state_free(h)
