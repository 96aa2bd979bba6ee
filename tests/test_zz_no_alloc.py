"""The allocation-free expectation entry point (qs_expval_pauli_sum_noalloc),
for callers that cannot allocate device memory while they evaluate an
observable. It must give the same value as qs_expval_pauli_sum on the same
state, call after call, although every call reuses one array compiled into
the library. This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own in a
fresh process (the first call sets up the array's address).
"""
import numpy as np
import pytest

import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {Q.QS_C128: 1e-12, Q.QS_C64: 2e-5}


@pytest.mark.parametrize("dt", [Q.QS_C128, Q.QS_C64])
def test_noalloc_expval_matches_allocating_entry_point_twice(dt):
    B.build()
    n = 14
    h = Q.qs_state_alloc(n, dt)
    try:
        Q.qs_apply_circuit(h, W.random_layered(n, 3, seed=11), None, Q.make_opts(fuse_k=3))
        _, _, ptr = Q.qs_state_info(h)
        H1 = W.random_pauli_sum(n, 300, seed=21)
        c2, x2, z2 = W.random_pauli_sum(n, 40, seed=22)
        # second Hamiltonian: fewer terms, diagonal strings and a shared x mask
        H2 = (np.concatenate([c2, [0.5, -1.5, 0.25]]),
              np.concatenate([x2, np.array([0, 0, x2[3]], dtype=np.uint64)]),
              np.concatenate([z2, np.array([3, 12, 7], dtype=np.uint64)]))
        for H in (H1, H2):          # two calls in a row on the shared array
            want = Q.qs_expval_pauli_sum(h, *H)
            got = Q.qs_expval_pauli_sum_noalloc(ptr, n, dt, None, *H)
            assert abs(got - want) <= TOL[dt] * float(np.abs(H[0]).sum())
        too_many = W.random_pauli_sum(n, 1025, seed=23)
        with pytest.raises(Q.QsError) as e:
            Q.qs_expval_pauli_sum_noalloc(ptr, n, dt, None, *too_many)
        assert e.value.status == Q.QS_ERR_ARG
    finally:
        Q.qs_state_free(h)
