"""CPU model of the tile pass's HBM addressing (kernels_tile.cuh).

A tile pass stages 2^m amplitudes: the L low qubits (contiguous runs of 2^L
amplitudes) and nh = m - L higher tile qubits (high[], ascending). The kernel
computes, per CTA, segoff[s] = OR_k bit k of s << high[k]; per tile number t,
base = insert_zero_bits(t << L, high); and reads tile element e from
base | segoff[e >> L] | (e & (2^L - 1)). This model replays exactly that
arithmetic on the tile qubit sets real plans hand the kernel and checks that
the tiles partition the state, that tile-local bit j is the pass's j-th tile
qubit (the bit positions the ops are compiled against), and that complex64
tiles can use 16-byte (two-amplitude) vector accesses. It runs without a GPU.
"""
import numpy as np
import pytest

import paper_2509_04955_gb300 as Q
from paper_2509_04955_gb300 import build as B
from paper_2509_04955_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def insert_zero_bits(x, pos):
    """The kernel's helper: make room for a zero bit at each (ascending) position."""
    for p in pos:
        lo = x & ((1 << p) - 1)
        x = ((x >> p) << (p + 1)) | lo
    return x


def tile_addresses(n, L, high):
    m = L + len(high)
    segoff = [0] * (1 << len(high))
    for s in range(1 << len(high)):
        for k, q in enumerate(high):
            segoff[s] |= ((s >> k) & 1) << q
    lmask = (1 << L) - 1
    e = np.arange(1 << m, dtype=np.int64)
    seg = np.array(segoff, dtype=np.int64)[e >> L]
    rows = []
    for t in range(1 << (n - m)):
        base = insert_zero_bits(t << L, high)
        rows.append(base | seg | (e & lmask))
    return np.array(rows)


@pytest.mark.parametrize("n,dt,opts", [
    (9, Q.QS_C64, Q.make_opts(fuse_k=2, tile_qubits=6, low_qubits=2)),
    (10, Q.QS_C128, Q.make_opts(fuse_k=3, tile_qubits=7, low_qubits=3)),
    (11, Q.QS_C64, Q.make_opts(fuse_k=4, tile_qubits=9, low_qubits=4)),
    (8, Q.QS_C128, Q.make_opts(fuse_k=1, tile_qubits=4, low_qubits=1)),
    (7, Q.QS_C64, Q.make_opts(fuse_k=5, tile_qubits=7, low_qubits=1)),     # one tile is the whole state
])
def test_tile_addressing_partitions_the_state(n, dt, opts):
    gates = W.random_gate_mix(n, 60, seed=n) + W.random_layered(n, 3, seed=n)
    plan = Q.qs_plan_create(n, dt, gates, opts)
    try:
        info = Q.qs_plan_info_get(plan)
        L = info["low_qubits"]
        assert L >= 1          # complex64 tiles move two amplitudes per 16-byte access
        seen_high = False
        for ps in Q.qs_plan_passes(plan):
            tile = sorted(ps["tile"])
            assert tile[:L] == list(range(L))
            high = [q for q in tile if q >= L]
            seen_high |= bool(high) and high[0] > L
            addr = tile_addresses(n, L, high)
            # every amplitude in exactly one tile slot
            assert np.array_equal(np.sort(addr.ravel()), np.arange(1 << n))
            # tile-local bit j holds qubit tile[j]; bits outside the tile are the tile number's, in order
            e = np.arange(addr.shape[1])
            for j, q in enumerate(tile):
                assert np.array_equal((addr >> q) & 1, np.broadcast_to((e >> j) & 1, addr.shape))
            rest = [q for q in range(n) if q not in tile]
            for k, q in enumerate(rest):
                t = np.arange(addr.shape[0])[:, None]
                assert np.array_equal((addr >> q) & 1, np.broadcast_to((t >> k) & 1, addr.shape))
            # vector accesses: even elements sit at even addresses, their neighbour next to them
            assert np.all(addr[:, 0::2] % 2 == 0) and np.array_equal(addr[:, 1::2], addr[:, 0::2] + 1)
        assert seen_high or n == len(tile)   # some pass selects non-adjacent high qubits
    finally:
        Q.qs_plan_free(plan)
