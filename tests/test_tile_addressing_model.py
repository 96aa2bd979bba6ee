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


def _bulk_tile_schedule(my, seed, wait_read=True):
    """The bulk-staged tile pass (k_tile_bulk) as a discrete-event model: warp 0
    issues the loads of tile i + 1 into buffer (i + 1) & 1 at the top of
    iteration i (after cp.async.bulk.wait_group.read for the stores it issued
    from that buffer), every thread waits for tile i's buffer, runs the ops,
    then warp 0 issues its stores. Copies complete after random delays; the
    model reports a buffer overwritten before its stores read it out, ops on a
    buffer before its load landed, or a tile not stored exactly once."""
    import random
    rng = random.Random(seed)
    now = 0.0
    landed = {}            # tile -> time its load completes
    buf_read_done = {0: 0.0, 1: 0.0}   # time the last stores from the buffer finished reading it
    buf_tile = {0: None, 1: None}
    stored, errors = [], []

    def load(i):
        nonlocal now
        b = i & 1
        if wait_read:
            now = max(now, buf_read_done[b])
        elif buf_read_done[b] > now:
            errors.append("buffer loaded before its stores read it out")
        buf_tile[b] = i
        landed[i] = now + rng.uniform(1, 6)

    if my:
        load(0)
    for i in range(my):
        if i + 1 < my:
            load(i + 1)
        now = max(now, landed[i])                    # mbarrier wait for tile i
        if buf_tile[i & 1] != i:
            errors.append("ops on a buffer holding another tile")
        now += rng.uniform(0.5, 4)                   # the ops
        buf_read_done[i & 1] = now + rng.uniform(0.5, 5)
        stored.append(i)
    if stored != list(range(my)):
        errors.append("tiles not stored exactly once in order")
    return errors


def test_bulk_tile_pipeline_has_no_buffer_hazard():
    for seed in range(300):
        for my in (0, 1, 2, 3, 7, 40):
            assert _bulk_tile_schedule(my, seed) == [], (seed, my)


def test_bulk_tile_pipeline_without_the_read_wait_is_caught():
    """Dropping cp.async.bulk.wait_group.read lets a load overwrite a buffer
    whose stores have not read it yet; the model reports it."""
    fails = sum(1 for seed in range(200) if _bulk_tile_schedule(20, seed, wait_read=False))
    assert fails > 100
