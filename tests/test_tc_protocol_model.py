"""Host-side models of the bulk-copy tensor-core pass (no GPU).

They restate, in Python, the index arithmetic and the barrier protocol of
k_tc_bulk and check the invariants the kernel relies on:

* slot reads: element (row, column) of a tile lands at its tile-local index
  (runs of >= 2^7 contiguous amplitudes copied in order), every converter
  lane reads the intended element after its column order is XORed with
  phi(lane), and a warp's 32 reads hit each shared-memory bank pair at most
  twice (optimal for 8-byte reads) for every block placement;
* stores: after the in-warp exchange of the column bits on qubits 0/1 with
  lane bits 4/3, every value goes to its own address and every warp store
  covers 8 whole 32-byte sectors;
* barriers: with parity waits (exact within one phase), in-order MMA
  completion and random copy / MMA delays, no schedule deadlocks or lets a
  copy overwrite W, a slot, an A buffer or an accumulator still in use, for
  1 to 128 tiles per state; the protocol in which the producer waited on the
  accumulator barrier before a W reload fails the same check.
"""
import random

import pytest


# ---------------------------------------------------------------- layout

def _geometry(n, Q):
    Q = sorted(Q)
    R = [q for q in range(n) if q not in Q][:7]
    T = sorted(Q + R)
    pr = 0
    while pr < 13 and T[pr] == pr:
        pr += 1
    lam = {q: i for i, q in enumerate(T)}
    lamcol = [sum(((c >> b) & 1) << lam[Q[b]] for b in range(6)) for c in range(64)]
    coff = [sum(((c >> b) & 1) << Q[b] for b in range(6)) for c in range(64)]
    return Q, R, T, pr, lam, lamcol, coff


def _phi(Q, R, lane):
    phi = xbits = 0
    k = 0
    for b in range(4):
        if Q[b] > 3:
            break
        while k < 5 and R[k] < 4:
            k += 1
        if k >= 5:
            break
        phi |= ((lane >> k) & 1) << b
        xbits |= 1 << b
        k += 1
    return phi, xbits


PLACEMENTS = [(0, 1, 2, 3, 4, 5), (0, 1, 2, 9, 10, 11), (1, 3, 7, 9, 11, 12), (0, 7, 8, 9, 10, 11),
              (7, 8, 9, 10, 11, 12), (2, 4, 5, 6, 8, 12), (24, 25, 26, 27, 28, 29), (0, 5, 11, 19, 21, 29),
              (1, 3, 9, 14, 22, 27), (0, 2, 4, 6, 8, 10), (3, 4, 5, 6, 7, 8), (0, 1, 6, 10, 11, 13),
              (2, 3, 5, 10, 11, 15), (1, 2, 3, 4, 5, 6)]


@pytest.mark.parametrize("Q", PLACEMENTS)
def test_slot_reads_land_on_their_elements_without_bank_conflicts(Q):
    n = 30
    Q, R, T, pr, lam, lamcol, coff = _geometry(n, Q)
    assert pr >= 7
    nontile = [q for q in range(n) if q not in T]
    # landing: run j of 2^pr amplitudes at slot offset j * 2^pr; local index = tile bits in order
    runoff = [sum(((j >> b) & 1) << T[pr + b] for b in range(13 - pr)) for j in range(1 << (13 - pr))]
    slot = {}
    for j, r in enumerate(runoff):
        for o in range(1 << pr):
            slot[j * (1 << pr) + o] = r | o
    assert sorted(slot) == list(range(8192))
    for w8 in range(8):                       # converter warps: (row quadrant, column half)
        quad, half = w8 & 3, w8 >> 2
        for chunk in range(2):
            banks = {}
            for lane in range(32):
                row = 32 * quad + lane
                lrow = sum(((row >> b) & 1) << lam[R[b]] for b in range(7))
                roff = sum(((row >> b) & 1) << R[b] for b in range(7))
                phi, xbits = _phi(Q, R, lane)
                c0 = 32 * half + 16 * chunk
                tb = lrow | lamcol[c0] | lamcol[phi]
                v = [slot[tb ^ lamcol[j]] for j in range(16)]
                for j in range(16):
                    banks.setdefault(j, []).append(((tb ^ lamcol[j]) * 8 // 4) % 32 // 2)
                for b in range(4):            # restore the column order (conditional swaps)
                    if xbits >> b & 1 and phi >> b & 1:
                        for j in range(16):
                            if not j & (1 << b):
                                v[j], v[j | (1 << b)] = v[j | (1 << b)], v[j]
                for j in range(16):
                    assert v[j] == roff | coff[c0 + j]
            for j, bs in banks.items():
                assert max(bs.count(x) for x in set(bs)) <= 2


@pytest.mark.parametrize("Q", PLACEMENTS + [tuple(sorted(random.Random(s).sample(range(30), 6))) for s in range(20)])
def test_drainer_stores_cover_whole_sectors(Q):
    n = 30
    Q, R, T, pr, lam, lamcol, coff = _geometry(n, Q)
    roff_full = lambda r: sum(((r >> b) & 1) << R[b] for b in range(7))
    s0, s1 = Q[0] <= 1, Q[0] == 0 and Q[1] == 1
    rbit4, rbit3 = 1 << R[4], 1 << R[3]
    for w8 in range(8):
        quad, half = w8 & 3, w8 >> 2
        for chunk in range(2):
            v = [[(32 * quad + l, 32 * half + 16 * chunk + q) for q in range(16)] for l in range(32)]

            def stage(J, M):
                new = [r[:] for r in v]
                for l in range(32):
                    up = (l >> M) & 1
                    p = l ^ (1 << M)
                    for q in range(16):
                        if q & (1 << J):
                            continue
                        q1 = q | (1 << J)
                        recv = v[p][q] if (p >> M) & 1 else v[p][q1]
                        if up:
                            new[l][q] = recv
                        else:
                            new[l][q1] = recv
                return new
            if s0:
                v = stage(0, 4)
            if s1:
                v = stage(1, 3)
            for q in range(16):
                addrs = []
                for l in range(32):
                    roff = roff_full(32 * quad + l)
                    if s0:
                        roff &= ~rbit4
                    if s1:
                        roff &= ~rbit3
                    a, qq = roff, q
                    if s0:
                        a |= rbit4 if q & 1 else 0
                        qq = (qq & ~1) | ((l >> 4) & 1)
                    if s1:
                        a |= rbit3 if q & 2 else 0
                        qq = (qq & ~2) | (((l >> 3) & 1) << 1)
                    a |= coff[32 * half + 16 * chunk + qq]
                    lr, lc = v[l][q]
                    assert a == roff_full(lr) | coff[lc]
                    addrs.append(a)
                assert len(set(addrs)) == 32
                assert len({a * 8 // 32 for a in addrs}) == 8


# ---------------------------------------------------------------- barriers

class _Bar:
    """mbarrier: `done` completed phases; try_wait.parity(P) passes iff (done & 1) != P."""

    def __init__(self, count):
        self.count, self.pending, self.done, self.tx = count, count, 0, 0

    def arrive(self):
        self.pending -= 1
        self._check()

    def expect_tx(self, b):
        self.tx += b
        self.arrive()

    def complete_tx(self, b):
        self.tx -= b
        self._check()

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.done += 1
            self.pending = self.count

    def ok(self, parity):
        return (self.done & 1) != parity


def _simulate(my, tiles_per_state, t_begin, seed, wfree_protocol):
    rng = random.Random(seed)
    state = lambda i: (t_begin + i) // tiles_per_state
    new_state = lambda i: i > 0 and state(i) != state(i - 1)
    full, empty, afull = [_Bar(1), _Bar(1)], [_Bar(8), _Bar(8)], [_Bar(8), _Bar(8)]
    mdone, dfree, wfull, wfree = [_Bar(1), _Bar(1)], [_Bar(8), _Bar(8)], _Bar(1), _Bar(1)
    events, now, last_finish = [], [0.0], [0.0]
    W = {"state": state(0), "writing": None}
    inflight, errors = {}, []

    def later(dt, fn):
        events.append((now[0] + dt, fn))

    def producer():
        issued = 0
        for i in range(my):
            s = i & 1
            if i >= 2:
                yield lambda: empty[s].ok(((i >> 1) - 1) & 1)
            full[s].expect_tx(1)
            later(rng.uniform(1, 5), lambda s=s: full[s].complete_tx(1))
            if new_state(i):
                if wfree_protocol:
                    yield lambda: wfree.ok(issued & 1)
                else:
                    yield lambda: mdone[(i - 1) & 1].ok(((i - 1) >> 1) & 1)
                if any(st != state(i) for st in inflight.values()):
                    errors.append("W overwritten under in-flight MMAs")
                W["writing"] = state(i)
                wfull.expect_tx(1)

                def land(st=state(i)):
                    W["state"], W["writing"] = st, None
                    wfull.complete_tx(1)
                later(rng.uniform(1, 5), land)
                issued += 1

    def mma():
        seen = 0
        for i in range(my):
            a = i & 1
            if new_state(i):
                yield lambda: wfull.ok(seen & 1)
                seen += 1
            yield lambda: afull[a].ok((i >> 1) & 1)
            if i >= 2:
                yield lambda: dfree[a].ok(((i >> 1) - 1) & 1)
            if W["state"] != state(i) or W["writing"] is not None:
                errors.append("MMA reads the wrong W")
            inflight[i] = state(i)

            def finish(i=i, a=a, last=(i + 1 < my and new_state(i + 1))):
                del inflight[i]
                mdone[a].arrive()
                if last:
                    wfree.arrive()
            last_finish[0] = max(last_finish[0], now[0] + rng.uniform(0.5, 3))   # in issue order
            events.append((last_finish[0], finish))

    def converter():
        for i in range(my):
            s = i & 1
            if i >= 2:
                yield lambda: mdone[s].ok(((i >> 1) - 1) & 1)
            yield lambda: full[s].ok((i >> 1) & 1)
            if (i - 2) in inflight:
                errors.append("A buffer overwritten under an MMA")
            yield ("sleep", rng.uniform(0, 1))
            empty[s].arrive()
            afull[s].arrive()

    def drainer():
        for i in range(my):
            d = i & 1
            yield lambda: mdone[d].ok((i >> 1) & 1)
            if i in inflight:
                errors.append("accumulator read before its MMA finished")
            yield ("sleep", rng.uniform(0, 1))
            dfree[d].arrive()

    roles = [producer(), mma()] + [converter() for _ in range(8)] + [drainer() for _ in range(8)]
    waiting, sleeping, alive = {}, {}, set(range(len(roles)))
    for _ in range(200000):
        if not alive:
            return errors
        progressed = False
        order = list(alive)
        rng.shuffle(order)
        for j in order:
            if j in sleeping:
                if sleeping[j] > now[0]:
                    continue
                del sleeping[j]
            w = waiting.get(j)
            if w is not None and not w():
                continue
            try:
                nxt = next(roles[j])
                if isinstance(nxt, tuple):
                    sleeping[j], waiting[j] = now[0] + nxt[1], None
                else:
                    waiting[j] = nxt
            except StopIteration:
                alive.discard(j)
            progressed = True
        if not progressed:
            if not events and not sleeping:
                return errors + ["deadlock"]
            now[0] = max(now[0], min([e[0] for e in events] + list(sleeping.values())))
            for e in [e for e in events if e[0] <= now[0]]:
                events.remove(e)
                e[1]()
    return errors + ["no progress"]


def test_barrier_protocol_has_no_hazard_or_deadlock():
    for seed in range(400):
        r = random.Random(seed * 7 + 3)
        tps = r.choice([1, 2, 3, 4, 8, 128])
        my = r.choice([1, 2, 3, 4, 5, 7, 20, 54])
        tb = r.randrange(0, 4 * tps)
        assert _simulate(my, tps, tb, seed, True) == [], (seed, tps, my, tb)


def test_earlier_reload_protocol_is_caught_by_the_model():
    fails = sum(1 for seed in range(200) if _simulate(20, 4, seed % 4, seed, False))
    assert fails > 20
