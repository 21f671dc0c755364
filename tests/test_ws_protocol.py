"""A model of the persistent row kernel's synchronisation protocol, run on the
CPU under random interleavings.

The roles are the kernel's: four gather warps (stage n by warp n % 4, ring
slot (n % 4) + 4 ((n / 4) % (S / 4))) that wait for a free slot, write the
stage's metadata, arrive on its transaction barrier with the bytes to
expect and issue the copies; the copies, which land later (each fill as a
process of its own); the MMA warp, which waits for a stage's transaction
barrier (copies landed and metadata written), runs the products and frees
the slot; the drain and the consumers, with the row hand-off through
row_ready / row_read.  Barriers keep mbarrier semantics: a wait tells
phases apart by parity only, and a transaction barrier's phase completes
once its arrival is in and its expected bytes have landed.  Every read is
checked against what it must see (the stage's metadata and data, the row's
record, the slot's row); the gather warps wait for their last copies before
they end; the run must end with every row consumed once, without a
deadlock.  With split copies (the long-row stages: the first feature block
by TMA, the rest by cp.async), every lane of the filling warp also arrives on
the stage's barrier once its own copies have landed, and the barrier counts
those arrivals.  Three planted protocol mistakes must be caught: a drain that
does not wait for a free consumer slot, gather warps that refill a slot
without waiting for it to be free, and a split-copy barrier that does not
count the lanes' arrivals.
"""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.phase = 0  # completed phases

    def arrive(self, k=1):
        for _ in range(k):
            self.pending -= 1
            assert self.pending >= 0
            if self.pending == 0:
                self.phase += 1
                self.pending = self.count

    def done(self, parity):
        # the phase with this parity has completed: the current one has the other parity
        return (self.phase & 1) != parity


class TxBar:
    """An mbarrier with `count` expected arrivals per phase and a transaction count."""

    def __init__(self, count=1):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive_expect(self, nbytes):
        self.tx += nbytes
        self.pending -= 1
        assert self.pending >= 0
        self._check()

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0, "an arrival the barrier does not count"
        self._check()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        assert self.tx >= 0, "copy bytes landed that no arrival announced"
        self._check()

    def done(self, parity):
        return (self.phase & 1) != parity


def ws_slot(n, S):
    return (n & 3) + 4 * ((n >> 2) % (S >> 2))


LANES = 4  # lanes of a filling warp in the model (the kernel's 32 arrive the same way)


def run(S, C, rows, seed, slot=ws_slot, mistake=None, split=False):
    rnd = random.Random(seed)
    count = 1 + LANES if split and mistake != "split_count" else 1
    tma = [TxBar(count) for _ in range(S)]
    data_cp = [[None] * LANES for _ in range(S)]  # stage whose cp.async part each lane landed
    empty = [Bar(1) for _ in range(S)]
    data = [None] * S  # stage whose copies last landed in each slot
    copies = []
    acc_full, acc_empty = [Bar(1), Bar(1)], [Bar(128), Bar(128)]
    slot_full = [Bar(128) for _ in range(C)]
    slot_empty = [Bar(1) for _ in range(C)]
    row_ready, row_read = Bar(1), Bar(128)
    RECS = 32
    recs = [("garbage", -1)] * RECS
    meta = [None] * S
    slots = [None] * C
    work = list(rows) + [None]  # None: no more rows
    published = {}
    consumed = []
    errors = []
    def copy(s, nn, nbytes):
        for _ in range(rnd.randint(0, 6)):
            yield
        data[s] = nn
        tma[s].complete_tx(nbytes)

    def cp_copy(s, nn, lane):
        # a lane's cp.async copies (none for a stage without ratings) land,
        # then its arrival on the stage's barrier
        for _ in range(rnd.randint(0, 6)):
            yield
        data_cp[s][lane] = nn
        tma[s].arrive()

    def gather(wg):
        n, q, last = 0, 0, {}
        while True:
            if wg == 0:
                if q > 0:
                    while not row_read.done((q - 1) & 1):
                        yield
                published["row"] = (q, work[q] if q < len(work) else None)
                row_ready.arrive()
            while not row_ready.done(q & 1):
                yield
            qq, nst_row = published["row"]
            assert qq == q, ("row hand-off", qq, q)
            row_read.arrive(32)
            final = nst_row is None
            nst = max(1, nst_row or 0)
            st = (wg - (n & 3)) & 3
            while st < nst:
                nn = n + st
                s = slot(nn, S)
                while mistake != "no_empty_wait" and not empty[s].done(((nn // S) & 1) ^ 1):
                    yield
                if st == 0:
                    recs[q % RECS] = ("sentinel" if final else "row", q)
                meta[s] = (q % RECS, st == 0, st == nst - 1, nn)
                nbytes = rnd.choice([0, 512, 4096])  # a stage without ratings copies nothing
                tma[s].arrive_expect(nbytes)
                if nbytes:
                    copies.append(copy(s, nn, nbytes))
                else:
                    data[s] = nn
                if split:
                    for lane in range(LANES):
                        copies.append(cp_copy(s, nn, lane))
                last[s] = nn
                st += 4
                if rnd.random() < 0.5:
                    yield
            n += nst
            if final:
                break
            q += 1
        # the copies issued land before the warp ends
        for s, m in last.items():
            while not tma[s].done((m // S) & 1):
                yield

    def mma():
        n, q = 0, 0
        while True:
            s = slot(n, S)
            while not tma[s].done((n // S) & 1):
                yield
            m = meta[s]
            assert m[3] == n, ("stage metadata", m, n)
            assert data[s] == n, ("stage data", data[s], n)
            if split:
                assert all(d == n for d in data_cp[s]), ("stage cp.async data", data_cp[s], n)
            rec = recs[m[0]]
            b = q & 1
            if m[1]:
                while not acc_empty[b].done(((q >> 1) & 1) ^ 1):
                    yield
            yield  # the MMAs run
            empty[s].arrive()
            n += 1
            if m[2]:
                acc_full[b].arrive()
                q += 1
                if rec[0] == "sentinel":
                    return

    def drain():
        q = 0
        while True:
            b = q & 1
            while not acc_full[b].done((q >> 1) & 1):
                yield
            rec = recs[q % RECS]
            assert rec[0] != "garbage" and rec[1] == q, ("row record", q, rec)
            if rec[0] == "sentinel":
                for i in range(C):
                    c, use = (q + i) % C, (q + i) // C
                    while not slot_empty[c].done((use & 1) ^ 1):
                        yield
                    slots[c] = "stop"
                    slot_full[c].arrive(128)
                return
            c = q % C
            while mistake != "no_slot_wait" and not slot_empty[c].done(((q // C) & 1) ^ 1):
                yield
            yield
            slots[c] = q
            acc_empty[b].arrive(128)
            slot_full[c].arrive(128)
            q += 1

    def consumer(c):
        qc = 0
        while True:
            while not slot_full[c].done(qc & 1):
                yield
            if slots[c] == "stop":
                return
            assert slots[c] == c + qc * C, ("slot row", c, qc, slots[c])
            consumed.append(slots[c])
            for _ in range(rnd.randint(1, 5)):
                yield
            slot_empty[c].arrive()
            qc += 1

    alive = [gather(w) for w in range(4)] + [mma(), drain()] + [consumer(c) for c in range(C)]
    steps = 0
    while alive and not errors:
        alive.extend(copies)
        copies.clear()
        a = rnd.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
        except AssertionError as e:
            errors.append(str(e))
        steps += 1
        if steps > 400_000:
            errors.append("deadlock")
    if not errors and sorted(consumed) != list(range(len(rows))):
        errors.append(("rows consumed", sorted(consumed)[:10], len(rows)))
    return errors


def _rows(seed):
    rnd = random.Random(1000 + seed)
    return [rnd.choice([0, 1, 1, 2, 3, 5, 9]) for _ in range(rnd.randint(1, 30))]


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("S,C", [(4, 6), (4, 1), (8, 2), (8, 3), (12, 1), (16, 2)])
def test_protocol_under_random_interleavings(S, C, split):
    for seed in range(25):
        errs = run(S, C, _rows(seed), seed, split=split)
        assert not errs, (S, C, seed, errs[:2])


@pytest.mark.parametrize("mistake", ["no_slot_wait", "no_empty_wait", "split_count"])
def test_planted_protocol_mistakes_are_caught(mistake):
    failures = sum(1 for seed in range(40)
                   if run(8, 2, _rows(seed), seed, mistake=mistake, split=mistake == "split_count"))
    assert failures > 0
