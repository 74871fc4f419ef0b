"""Models of the two hand-off protocols the persistent kernels rely on, run under random
interleavings of their parties (mbarrier semantics: a phase completes after `count` arrivals;
a wait with parity p returns once a phase of parity p has completed, i.e. when
completed_phases mod 2 != p).

* rf_tc_long.cu: the producer (q window, taps chunks; chunk 0 completes on a transaction
  barrier of its own, which the producer waits on before it arrives on the item's go
  barrier; at a tile change it first waits for a commit the MMA issuer makes after the
  last item of the previous tile; a tile of at most two chunks stays resident, copied at its
  first item; every item waits for the go phase of the item two back before arriving), the Y builders
  (released by the accumulator-full commit of the item two back), the epilogue (frees the
  accumulator for the item two ahead; pre-arrives once per buffer) and the MMA issuer (one
  go wait per item, waited before the last k-step of the previous item of the same tile; streamed chunks:
  stage waits for later chunks and a stage release per chunk; resident tiles: the second
  chunk waited on at the tile's first item only).  Checked: every go phase completes with
  the arrivals of exactly one item, the MMA reads the chunk it expects, no copy lands on a
  stage in use, no deadlock; and that dropping the go-phase wait breaks the first rule.
* rf_fft.cu: the two-buffer ring of template spectra: thread 0 copies template t + 1 once all
  groups released template t - 1; groups wait for their template's buffer and release it.
  Checked: every group reads the spectrum it expects, no copy lands on a buffer in use, no
  deadlock.
"""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.arr, self.done, self.log = count, [], 0, []

    def arrive(self, tag=None):
        self.arr.append(tag)
        if len(self.arr) == self.count:
            self.log.append(self.arr)
            self.arr, self.done = [], self.done + 1

    def ok(self, parity):
        return (self.done & 1) != parity


def _schedule(procs, rnd, limit=200000):
    alive = [True] * len(procs)
    steps = 0
    while any(alive):
        steps += 1
        assert steps < limit, "deadlock"
        k = rnd.choice([i for i in range(len(procs)) if alive[i]])
        try:
            next(procs[k])
        except StopIteration:
            alive[k] = False


def _long_kernel(tiles_nch, n_tb, rnd, gate=True):
    items = [(ti, tb) for ti in range(len(tiles_nch)) for tb in range(n_tb)]
    a = rnd.randrange(len(items))
    rng = items[a: rnd.randrange(a, len(items)) + 1]           # one CTA's contiguous range
    n = len(rng)
    AF, AE = [Bar(1), Bar(1)], [Bar(1), Bar(1)]
    GO, DF = [Bar(3), Bar(3)], [Bar(1), Bar(1)]               # go: producer, builders, epilogue
    T0 = [Bar(1), Bar(1)]                                     # chunk 0's own transaction barrier
    TB = Bar(1)                                               # all MMAs before a tile change done
    stage, inuse = [None, None], [0, 0]

    def producer():
        ka, t0u, prev, ntc = 0, [0, 0], None, 0
        for li, (ti, tb) in enumerate(rng):
            first, prev = ti != prev, ti
            nch, b = tiles_nch[ti], li & 1
            if first and li > 0:
                # a new tile: every MMA before it has completed (one phase per tile change)
                while not TB.ok(ntc & 1):
                    yield
                ntc += 1
            if gate and li >= 2:
                # the go phase of item li - 2 has completed before item li's arrival
                while not GO[b].ok(((li >> 1) & 1) ^ 1):
                    yield
            if nch <= 2:
                # resident tile: chunk c in stage c, copied at the tile's first item only
                if first:
                    assert inuse == [0, 0], "copy onto a stage in use"
                    for c in range(nch):
                        stage[c] = (ti, c)
                        if c > 0:
                            AF[1].arrive(li)
                    T0[b].arrive(li)
                    while not T0[b].ok(t0u[b] & 1):
                        yield
                    t0u[b] += 1
                GO[b].arrive(li)
                yield
                continue
            for c in range(nch):
                st, r = ka % 2, ka // 2
                while not AE[st].ok((r & 1) ^ 1):
                    yield
                assert inuse[st] == 0, "copy onto a stage in use"
                stage[st] = (ti, c)
                if c == 0:
                    T0[b].arrive(li)                          # the copy lands
                    while not T0[b].ok(t0u[b] & 1):
                        yield
                    t0u[b] += 1
                    GO[b].arrive(li)
                else:
                    AF[st].arrive(li)
                ka += 1
                yield
        # drain: the last phase armed on every copy barrier has completed
        assert all(T0[b].done == t0u[b] for b in range(2))

    def builders():
        for li in range(n):
            while not DF[li & 1].ok(((li >> 1) & 1) ^ 1):
                yield
            yield
            GO[li & 1].arrive(li)

    def epilogue():
        GO[0].arrive(0)
        GO[1].arrive(1)
        for li in range(n):
            while not DF[li & 1].ok((li >> 1) & 1):
                yield
            yield
            GO[li & 1].arrive(li + 2)

    def mma():
        ka, uf, go_seen, prev = 0, [0, 0], False, None
        for li, (ti, tb) in enumerate(rng):
            first, prev = ti != prev, ti
            nch = tiles_nch[ti]
            resident = nch <= 2
            if not go_seen:
                while not GO[li & 1].ok((li >> 1) & 1):
                    yield
            go_seen = False
            assert GO[li & 1].log[li >> 1] in ([li] * 3,), ("go phase of mixed items", li)
            for c in range(nch):
                st = c if resident else ka % 2
                if c > 0 and (not resident or first):
                    u = uf[st]
                    uf[st] += 1
                    while not AF[st].ok(u & 1):
                        yield
                if c == nch - 1 and li + 1 < n and rng[li + 1][0] == ti:
                    # (only inside a tile: at a tile change the producer waits for this item's
                    # MMAs before its arrival for the next one)
                    while not GO[(li + 1) & 1].ok(((li + 1) >> 1) & 1):
                        yield
                    go_seen = True
                assert stage[st] == (ti, c), "MMA reads the wrong taps chunk"
                inuse[st] = 1
                yield
                if not resident:
                    # a streamed chunk's reads end with the stage's release
                    inuse[st] = 0
                    AE[st].arrive()
                    ka += 1
            # the accumulator-full commit covers every read of the item (resident stages too)
            inuse[0] = inuse[1] = 0
            DF[li & 1].arrive()
            if li + 1 < n and rng[li + 1][0] != ti:
                TB.arrive()
            yield

    _schedule([producer(), builders(), epilogue(), mma()], rnd)


def _fft_ring(counts, groups, rnd):
    full, empty = [Bar(1), Bar(1)], [Bar(groups), Bar(groups)]
    buf, readers = [None, None], [set(), set()]
    seq = [(it, q) for it, c in enumerate(counts) for q in range(c)]

    def group(g):
        tq = 0
        for it, c in enumerate(counts):
            for q in range(c):
                if g == 0:
                    for k in (0, 1) if q == 0 else (1,):
                        if q + k >= c:
                            break
                        t2 = tq + k
                        while not empty[t2 & 1].ok(((t2 >> 1) & 1) ^ 1):
                            yield
                        assert not readers[t2 & 1], "copy onto a buffer in use"
                        buf[t2 & 1] = seq[t2]
                        full[t2 & 1].arrive()
                b = tq & 1
                while not full[b].ok((tq >> 1) & 1):
                    yield
                assert buf[b] == seq[tq], "group reads the wrong spectrum"
                readers[b].add(g)
                yield
                readers[b].discard(g)
                empty[b].arrive()
                tq += 1
                yield

    _schedule([group(g) for g in range(groups)], rnd)


@pytest.mark.parametrize("seed", range(0, 600, 3))
def test_long_kernel_handoffs(seed):
    rnd = random.Random(seed)
    tiles = [rnd.choice([1, 2, 2, 2, 3, 4]) for _ in range(rnd.randrange(1, 5))]
    _long_kernel(tiles, rnd.randrange(1, 12), rnd)


def test_long_kernel_resident_tiles_need_the_go_gate():
    # without the producer's wait on the go phase of item li - 2, a run of resident-tile items
    # lets two items' arrivals meet in one go phase under some interleaving
    failures = 0
    for seed in range(300):
        rnd = random.Random(seed)
        try:
            _long_kernel([2, 2], rnd.randrange(4, 12), rnd, gate=False)
        except AssertionError as e:
            assert "go phase of mixed items" in str(e) or "deadlock" in str(e) or "stage" in str(e)
            failures += 1
    assert failures > 0


@pytest.mark.parametrize("seed", range(0, 600, 3))
def test_block_fft_spectrum_ring(seed):
    rnd = random.Random(seed)
    _fft_ring([rnd.randrange(1, 6) for _ in range(rnd.randrange(1, 6))], 3, rnd)
