"""Host-side model of the pair-band kernel's boundary protocol (no GPU).

Bands of query rows run as a pipeline: band b writes its bottom row, one
64-bit entry per target column, into ring b mod nslots (`window` columns, two
tag bits: lap parity and the ring's generation bit) and band b + 1 reads it,
accepting a block of 16 entries only when every tag matches, then hands the
consumed columns back through a counter every `cons_every` blocks.  A band
writes column j only when the band below has consumed column j - window.
Warp w takes bands w, w + gw, ... in order.

The model runs these rules under random interleavings of the bands' blocks
(each block's writes in two halves, so that a reader can meet a half-written
block) and checks that every accepted entry carries exactly the value the
band above wrote for that column, that no entry is overwritten before it was
consumed, and that the schedule never deadlocks for ring sizes chosen by the
host's rule.  The ring sizes, the hand-back interval and the 63-column lag of
split lanes follow the kernel's constants; the payload of an entry is
(band, column) instead of (H, F).
"""

import random

import pytest

COL = 16  # columns per block


def host_window(npad, gw, ring_columns=0):
    """Ring columns and hand-back interval as the host sizes them."""
    window = ring_columns or 32768
    ceil_div = (npad + gw - 1) // gw
    rule = (((ceil_div + 64) * 8 // 7 + 1) + COL - 1) // COL * COL
    window = min(max(window, rule), npad)
    cons_every = max(1, min(16, window // COL // 8))
    return window, cons_every


def gen_bit(b, nslots):
    return ((b // nslots) & 1) ^ 1


class Band:
    def __init__(self, b, sim):
        self.b, self.sim = b, sim
        self.prev, self.next = b > 0, b + 1 < sim.nbands
        self.blk = 0
        self.half = 0          # 0: room check + first half of writes, 1: second half + land
        self.landed = 0        # blocks of the band above copied in
        self.since = 0
        self.rpos, self.rlap = 0, 0
        self.wpos, self.wlap = 0, 0
        self.t_done = False
        self.started_first = False

    def ring_in(self):
        return (self.b - 1) % self.sim.nslots

    def ring_out(self):
        return self.b % self.sim.nslots

    def try_land(self):
        """Accept the next block of the band above if all 16 entries are fresh."""
        s = self.sim
        base = self.ring_in() * s.window
        want_gen = gen_bit(self.b - 1, s.nslots)
        entries = [s.mem[base + self.rpos + i] for i in range(COL)]
        if not all(e is not None and e[0] == self.rlap and e[1] == want_gen for e in entries):
            return False
        for i, e in enumerate(entries):
            col = self.landed * COL + i
            assert e[2] == (self.b - 1, col), f"band {self.b} read {e[2]} for column {col}"
        self.landed += 1
        s.consumed_true[self.b - 1] = self.landed * COL
        self.rpos += COL
        if self.rpos == s.window:
            self.rpos, self.rlap = 0, self.rlap ^ 1
        self.since += 1
        if self.since == s.cons_every or self.landed * COL == s.npad:
            self.since = 0
            s.cons_pub[self.b - 1] = self.landed * COL
        return True

    def write(self, t0, t1):
        s = self.sim
        base = self.ring_out() * s.window
        for t in range(t0, t1):
            j = t - s.lag
            if 0 <= j < s.npad:
                old = s.mem[base + self.wpos]
                if old is not None and old[2][0] + 1 < s.nbands:
                    ob, oj = old[2]
                    assert s.consumed_true[ob] > oj, f"band {self.b} overwrote unread column {oj} of band {ob}"
                s.mem[base + self.wpos] = (self.wlap, gen_bit(self.b, s.nslots), (self.b, j))
                self.wpos += 1
                if self.wpos == s.window:
                    self.wpos, self.wlap = 0, self.wlap ^ 1

    def step(self):
        """One action; False when blocked."""
        s = self.sim
        if not self.started_first:
            if self.prev and not self.try_land():
                return False
            self.started_first = True
            return True
        blk = self.blk
        if self.half == 0:
            if self.next:
                jmax = min(blk * COL + COL - 1 - s.lag, s.npad - 1)
                need = jmax + 1 - s.window
                if jmax >= 0 and s.cons_pub[self.b] < need:
                    return False
            self.write(blk * COL, blk * COL + COL // 2)
            self.half = 1
            return True
        if self.half == 1:
            self.write(blk * COL + COL // 2, blk * COL + COL)
            self.half = 2
            return True
        # end of the block: land the next block of the band above
        if self.prev and blk + 1 < s.nreal and not self.try_land():
            return False
        self.half = 0
        self.blk += 1
        if self.blk == s.nblk:
            self.t_done = True
        return True


class Sim:
    def __init__(self, npad, nbands, gw, lag, ring_columns, seed):
        self.npad, self.nbands, self.gw, self.lag = npad, nbands, gw, lag
        self.nslots = min(nbands, gw + 1)
        self.window, self.cons_every = host_window(npad, gw, ring_columns)
        self.nreal = npad // COL
        self.nblk = (npad + lag + COL - 1) // COL
        self.mem = [None] * (self.nslots * self.window)   # zeroed rings: no valid entry
        self.cons_pub = [0] * nbands
        self.consumed_true = [0] * nbands
        self.rng = random.Random(seed)

    def run(self):
        queues = [[b for b in range(self.nbands) if b % self.gw == w] for w in range(self.gw)]
        current = {w: Band(q[0], self) for w, q in enumerate(queues) if q}
        done = 0
        while done < self.nbands:
            ws = list(current)
            self.rng.shuffle(ws)
            moved = False
            for w in ws:
                band = current[w]
                if band.step():
                    moved = True
                    if band.t_done:
                        done += 1
                        queues[w].pop(0)
                        if queues[w]:
                            current[w] = Band(queues[w][0], self)
                        else:
                            del current[w]
                    break
            assert moved, f"deadlock with {done} of {self.nbands} bands done"
        # every band's last block was read by the band below
        for b in range(self.nbands - 1):
            assert self.consumed_true[b] == self.npad


@pytest.mark.parametrize("npad,nbands,gw,ring", [
    (16, 3, 1, 0), (48, 5, 2, 0), (256, 7, 3, 0), (1008, 13, 4, 256), (1008, 40, 8, 256),
    (2000, 9, 2, 256), (4096, 24, 5, 0), (1600, 30, 3, 512)])
@pytest.mark.parametrize("lag", [31, 63])
def test_band_protocol(npad, nbands, gw, ring, lag):
    for seed in range(3):
        Sim(npad, nbands, gw, lag, ring, seed=1000 * seed + npad + nbands).run()


def test_generation_bits_differ_between_ring_users():
    # bands b and b + nslots share a ring; their generation bits differ, and
    # generation 0 never writes the zeroed rings' bit
    for nslots in (1, 2, 5, 9):
        for b in range(40):
            assert gen_bit(b, nslots) != gen_bit(b + nslots, nslots)
        assert gen_bit(0, nslots) == 1
