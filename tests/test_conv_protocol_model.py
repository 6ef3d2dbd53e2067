"""CPU model of the conv kernel's barrier protocol (k_conv_tc), run under random
interleavings.  compute-sanitizer is closed on the GPU pool, so the pipeline's ordering
argument is checked here instead, on a faithful model of its synchronisation:

* one or more producer warps that stage each unit's nrows + 2 input rows in a ring of NSLOT
  slots, taking the ring rows in turn (NSLOT is a multiple of their number, so a slot always
  has the same producer; with as many producers as slots this is the layer-1 kernel whose
  input warps each build the rows of one slot): wait `empty`, write the row record, copies landing asynchronously on
  `full`; then the end-of-work marker (from the warp whose turn it is), then a drain that
  waits for the warp's own newest copy in each of its slots;
* the MMA issuer: waits `full` for each row, reads the record at a unit's start, waits the
  accumulator-release barrier `bfree[k]` before block k's first MMA, queues the row's MMAs
  and commits (`empty` for the slot, `bfull[k - 2]` for the completed block), and gives the
  blocks a short unit leaves unused one release-wait + commit round;
* the tensor pipe, completing MMAs and commits in issue order after random delays;
* eight epilogue warps in two groups (blocks g, g + 2, ...), each waiting `bfull`, reading
  and zeroing its TMEM lane quarter, and arriving on `bfree` (four arrivals per block).

Barriers follow mbarrier parity semantics: a wait on parity q returns once the barrier's
current phase has parity != q, so a waiter that falls two phases behind stalls.  Checked:
no deadlock; every wait returns on exactly the phase it means; a slot is overwritten only
after the MMAs that read it completed and read only after its copy landed; a TMEM block is
accumulated into only after all four of its epilogue warps drained and zeroed it; a block
is drained only after its three contributing rows' MMAs completed.  Two earlier protocol
bugs are kept as variants that the model must catch."""
import random

import pytest

NSLOT = 6


class Bar:
    def __init__(self, name, count):
        self.name, self.count, self.pending, self.phases = name, count, count, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0, f"{self.name}: too many arrivals"
        if self.pending == 0:
            self.phases += 1
            self.pending = self.count

    def done(self, parity):
        return parity != (self.phases & 1)


class Violation(AssertionError):
    pass


def wait(bar, phase):
    """Generator: wait for completion of phase `phase` (0-based; -1 = the phase before the
    first, complete from the start) by its parity, then check it was exactly that phase."""
    parity = phase & 1
    while not bar.done(parity):
        yield lambda: bar.done(parity)              # blocked until this holds
    if bar.phases != phase + 1:
        raise Violation(f"{bar.name}: waited for phase {phase}, barrier at {bar.phases} completed phases")


class Sim:
    """One CTA's conv pipeline over a list of units (output rows per unit), scheduled at random."""

    def __init__(self, units, ru, rng, variant=None, nprod=1):
        self.units, self.ru, self.rng, self.variant, self.nprod = units, ru, rng, variant, nprod
        self.full = [Bar(f"full[{s}]", 1) for s in range(NSLOT)]
        self.empty = [Bar(f"empty[{s}]", 1) for s in range(NSLOT)]
        self.wbar, self.drain = Bar("wbar", 1), Bar("drain", 1)
        self.bfull = [Bar(f"bfull[{j}]", 1) for j in range(ru)]
        self.bfree = [Bar(f"bfree[{j}]", 4) for j in range(ru)]
        self.meta = [None] * NSLOT
        self.slot_row = [None] * NSLOT          # ring index of the row staged in the slot
        self.slot_landed = [False] * NSLOT
        self.slot_readers = [0] * NSLOT         # queued MMAs reading the slot, not yet completed
        self.pipe = []                          # tensor pipe, in issue order
        self.copies = [("w",)]                  # copies in flight (they land in any order)
        self.blk_unit = [-1] * ru               # unit whose sums the block holds
        self.blk_rows = [0] * ru                # its contributing rows completed so far
        self.blk_zeroed = [4] * ru              # epilogue warps that drained + zeroed it (4 = free)
        # relative speeds of this run: a slow epilogue, tensor pipe or copy engine lets the
        # other roles run as far ahead as the barriers allow
        self.speed = {k: rng.choice([1.0, 0.2, 0.03]) for k in ("epilogue", "#pipe", "#copy")}

    def _mine(self, p, li):
        # the "shared_turns" fault: both warps stage every row
        return self.variant == "shared_turns" or li % self.nprod == p

    def producer(self, p=0):
        li = 0
        last = [-1] * NSLOT
        for nrows in self.units:
            for r in range(nrows + 2):
                if not self._mine(p, li):               # the other warp's turn
                    li += 1
                    continue
                slot, rnd = li % NSLOT, li // NSLOT
                yield from wait(self.empty[slot], rnd - 1)
                if self.slot_readers[slot]:
                    raise Violation(f"slot {slot} overwritten while MMAs still read it")
                self.meta[slot] = (r, nrows)
                self.slot_row[slot], self.slot_landed[slot] = li, False
                if self.rng.random() < 0.25:            # a halo row: zero-filled, arrive at once
                    self.slot_landed[slot] = True
                    self.full[slot].arrive()
                else:
                    self.copies.append((slot, li))
                last[slot] = li
                li += 1
                yield None
        if self._mine(p, li):
            slot, rnd = li % NSLOT, li // NSLOT          # end-of-work marker
            yield from wait(self.empty[slot], rnd - 1)
            self.meta[slot] = (-1, 0)
            self.slot_row[slot], self.slot_landed[slot] = li, True
            self.full[slot].arrive()
            if self.variant != "marker_not_recorded":
                last[slot] = li
        for s in range(NSLOT):                            # drain: own newest phase of each of its slots
            if last[s] >= 0:
                yield from wait(self.full[s], last[s] // NSLOT)

    def mma(self):
        yield from wait(self.wbar, 0)
        li, uit, start, k, nrows = 0, 0, True, 0, 0
        while True:
            slot, rnd = li % NSLOT, li // NSLOT
            yield from wait(self.full[slot], rnd)
            if not self.slot_landed[slot] or self.slot_row[slot] != li:
                raise Violation(f"row {li} read before it landed")
            if start:
                k, nrows = self.meta[slot]
                if k < 0:
                    break
                start = False
            if k < nrows:
                yield from wait(self.bfree[k], uit)
                if self.blk_zeroed[k] != 4:
                    raise Violation(f"block {k} accumulated before all its epilogue warps drained it")
                self.blk_zeroed[k], self.blk_unit[k], self.blk_rows[k] = 0, uit, 0
            blocks = list(range(max(0, k - 2), min(nrows - 1, k) + 1))
            self.slot_readers[slot] += 1
            self.pipe.append(("mma", slot, uit, blocks))
            self.pipe.append(("commit", self.empty[slot]))
            if k >= 2:
                self.pipe.append(("commit", self.bfull[k - 2]))
            li += 1
            yield None
            if k == nrows + 1:
                for j in range(nrows, self.ru):           # unused blocks: one release / commit round
                    if self.variant != "skip_unused_wait":
                        yield from wait(self.bfree[j], uit)
                    self.pipe.append(("commit", self.bfull[j]))
                uit, start = uit + 1, True
            else:
                k += 1
        self.pipe.append(("commit", self.drain))
        yield from wait(self.drain, 0)

    def epilogue(self, g):
        for j in range(g, self.ru, 2):                   # blocks start zeroed and free
            self.bfree[j].arrive()
            yield None
        for uit, nrows in enumerate(self.units):
            for j in range(g, self.ru, 2):
                yield from wait(self.bfull[j], uit)
                if j < nrows:
                    if self.blk_unit[j] != uit or self.blk_rows[j] != 3:
                        raise Violation(f"block {j} of unit {uit} drained before its three rows completed")
                    yield None                             # TMEM read and zeroing of this warp's quarter
                    self.blk_zeroed[j] += 1
                self.bfree[j].arrive()
                yield None

    def step_pipe(self):
        op = self.pipe.pop(0)
        if op[0] == "commit":
            op[1].arrive()
            return
        _, slot, uit, blocks = op
        for j in blocks:
            if self.blk_unit[j] != uit:
                raise Violation(f"MMA of unit {uit} landed in block {j} held by unit {self.blk_unit[j]}")
            self.blk_rows[j] += 1
        self.slot_readers[slot] -= 1

    def step_copy(self):
        c = self.copies.pop(self.rng.randrange(len(self.copies)))
        if c[0] == "w":
            self.wbar.arrive()
            return
        slot, li = c
        assert self.slot_row[slot] == li
        self.slot_landed[slot] = True
        self.full[slot].arrive()

    def _procs(self):
        procs = {f"producer{p}": self.producer(p) for p in range(self.nprod)}
        procs["mma"] = self.mma()
        for g in range(2):
            for q in range(4):
                procs[f"epilogue{g}.{q}"] = self.epilogue(g)
        return procs

    def run(self):
        procs = self._procs()
        blocked = dict.fromkeys(procs)
        for _ in range(10 ** 6):
            if not procs and not self.pipe and not self.copies:
                return
            cands = [n for n in procs if blocked[n] is None or blocked[n]()]
            if self.pipe:
                cands.append("#pipe")
            if self.copies:
                cands.append("#copy")
            if not cands:
                raise Violation(f"deadlock: {sorted(procs)} wait forever")
            weights = [self.speed.get("epilogue" if n.startswith("epilogue") else n, 1.0) for n in cands]
            c = self.rng.choices(cands, weights)[0]
            if c == "#pipe":
                self.step_pipe()
            elif c == "#copy":
                self.step_copy()
            else:
                try:
                    blocked[c] = next(procs[c])
                except StopIteration:
                    del procs[c], blocked[c]
        raise AssertionError("simulation did not finish")


def _units(rng, ru):
    """A CTA's units: mostly full, with short ones (image bottoms, small images) and runs of
    consecutive short units."""
    n = rng.randint(1, 9)
    return [ru if rng.random() < 0.4 else rng.randint(1, ru) for _ in range(n)]


# (8, 8): the layer-1 kernel that builds its input, one input warp per ring slot
@pytest.mark.parametrize("nslot,nprod", [(6, 1), (6, 2), (8, 2), (8, 4), (8, 8)])
@pytest.mark.parametrize("ru", [3, 4, 5, 6, 7, 8])
def test_conv_pipeline_protocol_holds(ru, nslot, nprod, monkeypatch):
    monkeypatch.setattr(__import__(__name__), "NSLOT", nslot)
    rng = random.Random(1000 + ru)
    for trial in range(60):
        units = _units(rng, ru)
        Sim(units, ru, random.Random(rng.random()), nprod=nprod).run()


def test_model_catches_producers_not_owning_their_slots(monkeypatch):
    """Four producers on a ring of 6: a slot then passes between producers, and one can wait
    on a phase of it two phases ahead of the barrier (its parity is then already complete)."""
    monkeypatch.setattr(__import__(__name__), "NSLOT", 6)
    rng = random.Random(23)
    caught = 0
    for trial in range(60):
        try:
            Sim(_units(rng, 8), 8, random.Random(rng.random()), nprod=4).run()
        except (Violation, AssertionError):
            caught += 1
    assert caught >= 5, caught


def test_model_catches_two_producers_staging_the_same_rows():
    """Two producer warps that do not take turns: both stage every row into its slot."""
    rng = random.Random(17)
    caught = 0
    for trial in range(40):
        try:
            Sim(_units(rng, 8), 8, random.Random(rng.random()), "shared_turns", nprod=2).run()
        except (Violation, AssertionError):
            caught += 1
    assert caught >= 20, caught


@pytest.mark.parametrize("variant", ["skip_unused_wait", "marker_not_recorded"])
def test_model_catches_the_earlier_protocol_bugs(variant):
    """The two faults found on the GPU (both reported by the bounded waits' timeout record):
    committing a short unit's unused blocks without waiting for their release (two short
    units in a row run a block two phases ahead), and a drain that did not count the end
    marker as its slot's newest phase."""
    rng = random.Random(7)
    caught = 0
    for trial in range(60):
        units = [rng.randint(1, 2) for _ in range(rng.randint(3, 8))] if variant == "skip_unused_wait" \
            else _units(rng, 8)
        try:
            Sim(units, 8, random.Random(rng.random()), variant).run()
        except Violation:
            caught += 1
    assert caught >= 5, caught


# ---------------------------------------------------------------------------
# Row-streaming form of the conv pipeline (tall work units, TMEM blocks as a ring).  A
# unit is a strip of nrows output rows (tens to hundreds); output row G of the CTA (G
# counts the output rows of all its strips so far) accumulates in block G % 8, guarded by
# bfull / bfree[G % 8] at phase G // 8.  The MMA of a staged row covers output rows
# jlo .. jhi starting at block (G0 + jlo) % 8; where that window passes block 7 it is
# issued as two MMAs (blocks p .. 7, then 0 ..), so every row keeps one block.  Epilogue
# group g owns the rows with G % 2 == g (the blocks of its parity).
# ---------------------------------------------------------------------------
NRING = 8


class StreamSim(Sim):
    def __init__(self, units, rng, variant=None, nprod=2):
        super().__init__(units, 8, rng, variant, nprod)
        self.blk_row = [-1] * NRING               # global row whose sum the block holds
        self.row_contrib = {}                     # global row -> staged-row contributions completed

    def mma(self):
        yield from wait(self.wbar, 0)
        li, start, k, nrows, g0 = 0, True, 0, 0, 0
        while True:
            slot, rnd = li % NSLOT, li // NSLOT
            yield from wait(self.full[slot], rnd)
            if not self.slot_landed[slot] or self.slot_row[slot] != li:
                raise Violation(f"row {li} read before it landed")
            if start:
                k, nrows = self.meta[slot]
                if k < 0:
                    break
                start = False
            if k < nrows:
                g = g0 + k
                yield from wait(self.bfree[g % NRING], g // NRING)
                if self.blk_zeroed[g % NRING] != 4:
                    raise Violation(f"block {g % NRING} accumulated before its epilogue warps drained it")
                self.blk_zeroed[g % NRING], self.blk_row[g % NRING] = 0, g
                self.row_contrib[g] = 0
            jlo, jhi = max(0, k - 2), min(nrows - 1, k)
            p, r = (g0 + jlo) % NRING, jhi - jlo + 1
            r1 = r if self.variant == "stream_no_split" else min(r, NRING - p)
            parts = [(p, list(range(jlo, jlo + r1)))]
            if r1 < r:
                parts.append((0, list(range(jlo + r1, jhi + 1))))
            for b0, js in parts:
                if b0 + len(js) > NRING:
                    raise Violation(f"MMA window of blocks {b0} .. {b0 + len(js) - 1} leaves TMEM")
                rows = [g0 + j for j in js]
                for i, gr in enumerate(rows):
                    if b0 + i != gr % NRING:
                        raise Violation(f"row {gr} accumulated in block {b0 + i}")
                self.slot_readers[slot] += 1
                self.pipe.append(("smma", slot, [(b0 + i, gr) for i, gr in enumerate(rows)]))
            self.pipe.append(("commit", self.empty[slot]))
            if k >= 2:
                self.pipe.append(("commit", self.bfull[(g0 + k - 2) % NRING]))
            li += 1
            yield None
            if k == nrows + 1:
                g0 += nrows
                start = True
            else:
                k += 1
        self.pipe.append(("commit", self.drain))
        yield from wait(self.drain, 0)

    def epilogue(self, grp):
        for b in range(grp, NRING, 2):            # blocks start zeroed and free
            self.bfree[b].arrive()
            yield None
        g0 = 0
        for nrows in self.units:
            for j in range(nrows):
                g = j if self.variant == "stream_ring_restarts" else g0 + j
                if g % 2 != grp:
                    continue
                yield from wait(self.bfull[g % NRING], g // NRING)
                if self.blk_row[g % NRING] != g or self.row_contrib.get(g) != 3:
                    raise Violation(f"row {g} drained before its three staged rows completed")
                yield None                         # TMEM read and zeroing of this warp's quarter
                self.blk_zeroed[g % NRING] += 1
                self.bfree[g % NRING].arrive()
                yield None
            g0 += nrows

    def step_pipe(self):
        if self.pipe[0][0] == "smma":
            _, slot, blocks = self.pipe.pop(0)
            for b, gr in blocks:
                if self.blk_row[b] != gr:
                    raise Violation(f"MMA for row {gr} landed in block {b}, which holds row {self.blk_row[b]}")
                self.row_contrib[gr] += 1
            self.slot_readers[slot] -= 1
            return
        super().step_pipe()


def _tall_units(rng):
    """Strips of a CTA: tall ones, image bottoms of any height, tiny images."""
    n = rng.randint(1, 6)
    return [rng.choice([rng.randint(1, 5), rng.randint(6, 40), 64]) for _ in range(n)]


@pytest.mark.parametrize("nslot,nprod", [(6, 1), (6, 2), (8, 2), (8, 4), (8, 8)])
def test_stream_protocol_holds(nslot, nprod, monkeypatch):
    monkeypatch.setattr(__import__(__name__), "NSLOT", nslot)
    rng = random.Random(4242)
    for trial in range(150):
        StreamSim(_tall_units(rng), random.Random(rng.random()), nprod=nprod).run()


@pytest.mark.parametrize("variant", ["stream_no_split", "stream_ring_restarts"])
def test_stream_model_catches_protocol_faults(variant):
    """A window issued as one MMA where it passes block 7 (it would leave TMEM's 512
    columns), and an epilogue that restarts the ring at every strip instead of carrying the
    CTA's row count across strips."""
    rng = random.Random(99)
    caught = 0
    for trial in range(60):
        try:
            StreamSim(_tall_units(rng), random.Random(rng.random()), variant).run()
        except Violation:
            caught += 1
    assert caught >= 10, caught


# ---------------------------------------------------------------------------
# Weight-gradient kernel (k_wgrad_tc): an activation-row ring (NSA slots) and a
# gradient-row ring (NSG slots).  Per unit of nrows gradient rows the MMA warp needs
# activation rows base .. base + nrows + 1; gradient row j pairs with activation rows
# base + j .. base + j + 2 (the second half of the dy-2 tile also reads base + j + 3 into
# TMEM lanes that are never read back, so that read is not a dependence).  A gradient
# slot is released by the MMA commit and by the four bias-sum warps (count 5).
# ---------------------------------------------------------------------------
WG_NSA, WG_NSG = 8, 4


class WgSim:
    def __init__(self, units, rng, variant=None):
        self.units, self.rng, self.variant = units, rng, variant
        g_count = 1 if variant == "g_release_mma_only" else 5
        self.a_full = [Bar(f"a_full[{s}]", 1) for s in range(WG_NSA)]
        self.a_empty = [Bar(f"a_empty[{s}]", 1) for s in range(WG_NSA)]
        self.g_full = [Bar(f"g_full[{s}]", 1) for s in range(WG_NSG)]
        self.g_empty = [Bar(f"g_empty[{s}]", g_count) for s in range(WG_NSG)]
        self.tzero, self.done = Bar("tzero", 4), Bar("done", 1)
        self.a_meta, self.g_meta = [None] * WG_NSA, [None] * WG_NSG
        self.a_row, self.g_row = [None] * WG_NSA, [None] * WG_NSG
        self.a_landed, self.g_landed = [False] * WG_NSA, [False] * WG_NSG
        self.a_readers, self.g_readers = [0] * WG_NSA, [0] * WG_NSG
        self.g_epi_reads = [0] * WG_NSG          # bias-sum warps still to read the slot's row
        self.pipe, self.copies = [], []
        self.speed = {k: rng.choice([1.0, 0.2, 0.03]) for k in ("epilogue", "#pipe", "#copy")}

    def _stage(self, full, row, landed, meta, slot, li, rec, async_ok=True):
        meta[slot] = rec
        row[slot], landed[slot] = li, False
        if async_ok and self.rng.random() < 0.75:
            self.copies.append((full, row, landed, slot, li))
        else:
            landed[slot] = True
            full[slot].arrive()

    def producer(self):
        la = lg = 0
        a_last, g_last = [-1] * WG_NSA, [-1] * WG_NSG
        for nrows in self.units:
            for r in range(nrows + 2):
                sa = la % WG_NSA
                yield from wait(self.a_empty[sa], la // WG_NSA - 1)
                if self.a_readers[sa]:
                    raise Violation(f"activation slot {sa} overwritten while MMAs read it")
                self._stage(self.a_full, self.a_row, self.a_landed, self.a_meta, sa, la, (r, nrows))
                a_last[sa] = la
                la += 1
                yield None
                if r < 2:
                    continue
                sg = lg % WG_NSG
                yield from wait(self.g_empty[sg], lg // WG_NSG - 1)
                if self.g_readers[sg] or self.g_epi_reads[sg]:
                    raise Violation(f"gradient slot {sg} overwritten while it is still read")
                self._stage(self.g_full, self.g_row, self.g_landed, self.g_meta, sg, lg, (r - 2, nrows))
                self.g_epi_reads[sg] = 4
                g_last[sg] = lg
                lg += 1
                yield None
        sa, sg = la % WG_NSA, lg % WG_NSG                  # end markers on both rings
        yield from wait(self.a_empty[sa], la // WG_NSA - 1)
        yield from wait(self.g_empty[sg], lg // WG_NSG - 1)
        self._stage(self.a_full, self.a_row, self.a_landed, self.a_meta, sa, la, (-1, 0), async_ok=False)
        self._stage(self.g_full, self.g_row, self.g_landed, self.g_meta, sg, lg, (-1, 0), async_ok=False)
        a_last[sa], g_last[sg] = la, lg
        for s in range(WG_NSA):
            if a_last[s] >= 0:
                yield from wait(self.a_full[s], a_last[s] // WG_NSA)
        for s in range(WG_NSG):
            if g_last[s] >= 0:
                yield from wait(self.g_full[s], g_last[s] // WG_NSG)

    def _need_a(self, q):
        s = q % WG_NSA
        if not self.a_landed[s] or self.a_row[s] != q:
            raise Violation(f"activation row {q} read before it landed")
        return s

    def mma(self):
        yield from wait(self.tzero, 0)
        qa = qg = 0
        while True:
            base = qa
            yield from wait(self.a_full[base % WG_NSA], base // WG_NSA)
            k0, nrows = self.a_meta[base % WG_NSA]
            if k0 < 0:
                break
            yield from wait(self.a_full[(base + 1) % WG_NSA], (base + 1) // WG_NSA)
            for j in range(nrows):
                qn = base + j + 2
                yield from wait(self.a_full[qn % WG_NSA], qn // WG_NSA)
                yield from wait(self.g_full[qg % WG_NSG], qg // WG_NSG)
                sg = qg % WG_NSG
                if not self.g_landed[sg] or self.g_row[sg] != qg:
                    raise Violation(f"gradient row {qg} read before it landed")
                slots = [self._need_a(base + j + d) for d in range(3)]
                for s in slots:
                    self.a_readers[s] += 1
                self.g_readers[sg] += 1
                self.pipe.append(("mma", slots, sg))
                self.pipe.append(("commit", self.g_empty[sg]))
                self.pipe.append(("commit", self.a_empty[(base + j) % WG_NSA]))
                qg += 1
                yield None
            self.pipe.append(("commit", self.a_empty[(base + nrows) % WG_NSA]))
            self.pipe.append(("commit", self.a_empty[(base + nrows + 1) % WG_NSA]))
            qa = base + nrows + 2
        self.pipe.append(("commit", self.done))

    def epilogue(self):
        self.tzero.arrive()
        yield None
        qg = 0
        while True:
            sg = qg % WG_NSG
            yield from wait(self.g_full[sg], qg // WG_NSG)
            if self.g_meta[sg][0] < 0:
                break
            if not self.g_landed[sg] or self.g_row[sg] != qg:
                raise Violation(f"bias sums read gradient row {qg} before it landed")
            yield None                                     # the bias sums read the row
            if self.g_row[sg] != qg:
                raise Violation(f"gradient row {qg} overwritten while the bias sums read it")
            self.g_epi_reads[sg] -= 1
            if self.variant != "g_release_mma_only":
                self.g_empty[sg].arrive()
            qg += 1
            yield None
        yield from wait(self.done, 0)

    def step_pipe(self):
        op = self.pipe.pop(0)
        if op[0] == "commit":
            op[1].arrive()
            return
        _, slots, sg = op
        for s in slots:
            self.a_readers[s] -= 1
        self.g_readers[sg] -= 1

    def step_copy(self):
        full, row, landed, slot, li = self.copies.pop(self.rng.randrange(len(self.copies)))
        assert row[slot] == li
        landed[slot] = True
        full[slot].arrive()

    run = Sim.run

    def _procs(self):
        procs = {"producer": self.producer(), "mma": self.mma()}
        for q in range(4):
            procs[f"epilogue.{q}"] = self.epilogue()
        return procs


def test_wgrad_pipeline_protocol_holds():
    rng = random.Random(2024)
    for trial in range(150):
        units = [rng.choice([8, 8, rng.randint(1, 8)]) for _ in range(rng.randint(1, 7))]
        WgSim(units, random.Random(rng.random())).run()


def test_wgrad_model_catches_a_gradient_slot_released_by_the_mma_alone():
    """If the gradient ring's slots were released by the MMA commit alone, the producer
    could refill a slot the bias-sum warps are still reading."""
    rng = random.Random(5)
    caught = 0
    for trial in range(60):
        units = [rng.randint(1, 8) for _ in range(rng.randint(2, 7))]
        try:
            WgSim(units, random.Random(rng.random()), "g_release_mma_only").run()
        except Violation:
            caught += 1
    assert caught >= 5, caught


# ---------------------------------------------------------------------------
# CTA-pair form (k_conv_tc2, cluster of two CTAs, M = 256).  Each CTA stages its own
# 128-pixel half of every row in its own ring; the second CTA's relay warp forwards "my
# weights / my row landed" (and the end marker) to the first CTA's pwbar / pfull by
# remote arrives; the first CTA's MMA warp waits on both, reads both CTAs' slots and
# accumulates into both CTAs' TMEM blocks; its commits arrive on the barrier of both
# CTAs (multicast); the epilogue warps of both CTAs release blocks on the first CTA's
# bfree (8 arrivals).
# ---------------------------------------------------------------------------
class Ring:
    def __init__(self, cta):
        self.full = [Bar(f"cta{cta}.full[{s}]", 1) for s in range(NSLOT)]
        self.empty = [Bar(f"cta{cta}.empty[{s}]", 1) for s in range(NSLOT)]
        self.meta = [None] * NSLOT
        self.row = [None] * NSLOT
        self.landed = [False] * NSLOT
        self.readers = [0] * NSLOT


class PairSim:
    def __init__(self, units, ru, rng, variant=None):
        self.units, self.ru, self.rng, self.variant = units, ru, rng, variant
        self.ring = [Ring(0), Ring(1)]
        self.wbar = [Bar("cta0.wbar", 1), Bar("cta1.wbar", 1)]
        self.pwbar = Bar("cta0.pwbar", 1)
        self.pfull = [Bar(f"cta0.pfull[{s}]", 1) for s in range(NSLOT)]
        self.drain = [Bar("cta0.drain", 1), Bar("cta1.drain", 1)]
        self.bfull = [[Bar(f"cta{c}.bfull[{j}]", 1) for j in range(ru)] for c in range(2)]
        self.bfree = [Bar(f"cta0.bfree[{j}]", 8) for j in range(ru)]
        self.blk_unit = [[-1] * ru for _ in range(2)]
        self.blk_rows = [[0] * ru for _ in range(2)]
        self.blk_zeroed = [[4] * ru for _ in range(2)]
        self.pipe, self.copies = [], [("w", 0), ("w", 1)]
        self.speed = {k: rng.choice([1.0, 0.2, 0.03]) for k in ("epilogue", "#pipe", "#copy", "relay")}

    def producer(self, c):
        R = self.ring[c]
        li = 0
        last = [-1] * NSLOT
        for nrows in self.units:
            for r in range(nrows + 2):
                slot, rnd = li % NSLOT, li // NSLOT
                yield from wait(R.empty[slot], rnd - 1)
                if R.readers[slot]:
                    raise Violation(f"cta{c} slot {slot} overwritten while MMAs still read it")
                R.meta[slot] = (r, nrows)
                R.row[slot], R.landed[slot] = li, False
                if self.rng.random() < 0.25:
                    R.landed[slot] = True
                    R.full[slot].arrive()
                else:
                    self.copies.append(("row", c, slot, li))
                last[slot] = li
                li += 1
                yield None
        slot, rnd = li % NSLOT, li // NSLOT
        yield from wait(R.empty[slot], rnd - 1)
        R.meta[slot] = (-1, 0)
        R.row[slot], R.landed[slot] = li, True
        R.full[slot].arrive()
        if self.variant != "marker_not_recorded":
            last[slot] = li
        for s in range(NSLOT):
            if last[s] >= 0:
                yield from wait(R.full[s], last[s] // NSLOT)
        yield from wait(self.wbar[c], 0)

    def relay(self):
        R = self.ring[1]
        yield from wait(self.wbar[1], 0)
        self.pwbar.arrive()
        q = 0
        while True:
            slot = q % NSLOT
            yield from wait(R.full[slot], q // NSLOT)
            k = R.meta[slot][0]
            if k < 0 and self.variant == "relay_drops_marker":
                break
            self.pfull[slot].arrive()
            yield None
            if k < 0:
                break
            q += 1
        yield from wait(self.drain[1], 0)

    def mma(self):
        yield from wait(self.wbar[0], 0)
        yield from wait(self.pwbar, 0)
        li, uit, start, k, nrows = 0, 0, True, 0, 0
        while True:
            slot, rnd = li % NSLOT, li // NSLOT
            yield from wait(self.ring[0].full[slot], rnd)
            yield from wait(self.pfull[slot], rnd)
            if start:
                k, nrows = self.ring[0].meta[slot]
                if k < 0:
                    break
                start = False
            for c in range(2):
                R = self.ring[c]
                if not R.landed[slot] or R.row[slot] != li:
                    raise Violation(f"cta{c} row {li} read before it landed")
            if k < nrows:
                yield from wait(self.bfree[k], uit)
                for c in range(2):
                    if self.blk_zeroed[c][k] != 4:
                        raise Violation(f"cta{c} block {k} accumulated before its epilogue warps drained it")
                    self.blk_zeroed[c][k], self.blk_unit[c][k], self.blk_rows[c][k] = 0, uit, 0
            blocks = list(range(max(0, k - 2), min(nrows - 1, k) + 1))
            for c in range(2):
                self.ring[c].readers[slot] += 1
            self.pipe.append(("mma", slot, uit, blocks))
            # commits are multicast: they arrive on the barrier of both CTAs
            self.pipe.append(("commit", [self.ring[0].empty[slot], self.ring[1].empty[slot]]))
            if k >= 2:
                self.pipe.append(("commit", [self.bfull[0][k - 2], self.bfull[1][k - 2]]))
            li += 1
            yield None
            if k == nrows + 1:
                for j in range(nrows, self.ru):
                    yield from wait(self.bfree[j], uit)
                    self.pipe.append(("commit", [self.bfull[0][j], self.bfull[1][j]]))
                uit, start = uit + 1, True
            else:
                k += 1
        self.pipe.append(("commit", list(self.drain)))
        yield from wait(self.drain[0], 0)

    def epilogue(self, c, g):
        for j in range(g, self.ru, 2):
            self.bfree[j].arrive()                         # the second CTA's arrive is remote
            yield None
        for uit, nrows in enumerate(self.units):
            for j in range(g, self.ru, 2):
                yield from wait(self.bfull[c][j], uit)
                if j < nrows:
                    if self.blk_unit[c][j] != uit or self.blk_rows[c][j] != 3:
                        raise Violation(f"cta{c} block {j} of unit {uit} drained before its rows completed")
                    yield None
                    self.blk_zeroed[c][j] += 1
                self.bfree[j].arrive()
                yield None

    def step_pipe(self):
        op = self.pipe.pop(0)
        if op[0] == "commit":
            for b in op[1]:
                b.arrive()
            return
        _, slot, uit, blocks = op
        for c in range(2):
            for j in blocks:
                if self.blk_unit[c][j] != uit:
                    raise Violation(f"MMA of unit {uit} landed in cta{c} block {j} held by unit {self.blk_unit[c][j]}")
                self.blk_rows[c][j] += 1
            self.ring[c].readers[slot] -= 1

    def step_copy(self):
        cp = self.copies.pop(self.rng.randrange(len(self.copies)))
        if cp[0] == "w":
            self.wbar[cp[1]].arrive()
            return
        _, c, slot, li = cp
        R = self.ring[c]
        assert R.row[slot] == li
        R.landed[slot] = True
        R.full[slot].arrive()

    def _procs(self):
        procs = {"producer0": self.producer(0), "producer1": self.producer(1), "mma": self.mma(),
                 "relay": self.relay()}
        for c in range(2):
            for g in range(2):
                for q in range(4):
                    procs[f"epilogue{c}{g}.{q}"] = self.epilogue(c, g)
        return procs

    run = Sim.run


@pytest.mark.parametrize("ru", [3, 5, 8])
def test_cta_pair_protocol_holds(ru):
    rng = random.Random(3000 + ru)
    for trial in range(40):
        PairSim(_units(rng, ru), ru, random.Random(rng.random())).run()


@pytest.mark.parametrize("variant", ["marker_not_recorded", "relay_drops_marker"])
def test_pair_model_catches_marker_faults(variant):
    rng = random.Random(9)
    caught = 0
    for trial in range(30):
        try:
            PairSim(_units(rng, 8), 8, random.Random(rng.random()), variant).run()
        except Violation:
            caught += 1
    assert caught >= 5, caught
