"""CPU models of the stage handshakes of the two tensor-core kernels: the 3PCF
Gram (gram_tc_kernel, first) and the 4PCF contraction (tc4_kernel, below).

The kernel's roles are modelled as interleaved programs under a random
scheduler:
- one loader fills raw stage k mod 6 with the copy of K-block k;
- 4 producer groups of 2 warps each take the K-blocks k = g (mod 4), read the
  raw stage, release it, and then fill operand stage k mod 6;
- one MMA issuer consumes the operand stages in order.

mbarriers follow the PTX semantics of `mbarrier.try_wait.parity`: a wait on
parity P passes as soon as the barrier's current (incomplete) phase has the
other parity.  So a waiter that is two phases behind passes at once.  Copies
into different raw stages land in any order (TMA gives no order between
them).  MMAs, and so their releases of the operand stages, complete in issue
order (tcgen05.commit tracks all earlier MMAs of the issuing thread).

Checked on every run:
- a producer reads a raw stage only after its K-block's copy has landed, and
  before the loader refills it;
- the loader refills a stage only after both warps of its last user have
  released it;
- a producer overwrites an operand stage only after the MMAs that read it
  have completed;
- the MMA issuer consumes a stage only after both warps formed it.

Raw stages rotate over the groups (6 stages, 4 groups), so a stage alternates
between two groups.  Before waiting for its copy, a group therefore waits for
the stage's release of the previous K-block by the other group (the kernel's
wait code 59).  The model shows that this wait is needed: without it, a copy
that lands late lets the next waiter on that stage pass two phases early.
"""
import random

import pytest

RAW = 6      # raw stages
OPS = 6      # operand stages
GROUPS = 4   # producer groups
WARPS = 2    # warps per group (each arrives on the stage barriers)


class Barrier:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.completed = 0  # phases completed; the current phase has this index

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.completed += 1
            self.pending = self.count

    def passes(self, parity):
        # try_wait.parity(P): the phase of parity P is the current or the
        # immediately preceding one; it has completed iff the current phase
        # has the other parity
        return (self.completed & 1) != parity


class Violation(Exception):
    pass


def check(cond, what):
    if not cond:
        raise Violation(what)


def run(nk, seed, release_wait=True):
    rng = random.Random(seed)
    raw_full = [Barrier(1) for _ in range(RAW)]        # completes when the stage's copy lands
    raw_empty = [Barrier(WARPS) for _ in range(RAW)]   # both warps of the consumer released it
    op_full = [Barrier(WARPS) for _ in range(OPS)]     # both warps formed it
    op_empty = [Barrier(1) for _ in range(OPS)]        # the MMAs that read it completed
    stage = [None] * RAW           # K-block whose copy was last issued into a raw stage
    landed = set()
    in_flight = []                 # copies issued, not landed
    released = [0] * nk            # warps that released K-block k's raw stage
    formed = [0] * nk              # warps that formed K-block k's operand stage
    mma_queue = []                 # MMAs issued, completing in order
    mma_done = set()

    def loader():
        for k in range(nk):
            rs = k % RAW
            yield raw_empty[rs], ((k // RAW) & 1) ^ 1
            check(k < RAW or released[k - RAW] == WARPS, f"raw stage {rs} refilled with K-block {k} before "
                                                          f"K-block {k - RAW} was released")
            stage[rs] = k
            in_flight.append(k)

    def producer(g):
        for k in range(g, nk, GROUPS):
            rs, os = k % RAW, k % OPS
            if release_wait and k >= RAW:
                yield raw_empty[rs], ((k // RAW) - 1) & 1
            yield raw_full[rs], (k // RAW) & 1
            check(stage[rs] == k and k in landed, f"K-block {k} read from raw stage {rs} before its copy landed")
            yield None  # reading the stage into registers takes time
            check(stage[rs] == k, f"raw stage {rs} refilled while K-block {k} was read")
            released[k] += 1
            raw_empty[rs].arrive()
            yield op_empty[os], ((k // OPS) & 1) ^ 1
            check(k < OPS or (k - OPS) in mma_done, f"operand stage {os} overwritten with K-block {k} before "
                                                    f"the MMAs of K-block {k - OPS} completed")
            yield None  # forming the operands takes time
            formed[k] += 1
            op_full[os].arrive()

    def mma():
        for k in range(nk):
            os = k % OPS
            yield op_full[os], (k // OPS) & 1
            check(formed[k] == WARPS, f"MMAs of K-block {k} issued before its operand stage was formed")
            mma_queue.append(k)

    actors = [loader(), mma()] + [producer(g) for g in range(GROUPS) for _ in range(WARPS)]
    waits, live = [None] * len(actors), []
    for i, a in enumerate(actors):
        try:
            waits[i] = next(a)
            live.append(i)
        except StopIteration:  # a producer group with no K-block
            pass
    while live or in_flight or mma_queue:
        options = [("actor", i) for i in live if waits[i] is None or waits[i][0].passes(waits[i][1])]
        options += [("land", j) for j in range(len(in_flight))]
        if mma_queue:
            options.append(("mma", 0))
        check(options, "deadlock")
        kind, i = rng.choice(options)
        if kind == "land":
            k = in_flight.pop(i)
            landed.add(k)
            raw_full[k % RAW].arrive()
        elif kind == "mma":
            k = mma_queue.pop(0)
            mma_done.add(k)
            op_empty[k % OPS].arrive()
        else:
            try:
                waits[i] = next(actors[i])
            except StopIteration:
                live.remove(i)
    check(all(r == WARPS for r in released) and len(mma_done) == nk, "incomplete run")


@pytest.mark.parametrize("nk", [1, 5, 7, 24, 61])
def test_gram_tc_stage_protocol_is_safe(nk):
    for seed in range(200):
        run(nk, seed)


def test_without_the_release_wait_a_late_copy_is_read_early():
    found = 0
    for seed in range(300):
        try:
            run(48, seed, release_wait=False)
        except Violation as e:
            assert "before its copy landed" in str(e)
            found += 1
    assert found > 0


# ---------------------------------------------------------------------------
# The tensor-core 4PCF contraction (tc4_kernel).  Its roles, per CTA, over a
# sequence of work units (tile, x-range) of nk K-blocks each:
# - a B warp copies the B image of K-block kb into operand stage kb mod 4 once
#   the MMAs of that stage's previous K-block have completed (op_empty); the
#   copy completes on b_full;
# - loader warps copy the singles of K-block kb into the raw stages of producer
#   group kb mod 4 (RAW4 stages per group, used in order);
# - producer group g forms the A tile of its K-blocks kb = g (mod 4) in operand
#   stage g: it waits for its raw stage and for op_empty, forms, then its first
#   warp waits for the stage's B copy, and every warp arrives on op_full and
#   releases the raw stage;
# - the MMA issuer consumes the stages in K-block order, commits op_empty per
#   K-block and acc_full at the end of each accumulation range of FLUSH4
#   K-blocks; the first MMA of a range overwrites the inner accumulator;
# - group 0 folds range i - 1 before it forms the first K-block of range i, and
#   the unit's last range after its loop, each fold after acc_full.
# Checked besides the stage properties: a range is folded only after all its
# MMAs completed, and the first MMA of a range is issued only after every fold
# of the previous range has read the accumulator.

GROUPS4 = 4   # producer groups = operand stages
RAW4 = 2      # raw stages per producer group
FLUSH4 = 8    # K-blocks per accumulation range (a multiple of GROUPS4)


def run_tc4(units, seed, fold_first=True, b_wait=True):
    rng = random.Random(seed)
    nranges = [(nk + FLUSH4 - 1) // FLUSH4 for nk in units]
    base = [sum(nranges[:u]) for u in range(len(units))]   # global index of a unit's first range
    raw_full = [Barrier(1) for _ in range(GROUPS4 * RAW4)]
    raw_empty = [Barrier(WARPS) for _ in range(GROUPS4 * RAW4)]
    op_full = [Barrier(WARPS) for _ in range(GROUPS4)]
    op_empty = [Barrier(1) for _ in range(GROUPS4)]
    b_full = [Barrier(1) for _ in range(GROUPS4)]
    acc_full = Barrier(1)
    raw_stage, b_stage, a_stage = [None] * (GROUPS4 * RAW4), [None] * GROUPS4, [None] * GROUPS4
    landed = set()                 # ("raw" | "b", unit, kb) copies that have landed
    in_flight = []
    formed, released = {}, {}
    mma_issued, mma_done = set(), set()
    queue = []                     # MMAs (and acc_full commits) completing in order
    folded = {}                    # global range -> warps of group 0 that folded it

    def b_warp():
        issued = [0] * GROUPS4
        for u, nk in enumerate(units):
            for kb in range(nk):
                os = kb % GROUPS4
                yield op_empty[os], (issued[os] & 1) ^ 1
                check(b_stage[os] is None or b_stage[os] in mma_done,
                      f"B stage {os} refilled before the MMAs of {b_stage[os]} completed")
                issued[os] += 1
                b_stage[os] = (u, kb)
                in_flight.append(("b", u, kb))

    def loader():
        count = [0] * GROUPS4
        for u, nk in enumerate(units):
            for kb in range(nk):
                g = kb % GROUPS4
                n = count[g]
                count[g] += 1
                rs = RAW4 * g + n % RAW4
                yield raw_empty[rs], ((n // RAW4) & 1) ^ 1
                check(raw_stage[rs] is None or released.get(raw_stage[rs], 0) == WARPS,
                      f"raw stage {rs} refilled before {raw_stage[rs]} was released")
                raw_stage[rs] = (u, kb)
                in_flight.append(("raw", u, kb))

    def fold(g_range):
        yield acc_full, g_range & 1
        u = max(i for i in range(len(units)) if base[i] <= g_range)
        i = g_range - base[u]
        kbs = range(i * FLUSH4, min(units[u], (i + 1) * FLUSH4))
        check(all((u, kb) in mma_done for kb in kbs), f"range {g_range} folded before its MMAs completed")
        yield None  # reading the accumulator
        folded[g_range] = folded.get(g_range, 0) + 1

    def producer(g, w):
        uses = 0
        for u, nk in enumerate(units):
            done = 0  # ranges of this unit folded so far (group 0)
            for kb in range(g, nk, GROUPS4):
                if g == 0 and fold_first and kb % FLUSH4 == 0 and kb // FLUSH4 >= 1:
                    yield from fold(base[u] + kb // FLUSH4 - 1)
                    done = kb // FLUSH4
                rs = RAW4 * g + uses % RAW4
                yield raw_full[rs], (uses // RAW4) & 1
                check(raw_stage[rs] == (u, kb) and ("raw", u, kb) in landed,
                      f"K-block {(u, kb)} read from raw stage {rs} before its copy landed")
                yield op_empty[g], (uses & 1) ^ 1
                # the group's warps write their own rows of the same K-block
                check(a_stage[g] in (None, (u, kb)) or a_stage[g] in mma_done,
                      f"A stage {g} overwritten before the MMAs of {a_stage[g]} completed")
                uses += 1
                yield None  # forming the A tile
                a_stage[g] = (u, kb)
                formed[(u, kb)] = formed.get((u, kb), 0) + 1
                if w == 0 and b_wait:
                    yield b_full[g], (uses - 1) & 1
                    check(b_stage[g] == (u, kb) and ("b", u, kb) in landed,
                          f"B image of {(u, kb)} not landed when its stage was published")
                op_full[g].arrive()
                released[(u, kb)] = released.get((u, kb), 0) + 1
                raw_empty[rs].arrive()
            if g == 0:
                for i in range(done, nranges[u]):
                    yield from fold(base[u] + i)

    def mma():
        uses = [0] * GROUPS4
        for u, nk in enumerate(units):
            for kb in range(nk):
                os = kb % GROUPS4
                yield op_full[os], uses[os] & 1
                check(formed.get((u, kb), 0) == WARPS and a_stage[os] == (u, kb) and b_stage[os] == (u, kb)
                      and ("b", u, kb) in landed, f"MMAs of {(u, kb)} issued before its operands were ready")
                uses[os] += 1
                g_range = base[u] + kb // FLUSH4
                if kb % FLUSH4 == 0 and g_range > 0:
                    check(folded.get(g_range - 1, 0) == WARPS,
                          f"range {g_range} overwrote the accumulator before range {g_range - 1} was folded")
                mma_issued.add((u, kb))
                queue.append(("mma", u, kb))
                if (kb + 1) % FLUSH4 == 0 or kb + 1 == nk:
                    queue.append(("acc",))

    actors = [b_warp(), loader(), mma()] + [producer(g, w) for g in range(GROUPS4) for w in range(WARPS)]
    waits, live = [None] * len(actors), []
    for i, a in enumerate(actors):
        try:
            waits[i] = next(a)
            live.append(i)
        except StopIteration:
            pass
    while live or in_flight or queue:
        options = [("actor", i) for i in live if waits[i] is None or waits[i][0].passes(waits[i][1])]
        options += [("land", j) for j in range(len(in_flight))]
        if queue:
            options.append(("done", 0))
        check(options, "deadlock")
        kind, i = rng.choice(options)
        if kind == "land":
            c = in_flight.pop(i)
            landed.add(c)
            if c[0] == "raw":
                # the raw stage this copy went to: the one that holds it
                raw_full[raw_stage.index((c[1], c[2]))].arrive()
            else:
                b_full[c[2] % GROUPS4].arrive()
        elif kind == "done":
            e = queue.pop(0)
            if e[0] == "mma":
                mma_done.add((e[1], e[2]))
                op_empty[e[2] % GROUPS4].arrive()
            else:
                acc_full.arrive()
        else:
            try:
                waits[i] = next(actors[i])
            except StopIteration:
                live.remove(i)
    check(len(mma_done) == sum(units) and all(folded.get(r, 0) == WARPS for r in range(sum(nranges))),
          "incomplete run")


@pytest.mark.parametrize("units", [[1], [5], [8], [13, 3], [9, 16, 2], [17, 1, 8, 11]])
def test_tc4_stage_protocol_is_safe(units):
    for seed in range(150):
        run_tc4(units, seed)


def test_tc4_without_the_fold_first_the_next_range_overwrites_the_accumulator():
    found = 0
    for seed in range(150):
        try:
            run_tc4([20, 9], seed, fold_first=False)
        except Violation as e:
            assert "overwrote the accumulator" in str(e) or "folded before" in str(e)
            found += 1
    assert found > 0


def test_tc4_without_the_b_wait_the_mmas_can_read_a_b_image_in_flight():
    found = 0
    for seed in range(150):
        try:
            run_tc4([13, 6], seed, b_wait=False)
        except Violation as e:
            assert "operands were ready" in str(e)
            found += 1
    assert found > 0
