"""CPU model of the stage handshakes of the tensor-core 3PCF Gram (gram_tc_kernel).

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
