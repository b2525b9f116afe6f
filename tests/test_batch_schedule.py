"""Host model of the persistent batch schedule (k_fused_batch_persist).

The kernel lists the work items of every wave in wave order (pass w of a
register before pass w + 1), CTAs claim runs of consecutive items from a
global ticket, and before the first item of a register's pass w > 0 a CTA
waits until every tile of pass w - 1 is done.  The argument that this
cannot deadlock: a waited-on item has a smaller index than the waiting one,
so it was claimed earlier by a running CTA, which never waits on a later
item.  This model runs the same rules under random interleavings of CTAs
(any number of CTAs, run lengths 1, 2 and 8) and checks that every schedule
finishes and that no tile starts before its register's previous pass is
complete.  No GPU involved."""
import random

import pytest


def make_items(rnd, nreg):
    """Wave-ordered items (pass id, tile) and, per pass, (previous pass, its tiles)."""
    npass = [rnd.randint(1, 6) for _ in range(nreg)]
    ids, tiles = {}, []
    for r in range(nreg):
        for w in range(npass[r]):
            ids[(r, w)] = len(tiles)
            tiles.append(rnd.randint(1, 9))
    items = []
    for w in range(max(npass)):
        regs = [r for r in range(nreg) if npass[r] > w]
        rnd.shuffle(regs)            # any order inside a wave
        for r in regs:
            p = ids[(r, w)]
            items += [(p, t) for t in range(tiles[p])]
    dep = {p: ((ids[(r, w - 1)], tiles[ids[(r, w - 1)]]) if w else (-1, 0)) for (r, w), p in ids.items()}
    return items, dep, tiles


def run_schedule(seed):
    rnd = random.Random(seed)
    items, dep, tiles = make_items(rnd, rnd.randint(1, 30))
    chunk = rnd.choice([1, 2, 8])
    ctas = rnd.randint(1, 12)
    done = [0] * len(tiles)
    ticket = 0
    state = [None] * ctas          # (run end, next item) of the CTA's claimed run
    finished = [False] * ctas
    for _ in range(10 ** 6):
        if all(finished):
            break
        movable = []
        for c in range(ctas):
            if finished[c]:
                continue
            if state[c] is not None:
                p, _ = items[state[c][1]]
                prev, need = dep[p]
                if prev >= 0 and done[prev] < need:
                    continue           # waiting for the previous pass
            movable.append(c)
        assert movable, "deadlock"
        c = rnd.choice(movable)
        if state[c] is None:           # claim the next run
            first = ticket * chunk
            ticket += 1
            if first >= len(items):
                finished[c] = True
            else:
                state[c] = (min(len(items), first + chunk), first)
            continue
        end, i = state[c]
        p, _ = items[i]
        prev, need = dep[p]
        assert prev < 0 or done[prev] == need
        done[p] += 1
        state[c] = (end, i + 1) if i + 1 < end else None
    assert all(finished)
    assert done == tiles


@pytest.mark.parametrize("block", range(6))
def test_claim_order_schedule_never_deadlocks(block):
    for seed in range(block * 400, (block + 1) * 400):
        run_schedule(seed)
