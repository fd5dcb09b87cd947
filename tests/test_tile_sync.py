"""Race-freedom of the TMA step kernel's per-tile synchronisation, checked on a
model of its shared-memory accesses (no GPU).

A CTA runs tiles k = 0, 1, ...; tile k's input box lives in buffer k % NBUF
(filled by a TMA load whose completion the tile waits for on an mbarrier), and
its stages exchange micro-tile boundary rows through an exchange buffer Y
(one buffer, or two alternating between tiles).  Per tile:

  prologue + stage 0: read box(k); write Y(k)
  stage 1: read Y(k); write boundary rows of box(k)
  stage 2: read box(k); write Y(k)
  stage 3: read Y(k); epilogue stores go to global memory only

with a CTA barrier after stages 0, 1 and 2, plus (one exchange buffer) a
barrier that opens every tile.  The TMA refill of box(k)'s buffer for tile
k + NBUF is issued by one thread right after a barrier: after the barrier that
opens tile k + 1 (one exchange buffer) or after tile k's third stage barrier
(two).  Warps run freely between barriers, so two accesses of different warps
are ordered iff they lie in different barrier epochs.  The model checks that
no two conflicting accesses (at least one write) to the same buffer share an
epoch, and that no access to a box buffer falls between the issue of its TMA
refill and the consuming tile's mbarrier wait."""
import pytest


def schedule(ntiles, nbuf, two_y):
    """(epoch, buffer, kind) for every shared-memory access; kind in
    'r', 'w' (generic, any warp), 'tma' (async write of a refill: epoch of the
    issue; the consuming tile waits on its mbarrier before touching it)."""
    acc = []
    epoch = 0
    # prologue: loads of the first tiles before any barrier
    for k in range(min(nbuf if two_y else nbuf - 1, ntiles)):
        acc.append((-1, ("box", k % nbuf), "tma", k))
    for k in range(ntiles):
        y = ("Y", k & 1) if two_y else ("Y", 0)
        box = ("box", k % nbuf)
        if not two_y:
            epoch += 1  # the barrier that opens the tile
            kn = k + nbuf - 1
            if kn < ntiles:  # refill of the buffer the previous tile used
                acc.append((epoch, ("box", kn % nbuf), "tma", kn))
        acc.append((epoch, box, "r", k))   # prologue and stage 0 read the box
        acc.append((epoch, y, "w", k))     # stage 0 writes Y
        epoch += 1                         # stage barrier 1
        acc.append((epoch, y, "r", k))     # stage 1 reads Y
        acc.append((epoch, box, "w", k))   # and writes boundary rows into the box
        epoch += 1                         # stage barrier 2
        acc.append((epoch, box, "r", k))   # stage 2 reads the box
        acc.append((epoch, y, "w", k))     # and writes Y
        epoch += 1                         # stage barrier 3
        if two_y and k + nbuf < ntiles:    # refill right after the last barrier
            acc.append((epoch, box, "tma", k + nbuf))
        acc.append((epoch, y, "r", k))     # stage 3 reads Y
    return acc


def check(acc):
    # 1. generic accesses: conflicts only across epochs
    by_key = {}
    for e, buf, kind, tile in acc:
        if kind == "tma":
            continue
        by_key.setdefault((e, buf), []).append((kind, tile))
    for (e, buf), lst in by_key.items():
        tiles_w = {t for k, t in lst if k == "w"}
        tiles_all = {t for _, t in lst}
        # accesses of one tile in one epoch are that tile's own (one stage):
        # a write of one tile with any access of another tile is a race
        assert not (tiles_w and len(tiles_all) > 1), (e, buf, lst)
    # 2. a TMA refill of a box buffer for tile c, issued at epoch e: every
    #    generic access of that buffer by an earlier tile has epoch < e, and
    #    none by tile c comes before c's wait (all of c's accesses are after)
    for e, buf, kind, c in acc:
        if kind != "tma":
            continue
        for e2, buf2, kind2, t2 in acc:
            if buf2 != buf or kind2 == "tma":
                continue
            if t2 < c:
                assert e2 < e, ("refill of", buf, "for tile", c, "at epoch", e,
                                "while tile", t2, "accesses it at epoch", e2)


@pytest.mark.parametrize("nbuf", [2, 3])
@pytest.mark.parametrize("two_y", [False, True])
def test_tile_schedule_is_race_free(nbuf, two_y):
    check(schedule(9, nbuf, two_y))


def test_one_exchange_buffer_needs_the_opening_barrier():
    """Dropping the opening barrier with a single exchange buffer races: the
    next tile's stage 0 writes Y while the previous tile's stage 3 reads it."""
    acc = []
    for e, buf, kind, t in schedule(4, 2, two_y=True):
        if buf[0] == "Y":
            buf = ("Y", 0)
        acc.append((e, buf, kind, t))
    with pytest.raises(AssertionError):
        check(acc)


def test_refill_before_the_last_stage_barrier_races():
    """Issuing the refill one barrier earlier (after stage barrier 2) would
    overwrite the box while stage 2 still reads it."""
    acc = []
    for e, buf, kind, t in schedule(5, 2, two_y=True):
        if kind == "tma" and e >= 0:
            e -= 1
        acc.append((e, buf, kind, t))
    with pytest.raises(AssertionError):
        check(acc)
