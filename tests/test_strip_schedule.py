"""Host-side model of the strip-pipelined BLU-SGS half-sweep
(k_blusgs_strip): the cells each step updates, the waits on the previous
strip and the progress each strip publishes, restated from the kernel's index
arithmetic.  Run over random interleavings that the wait protocol allows, it
checks the lexicographic sweep's dependencies (Algorithm 1, BLU-SGS): every
cell is updated exactly once, its neighbours before it in the sweep order are
already updated, the ones after it are not, and the lane that publishes a
strip's progress is the lane that wrote the published cell."""
import random

import pytest


def cells_of_step(nx, ny, R, GRP, q, t, forward):
    rows = min(R, ny - q * R)
    c_lo, c_hi = max(0, t - rows + 1), min(nx - 1, t)
    ncell = c_hi - c_lo + 1
    if forward:
        d, ix0 = q * R + t, c_lo
    else:
        d, ix0 = (nx - 1) + (ny - 1) - (q * R + t), nx - 1 - c_hi
    out = []
    for lane in range(32):
        cell, g = lane // GRP, lane % GRP
        if cell < ncell and g == 0:
            ix = ix0 + cell; iy = d - ix
            out.append((lane, ix, iy))
    return out, ncell, rows

def check(nx, ny, R, GRP, forward, seed):
    rng = random.Random(seed)
    nstrips = (ny + R - 1) // R
    done = {}            # (ix, iy) -> order
    prog = [0] * nstrips
    tpos = [0] * nstrips
    order = 0
    active = list(range(nstrips))
    while active:
        # pick a strip that may run its next step (random interleaving)
        runnable = []
        for q in active:
            t = tpos[q]
            rows = min(R, ny - q * R)
            if q > 0 and t < nx and prog[q - 1] < t + 1:
                continue
            runnable.append(q)
        assert runnable, "deadlock"
        q = rng.choice(runnable)
        t = tpos[q]
        cells, ncell, rows = cells_of_step(nx, ny, R, GRP, q, t, forward)
        for lane, ix, iy in cells:
            assert 0 <= ix < nx and 0 <= iy < ny, (ix, iy)
            assert q * R <= (iy if forward else ny - 1 - iy) < q * R + rows
            assert (ix, iy) not in done, "twice"
            before = [(ix - 1, iy), (ix, iy - 1)] if forward else [(ix + 1, iy), (ix, iy + 1)]
            after = [(ix + 1, iy), (ix, iy + 1)] if forward else [(ix - 1, iy), (ix, iy - 1)]
            for b in before:
                if 0 <= b[0] < nx and 0 <= b[1] < ny:
                    assert b in done, ("before not done", (ix, iy), b)
            for a in after:
                assert a not in done, ("after already done", (ix, iy), a)
        for lane, ix, iy in cells:
            done[(ix, iy)] = order
        order += 1
        dn = t - rows + 2
        if q + 1 < nstrips and 1 <= dn <= nx:
            rel = 0 if forward else (ncell - 1) * GRP
            # the releasing lane owns the last row's cell at column dn - 1
            col = dn - 1
            ix_last = col if forward else nx - 1 - col
            iy_last = q * R + rows - 1 if forward else ny - 1 - (q * R + rows - 1)
            assert any(l == rel and (ix, iy) == (ix_last, iy_last) for l, ix, iy in cells), (q, t)
            assert dn > prog[q]
            prog[q] = dn
        tpos[q] += 1
        if tpos[q] == nx + rows - 1:
            active.remove(q)
    assert len(done) == nx * ny



SIZES = [(1, 1), (5, 1), (1, 7), (3, 3), (4, 5), (7, 2), (16, 16), (9, 13), (32, 8), (6, 31)]


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("forward", [True, False])
def test_strip_schedule_keeps_sweep_order(nx, ny, forward):
    for seed in range(6):
        check(nx, ny, 2, 16, forward, seed)        # 2D: 16 lanes per cell, 2 rows per strip
        if ny == 1:
            check(nx, ny, 4, 8, forward, seed)     # 1D: 8 lanes per cell


def _batch_tickets(sizes, R):
    """(problem, strip) tickets in claim order: strip index first, then problem."""
    out = []
    for q in range(max((ny + R - 1) // R for _, ny in sizes)):
        for p, (_, ny) in enumerate(sizes):
            if q < (ny + R - 1) // R:
                out.append((p, q))
    return out


def _run_batch(sizes, R, warps, rng):
    """G warps claim tickets in order and run their strips step by step in a
    random interleaving; a warp whose strip waits on the previous strip of
    its problem stays put.  Returns False on a deadlock."""
    tickets = _batch_tickets(sizes, R)
    nxt = 0
    prog = {}
    state = [None] * warps            # (p, q, t) of the strip a warp holds
    done_cells = {p: set() for p in range(len(sizes))}
    while True:
        for w in range(warps):
            if state[w] is None and nxt < len(tickets):
                p, q = tickets[nxt]
                nxt += 1
                state[w] = (p, q, 0)
        live = [w for w in range(warps) if state[w] is not None]
        if not live:
            break
        movable = []
        for w in live:
            p, q, t = state[w]
            nx, ny = sizes[p]
            if q > 0 and t < nx and prog.get((p, q - 1), 0) < t + 1:
                continue
            movable.append(w)
        if not movable:
            return False
        w = rng.choice(movable)
        p, q, t = state[w]
        nx, ny = sizes[p]
        rows = min(R, ny - q * R)
        for r in range(rows):
            c = t - r
            if 0 <= c < nx:
                done_cells[p].add((c, q * R + r))
        dn = t - rows + 2
        if 1 <= dn <= nx:
            prog[(p, q)] = dn
        t += 1
        state[w] = None if t == nx + rows - 1 else (p, q, t)
    return all(len(done_cells[p]) == nx * ny for p, (nx, ny) in enumerate(sizes))


@pytest.mark.parametrize("warps", [1, 2, 3, 7])
def test_batch_tickets_never_deadlock(warps):
    """Batched strips: with any number of resident warps, every problem of a
    mixed-size batch completes (a strip waits only for an earlier ticket)."""
    rng = random.Random(warps)
    for trial in range(20):
        sizes = [(rng.randint(1, 9), rng.randint(1, 9)) for _ in range(rng.randint(1, 5))]
        assert _run_batch(sizes, 2, warps, rng), sizes
