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
