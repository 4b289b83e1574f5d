"""Tile-shape autotuner for the dust contexts.

The zone sort groups grains by tiles of zones and the step kernels stage one
tile's gas and deposit box per thread block, so the tile shape sets the
number of blocks, the halo overhead and the shared-memory footprint.  The
slab kernel's integer deposit does not depend on the tile shape (runs are
cut into chunks by rank inside a zone), so the tuner may pick any candidate
without changing results.

The tuner only orchestrates: it creates contexts through the C interface,
times a few steps of each candidate with the library's own device timers
(dust_get_kernel_times) and keeps the fastest.  Every step runs in the
library's kernels.
"""
from . import dust as D


def candidate_tiles(w):
    """Tile shapes to try for a workload: the default first, then shapes that
    trade halo overhead against the number of blocks."""
    n = w.n
    gridded = [d for d in range(3) if n[d] > 1]
    if len(gridded) == 3:
        shapes = [(8, 8, 8), (16, 8, 4), (8, 8, 4), (16, 8, 8), (4, 4, 4)]
    elif len(gridded) == 2:
        a, b = gridded
        shapes = []
        for ta, tb in ((16, 16), (32, 8), (8, 8), (32, 16), (16, 8)):
            t = [1, 1, 1]
            t[a], t[b] = ta, tb
            shapes.append(tuple(t))
    else:
        shapes = [tuple(256 if n[d] > 1 else 1 for d in range(3))]
    out = []
    for s in shapes:
        s = tuple(min(s[d], n[d]) if n[d] > 1 else 1 for d in range(3))
        if s not in out:
            out.append(s)
    return out


def time_tile(w, tile, precision=D.DUST_MIXED, steps=4, warmup=2, **kw):
    """Device time per step (sort + step + other, ms) of one tile shape."""
    ctx = D.Context(w, precision=precision, tile=tile, timing=1, sort_interval=1, **kw)
    try:
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v, w.species, w.param)
        for _ in range(warmup):
            ctx.step(w.dt)
        ctx.sync(check=False)
        ctx.kernel_times(reset=True)
        for _ in range(steps):
            ctx.step(w.dt)
        ctx.sync(check=False)
        t = ctx.kernel_times(reset=True)
        return (t.step_ms + t.sort_ms + t.other_ms) / steps
    finally:
        ctx.close()


def tune_tile(w, precision=D.DUST_MIXED, steps=4, candidates=None, **kw):
    """Returns (best tile, {tile: ms per step})."""
    cands = candidates or candidate_tiles(w)
    times = {}
    for tile in cands:
        try:
            times[tile] = time_tile(w, tile, precision, steps, **kw)
        except D.DustError:
            continue  # e.g. a tile whose boxes do not fit in shared memory
    best = min(times, key=times.get)
    return best, times
