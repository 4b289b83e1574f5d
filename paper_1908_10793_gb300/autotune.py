"""Autotuner for the dust contexts and batches: tile shape, and for a batch
the sort interval, each candidate timed in the configuration it is for.

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


# ---- batches -------------------------------------------------------------

def batch_candidates(ws, sort_intervals=(1, 2), modes=(0, 1)):
    """Configurations of a batch to try: a tile policy (None = the library's
    default for every instance, or one shape applied to every instance,
    clipped to its grid), the batch's sort interval, and the execution mode
    (dust_options.batch_mode: 0 one persistent launch, 1 a graph of
    per-instance kernels, which sorts every step).  The default
    configuration comes first."""
    shapes = candidate_tiles(max(ws, key=lambda w: w.ncell))
    policies = [None] + [s for s in shapes if s != shapes[0]]
    out = []
    for m in modes:
        for k in sort_intervals:
            if m == 1 and k != 1:
                continue
            out += [(p, k, m) for p in policies]
    return out


def _tile_for(w, policy):
    if policy is None:
        return (0, 0, 0)
    return tuple(min(policy[d], w.n[d]) if w.n[d] > 1 else 1 for d in range(3))


def time_batch(ws, policy=None, sort_interval=1, steps=4, warmup=2, device=0, batch_mode=0):
    """Device time per step (ms, CUDA events on the batch's stream) of a
    batch of the workloads ws in one configuration: every instance a mixed
    precision context with the policy's tile, one dust_batch_step call of
    `steps` steps after `warmup` steps."""
    import torch
    stream = torch.cuda.Stream(device)
    ctxs = []
    b = None
    try:
        for w in ws:
            c = D.Context(w, precision=D.DUST_MIXED, sort_interval=sort_interval, device=device,
                          tile=_tile_for(w, policy))
            c.set_gas(w.rho, w.vgas)
            c.load(w.q, w.v, w.species, w.param)
            ctxs.append(c)
        opt = D.dust_options(stream=stream.cuda_stream, sort_interval=sort_interval,
                             batch_mode=batch_mode)
        b = D.dust_batch_create([c.handle for c in ctxs], opt)
        dts = [w.dt for w in ws]
        D.dust_batch_step(b, dts, warmup)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        D.dust_batch_step(b, dts, steps)
        e1.record(stream)
        torch.cuda.synchronize(device)
        bad = [rc for rc in (c.sync(check=False)[0] for c in ctxs) if rc not in (0, D.DUST_ECFL)]
        if bad:
            raise D.DustError(bad[0], "batch status %d" % bad[0])
        return e0.elapsed_time(e1) / steps
    finally:
        if b is not None:
            D.dust_batch_destroy(b)
        for c in ctxs:
            c.close()


def tune_batch(ws, steps=4, candidates=None, device=0):
    """Times every candidate configuration in the batch (not instance by
    instance) and returns (best (policy, sort interval, mode), {config: ms
    per step}).  Candidates that do not fit are skipped."""
    cands = candidates or batch_candidates(ws)
    times = {}
    for cfg in cands:
        try:
            times[cfg] = time_batch(ws, cfg[0], cfg[1], steps=steps - steps % 2 if cfg[2] else steps,
                                    device=device, batch_mode=cfg[2])
        except D.DustError:
            continue
    best = min(times, key=times.get)
    return best, times
