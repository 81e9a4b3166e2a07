"""Host-side tuning of a batch's tile size (samples per block).

The tile is fixed when a controller is created (it sets the workspace layout),
so it is chosen before the controllers of a batch are built: the same
controllers are created at each candidate tile, a few batched ticks are timed
on the device, and the fastest tile is kept.  The launch mode is tuned
afterwards by the library itself (``Batch.autotune``).  The candidates' results
are identical up to rounding order (per-tile partial sums), so the choice
affects speed only.
"""
from __future__ import annotations

from . import sbs as S


def tile_for_batch(cfgs, inputs, tiles=(128, 256), ticks=5, inflight=2):
    """cfgs: controller configurations; inputs: per controller (x0, xref, gait,
    f_ext[, feet]) with x0, xref, f_ext (and feet, for ground-fixed feet) CUDA
    tensors.  Returns (best tile, {tile: mean ms per tick}).  The controllers
    built here are discarded."""
    import torch
    n = len(cfgs)
    if n == 0 or len(inputs) != n:
        raise ValueError("one input per controller, at least one controller")
    ms = {}
    for tile in tiles:
        ctls = [S.Controller(c, tile=tile) for c in cfgs]
        batch = S.Batch(n, inflight * sum(c.workspace_bytes() + 256 for c in ctls), inflight=inflight)
        res = torch.empty(n * S.RESULT_BYTES, dtype=torch.uint8, device="cuda")
        packed = [S.Packed(ctls, [ctls[i].problem(*inputs[i][:4], shift,
                                                  feet=inputs[i][4] if len(inputs[i]) > 4 else None)
                                  for i in range(n)]) for shift in (0, 1)]
        batch.solve_packed(packed[0], res)
        for _ in range(2):
            batch.solve_packed(packed[1], res)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(ticks):
            batch.solve_packed(packed[1], res)
        e1.record()
        torch.cuda.synchronize()
        ms[tile] = e0.elapsed_time(e1) / ticks
        batch.close()
        for c in ctls:
            c.close()
    best = min(ms, key=ms.get)
    return best, ms
