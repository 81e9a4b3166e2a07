"""Host-side tuning of a batch's tile size (samples per block).

The tile is fixed when a controller is created (it sets the workspace layout),
so it is chosen before the controllers of a batch are built: the same
controllers are created at each candidate tile, and the library's launch
autotuner (``Batch.autotune``: launch mode, samples per thread, stored or
regenerated deviations) times each candidate at its own best setting, so that
tiles are compared as they will run (in the default setting two tiles can be
within noise of each other while one is 10 % faster in the setting chosen
afterwards).  The fastest tile is kept; the launch setting is tuned again on the
final controllers.  The candidates' results are identical up to rounding order
(per-tile partial sums), so the choice affects speed only.
"""
from __future__ import annotations

from . import sbs as S


def tile_for_batch(cfgs, inputs, tiles=(128, 256), ticks=5, inflight=2):
    """cfgs: controller configurations; inputs: per controller (x0, xref, gait,
    f_ext[, feet]) with x0, xref, f_ext (and feet, for ground-fixed feet) CUDA
    tensors.  Returns (best tile, {tile: ms per tick at that tile's best launch
    setting, from the launch autotuner's profiled ticks}).  The controllers built
    here are discarded."""
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
        probs = [ctls[i].problem(*inputs[i][:4], 1, feet=inputs[i][4] if len(inputs[i]) > 4 else None)
                 for i in range(n)]
        ms[tile] = min(batch.autotune(ctls, probs, res, ticks=ticks))
        torch.cuda.synchronize()
        batch.close()
        for c in ctls:
            c.close()
    best = min(ms, key=ms.get)
    return best, ms
