"""Sample sharding of one controller over the ranks of a torch.distributed group.

The K samples of one solve are independent until the update (Alg. 1 Sampling
and Rollout, Alg. 4), and the tile is the unit of the rollout, so the ranks
split the controller's tiles into contiguous ranges.  One iteration is

1. every rank rolls its tiles out into an exchange buffer (``sbs_shard_rollout``):
   its samples' costs and quantised frequencies, its tiles' MPPI rows;
2. the buffer is summed over the ranks as int32 words: every word is written by
   at most one rank and is zero on the others, so the sum is the written bits,
   with no floating-point arithmetic;
3. every rank runs the update (``sbs_shard_update``): the MPPI combine of
   Alg. 5 over all tile rows in tile order, or the selection of Alg. 1 / Alg. 3
   over all costs and the refit from regenerated elite deviations.

Every rank then holds what an unsharded solve of the same controller gives, bit
for bit.  The collective of step 2 is the only exchange: NCCL on the device
buffer, or (gloo) a copy through host memory.
"""
from typing import Optional

import torch
import torch.distributed as dist

from . import sbs as S


def exchange(buf: torch.Tensor, group=None) -> torch.Tensor:
    """Sum ``buf`` (a byte tensor, a multiple of 4 bytes long) over the group's
    ranks as int32 words, in place, on the current stream."""
    if buf.numel() % 4:
        raise ValueError("the exchange buffer holds whole 32-bit words")
    words = buf.view(torch.int32)
    if words.is_cuda and dist.get_backend(group) == "nccl":
        dist.all_reduce(words, op=dist.ReduceOp.SUM, group=group)
        return buf
    host = words.cpu() if words.is_cuda else words
    dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
    if host is not words:
        words.copy_(host)
    return buf


class ShardedController:
    """One controller whose samples are split over the ranks of ``group``.

    Every rank creates it with the same configuration (the same seed and
    controller id: the samples are a function of their index) and calls
    ``solve`` with the same problem.  ``controller`` may be passed in place of
    a new ``sbs.Controller`` (anything with its shard methods)."""

    def __init__(self, cfg: dict, group=None, tile: int = 0, controller=None, device: str = "cuda"):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.ctl = controller if controller is not None else S.Controller(cfg, tile)
        self.iterations = int(cfg.get("iterations", 1))
        self.xbuf = torch.zeros(self.ctl.shard_exchange_bytes(), dtype=torch.uint8, device=device)
        self.result = torch.empty(S.RESULT_BYTES, dtype=torch.uint8, device=device)
        self.tiles = S.shard_range(self.ctl.shard_tiles(), self.rank, self.world)

    def solve(self, x0, xref, gait: dict, f_ext=None, shift: int = 0, feet=None,
              result: Optional[torch.Tensor] = None) -> torch.Tensor:
        """One tick (all iterations) on the current stream; device inputs as for
        ``Controller.solve``.  Returns the device result (the same on every rank)."""
        out = self.result if result is None else result
        p = self.ctl.problem(x0, xref, gait, f_ext, shift, feet=feet)
        for _ in range(self.iterations):
            self.ctl.shard_rollout(p, self.rank, self.world, self.xbuf)
            exchange(self.xbuf, self.group)
            self.ctl.shard_update(self.xbuf, out)
        return out

    def close(self):
        self.ctl.close()
