"""One rank of a sample-sharded solve, launched by the sharding tests as a
separate process (gloo process group over 127.0.0.1; RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT from the environment).

    python tests/shard_worker.py host OUT.npz      CPU only: the exchange and the
                                                   ShardedController loop with a
                                                   stand-in controller
    python tests/shard_worker.py gpu CASE OUT.npz  a real controller on cuda:0
                                                   (rank 0 also solves unsharded)
"""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2403_11383_b300 import sbs as S  # noqa: E402
from paper_2403_11383_b300 import sharding  # noqa: E402

# bit patterns the exchange must carry unchanged: NaN payloads, infinities,
# signed zero, subnormals, the largest finite values
SPECIAL = np.array([0x7FC00001, 0x7F800001, 0xFFC12345, 0x7F800000, 0xFF800000, 0x80000000, 0x00000001,
                    0x807FFFFF, 0x7F7FFFFF, 0xFF7FFFFF, 0x3F800000, 0xFFFFFFFF], dtype=np.uint32)


def host_words(n, seed=5):
    """The words every rank's slice is cut from: SPECIAL then seeded random words."""
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    w[:len(SPECIAL)] = SPECIAL
    return w


class StandIn:
    """A controller stand-in on the host: K 'samples' in tiles of T; a sample's
    two words are host_words at its index, a tile's row is the tile's first
    word repeated PS times.  The update records the buffer it is given."""

    def __init__(self, K=1000, T=64, PS=5):
        self.K, self.T, self.PS = K, T, PS
        self.ntiles = (K + T - 1) // T
        self.Kp = (K + 63) // 64 * 64
        self.words = host_words(K)
        self.seen = []

    def full(self):
        b = np.zeros(2 * self.Kp + self.ntiles * self.PS, dtype=np.uint32)
        b[:self.K] = self.words
        b[self.Kp:self.Kp + self.K] = self.words[::-1]
        for t in range(self.ntiles):
            b[2 * self.Kp + t * self.PS:2 * self.Kp + (t + 1) * self.PS] = self.words[t * self.T]
        return b

    def shard_exchange_bytes(self):
        return 4 * (2 * self.Kp + self.ntiles * self.PS)

    def shard_tiles(self):
        return self.ntiles

    def problem(self, *a, **k):
        return None

    def shard_rollout(self, problem, rank, world, xbuf):
        b, e = S.shard_range(self.ntiles, rank, world)
        full = self.full()
        mine = np.zeros_like(full)
        lo, hi = b * self.T, min(e * self.T, self.K)
        mine[lo:hi] = full[lo:hi]
        mine[self.Kp + lo:self.Kp + hi] = full[self.Kp + lo:self.Kp + hi]
        r0 = 2 * self.Kp
        mine[r0 + b * self.PS:r0 + e * self.PS] = full[r0 + b * self.PS:r0 + e * self.PS]
        xbuf.view(torch.int32).copy_(torch.from_numpy(mine.view(np.int32)))

    def shard_update(self, xbuf, result):
        self.seen.append(xbuf.view(torch.int32).numpy().view(np.uint32).copy())
        return result

    def close(self):
        pass


def run_host(out):
    rank, world = dist.get_rank(), dist.get_world_size()
    # 1. the exchange alone: rank r owns the words i with i % world == r
    n = 4099
    ref = host_words(n, seed=11)
    mine = np.where(np.arange(n) % world == rank, ref, 0).astype(np.uint32)
    buf = torch.from_numpy(mine.view(np.uint8).copy())
    sharding.exchange(buf)
    exch = buf.numpy().view(np.uint32).copy()
    # 2. the solve loop: two iterations per tick, three ticks
    fake = StandIn()
    sc = sharding.ShardedController({"iterations": 2}, controller=fake, device="cpu")
    for _ in range(3):
        sc.solve(None, None, None)
    np.savez(out, exch=exch, ref=ref, seen=np.stack(fake.seen), full=fake.full(),
             tiles=np.array(sc.tiles))


def run_gpu(case, out):
    from paper_2403_11383_b300 import workloads as W
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from shard_cases import CASES, problem_tensors, ticks
    rank = dist.get_rank()
    torch.cuda.set_device(0)
    cfg = CASES[case]()
    prob = W.problem(cfg)
    x0, xr, fe, feet = problem_tensors(prob)
    sc = sharding.ShardedController(cfg, tile=cfg.get("tile", 0))
    ref = S.Controller(cfg, cfg.get("tile", 0)) if rank == 0 else None
    for c in (sc.ctl, ref):
        if c is not None and cfg.get("spt"):
            c.set_samples_per_thread(cfg["spt"])
    rec = {}
    for tick, (g, shift) in enumerate(ticks(cfg, prob)):
        r = sc.solve(x0, xr, g, fe, shift, feet=feet)
        rec[f"res{tick}"] = r.cpu().numpy()
        rec[f"mean{tick}"] = sc.ctl.read(S.BUF_MEAN).cpu().numpy()
        rec[f"cost{tick}"] = sc.ctl.read(S.BUF_COST).cpu().numpy()
        if ref is not None:
            rr = ref.solve(x0, xr, g, fe, shift, feet=feet)
            rec[f"ref_res{tick}"] = rr.cpu().numpy()
            rec[f"ref_mean{tick}"] = ref.read(S.BUF_MEAN).cpu().numpy()
            rec[f"ref_cost{tick}"] = ref.read(S.BUF_COST).cpu().numpy()
    torch.cuda.synchronize()
    rec["tiles"] = np.array(sc.tiles)
    np.savez(out, **rec)
    sc.close()
    if ref is not None:
        ref.close()


if __name__ == "__main__":
    dist.init_process_group("gloo", init_method="env://")
    try:
        if sys.argv[1] == "host":
            run_host(sys.argv[2])
        else:
            run_gpu(sys.argv[2], sys.argv[3])
        dist.barrier()
    finally:
        dist.destroy_process_group()
