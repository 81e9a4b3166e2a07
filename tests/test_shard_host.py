"""Host logic of sample sharding, on the CPU: the tile partition
(sbs_shard_range) and, in a world-size-2 gloo group of two processes, the
exchange (an int32 sum of disjoint words that carries every bit pattern) and
the ShardedController iteration loop around a stand-in controller."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_range_partitions_tiles():
    for ntiles in list(range(0, 40)) + [313, 4375, 65536]:
        for world in range(1, 10):
            spans = [S.shard_range(ntiles, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == ntiles
            sizes = []
            for r in range(world):
                b, e = spans[r]
                assert b <= e
                if r:
                    assert b == spans[r - 1][1]  # contiguous, in rank order
                sizes.append(e - b)
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("args", [(10, -1, 2), (10, 2, 2), (10, 0, 0), (-1, 0, 1)])
def test_shard_range_refuses(args):
    with pytest.raises(S.SBSError):
        S.shard_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_exchange_and_loop_gloo_world2(tmp_path):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "shard_worker.py"), "host",
                                       str(tmp_path / f"r{r}.npz")], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        try:
            out, _ = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append(out)
    for r, p in enumerate(procs):
        assert p.returncode == 0, f"rank {r}:\n{outs[r][-3000:]}"
    d = [np.load(tmp_path / f"r{r}.npz") for r in range(2)]
    for r in range(2):
        np.testing.assert_array_equal(d[r]["exch"], d[r]["ref"])  # every bit pattern, NaN payloads included
        assert d[r]["seen"].shape[0] == 6  # 3 ticks x 2 iterations
        for s in d[r]["seen"]:
            np.testing.assert_array_equal(s, d[r]["full"])
    assert d[0]["tiles"][0] == 0 and d[0]["tiles"][1] == d[1]["tiles"][0]
