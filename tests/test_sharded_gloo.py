"""A problem split by job range across two CPU ranks (torch.distributed with
the gloo backend), each evaluating its shard with the FP64 oracle: the
shards' per-block sums, all-gathered with the package's own all-gather and
added in rank order, give bit for bit the unsharded evaluation (the oracle
adds its 4096-job blocks in job order, and the shard boundaries fall on
block boundaries).  Also checks the package's shard boundaries."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_bounds_cover_the_jobs_in_aligned_ranges():
    from paper_2104_00282_gb300 import sharded
    for n, world in ((10_000_000, 8), (1_000_003, 3), (4096 * 5 + 7, 2), (300, 1)):
        b = sharded.shard_bounds(n, world)
        assert b[0][0] == 0 and b[-1][1] == n and len(b) == world
        for (s0, e0), (s1, e1) in zip(b, b[1:]):
            assert e0 == s1 and s0 < e0
            assert s1 % sharded.ALIGN == 0
    with pytest.raises(ValueError):
        sharded.shard_bounds(100, 4)


WORKER = textwrap.dedent("""
    import os, sys
    import numpy as np
    import torch
    import torch.distributed as dist
    sys.path.insert(0, {root!r})
    from oracle import oracle as O
    from paper_2104_00282_gb300 import sharded
    from paper_2104_00282_gb300 import workloads as W

    rank, world = int(sys.argv[1]), int(sys.argv[2])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    gather = sharded.torch_gather()
    for cap in (False, True):
        prob = W.config_large(n=45_000, m=6, seed=3)       # the same problem on every rank
        lam = O.init_prices(prob, cap=cap)
        s, e = sharded.shard_bounds(prob.n, world, align=O.BLOCK)[rank]
        sub = W.Problem(prob.A[s:e], prob.kind[s:e], prob.w[s:e], prob.param[s:e], prob.R)
        part = O.dual_blocks(sub, lam, cap=cap)
        counts = torch.zeros(world, dtype=torch.int64)
        gather(torch.tensor([part.shape[0]], dtype=torch.int64), counts)
        rows = int(counts.max())
        send = torch.zeros(rows, part.shape[1], dtype=torch.float64)
        send[:part.shape[0]] = torch.from_numpy(part)
        recv = torch.zeros(world * rows, part.shape[1], dtype=torch.float64)
        gather(send.view(-1), recv.view(-1))
        blocks = np.concatenate([recv[r * rows:r * rows + int(counts[r])].numpy() for r in range(world)])
        # rank-order combine, the oracle's own order of addition
        sh, r = 0.0, np.zeros(prob.m)
        for b in blocks:
            sh += b[0]
            r += b[2:2 + prob.m]
        lr = 0.0
        for j in range(prob.m):
            lr += lam[j] * prob.R[j]
        g_ref, r_ref, _ = O.dual(prob, lam, cap=cap)
        assert lr + sh == g_ref, (lr + sh, g_ref)
        assert np.array_equal(r, r_ref)
    dist.barrier()
    dist.destroy_process_group()
    print("rank", rank, "ok")
""")


def test_two_gloo_ranks_combine_to_the_unsharded_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(29500 + os.getpid() % 1000))
    procs = [subprocess.Popen([sys.executable, str(script), str(r), "2"], env=env,
                              stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        try:
            out, _ = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append((p.returncode, out))
    for rc, out in outs:
        assert rc == 0, out[-3000:]
        assert "ok" in out
