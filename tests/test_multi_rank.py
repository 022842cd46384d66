"""Grid sharding over ranks (world size 2, gloo, CPU): the concatenated shards
equal the single-rank cross section bit for bit, with no data-path collective
other than the final gather of the disjoint slices."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1801_09803_gb300.shard import grid_shard, halo_line_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import oracle
    import xcsynth as xs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = xs.gen_lines(41, 0, 4000, 990.0, 1060.0)
    o = np.argsort(L["nu"], kind="stable")
    S = {k: v[o] for k, v in L.items()}
    E, g = xs.gen_states(41, 500)
    Q, dQ = oracle.partition_function(E, g, 1300.0)
    cond = oracle.make_condition(1300.0, 1.0, Q, dQ)
    # step 2^-7: every grid point nu_A + k*step is exact in binary, so a shard that starts
    # its own grid at point k0 produces bit-identical grid points
    nu_A, step, n, cut = 1000.0, 1.0 / 128.0, 6401, 5.0
    k0, k1 = grid_shard(n, world, rank)
    l0, l1 = halo_line_range(S["nu"], nu_A, step, k0, k1, cut)
    sub = {k: v[l0:l1] for k, v in S.items()}
    part = oracle.cross_section(sub, cond, nu_A + k0 * step, step, k1 - k0, oracle.make_opts("voigt_w4", cut))
    # gather the disjoint slices (sizes differ by at most one point)
    size = torch.tensor([k1 - k0])
    sizes = [torch.zeros(1, dtype=torch.long) for _ in range(world)]
    dist.all_gather(sizes, size)
    mx = int(max(s.item() for s in sizes))
    buf = torch.zeros(mx, dtype=torch.float64)
    buf[: k1 - k0] = torch.from_numpy(part)
    bufs = [torch.zeros(mx, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, buf)
    if rank == 0:
        full = np.concatenate([b[: int(s.item())].numpy() for b, s in zip(bufs, sizes)])
        ref = oracle.cross_section(S, cond, nu_A, step, n, oracle.make_opts("voigt_w4", cut))
        out.put((bool(np.array_equal(full, ref)), int((l1 - l0)), len(S["nu"])))
    dist.barrier()
    dist.destroy_process_group()


def test_grid_shards_concatenate_to_the_full_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    equal, halo_lines, total = q.get(timeout=180)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert equal
    assert halo_lines < total  # each rank reads only its halo range


def test_grid_shard_covers_the_grid():
    for n in (0, 1, 7, 200001):
        for world in (1, 2, 3, 8):
            parts = [grid_shard(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
