"""Multi-rank host logic of bench.py on CPU: world_size 2 over gloo, each rank an independent
replica; the reported time is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, loc = bench.dist_env()
    value = bench.max_over_ranks(1.5 + 2.0 * rank)          # rank-specific "step time"
    dist.barrier()
    q.put((r, w, loc, value))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 3.5 for o in out)        # both ranks report the slowest rank's value
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(2.25) == 2.25


def test_gl_flop_model_and_rel_l2():
    import math

    import torch

    import bench
    # 512^2 grid, 768^2 padded: (512 + 768) * 5 * 768 * log2(768) per transform, two per stage,
    # plus 11 flops per padded point and 16 per retained coefficient; four stages
    fft = 5 * 768 * math.log2(768)
    expect = 4 * (2 * 1280 * fft + 11 * 768 ** 2 + 16 * 512 ** 2)
    assert abs(bench.gl_flops_per_step(512) - expect) < 1e-6 * expect
    assert 0.41e9 < bench.gl_flops_per_step(512) < 0.43e9
    assert abs(bench.FP32_PEAK_TFLOPS - 80.5) < 0.1
    a = torch.tensor([1 + 1j, 2.0], dtype=torch.complex64)
    b = torch.tensor([1 + 1j, 2.0 + 1e-3], dtype=torch.complex128)
    assert abs(bench.rel_l2(a, b) - 1e-3 / math.sqrt(2 + 2.001 ** 2)) < 1e-9
