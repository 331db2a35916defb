"""The multi-GPU path is replicas only: every rank renders its own frames of
the same scene and the benchmark reports all ranks' frames over the slowest
rank's time.  This runs the host side of that path (process group, camera
dealing, max-over-ranks aggregation, barrier) as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2409_08669_gb300 import scenes as S
    w, r, local, pg = bench.dist_setup(None)
    assert (w, r) == (world, rank) and pg is not None
    cams = bench.deal_cameras(S.orbit_cameras(6, width=32, height=24), rank)
    bench.barrier(pg, device_sync=False)
    fps, t = bench.aggregate_fps(pg, 1.0 + rank, steps=10, world=world)
    out.put((rank, cams[0].cam_pos.tolist(), fps, t))
    pg.destroy_process_group()


def test_two_gloo_replicas_aggregate_over_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, cam0, fps0, t0), (r1, cam1, fps1, t1) = res
    assert cam0 != cam1                       # replicas render different frames
    assert t0 == t1 == 2.0                    # max over ranks
    assert fps0 == fps1 == pytest.approx(10 * world / 2.0)
