"""The N > 1 path of bench.py on CPU: replicas with a gloo process group
(world size 2, 127.0.0.1).  The path has no data-path collective: every rank
walks its own full workload; the job's step time is the slowest rank's
(barrier + all-reduce MAX) and the job's throughput counts every rank's rays.
The reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [7.5, 9.25][rank]  # rank 1 is the slower replica
        ms = bench.job_step_ms(dist, local_ms)
        value = bench.job_rays_per_s(1000, world, ms)
        # the reference arm: rank 0 runs and prints, the others return 0 without work
        ref = None
        if rank != 0:
            class A:
                steps, warmup, gpus = 1, 1, world
            ref = bench.run_reference(A())
        out.put((rank, ms, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_and_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, _), (r1, ms1, v1, ref1) = res
    assert ms0 == ms1 == 9.25  # every rank reports the slowest rank's time
    assert v0 == v1 == pytest.approx(1000 * 2 / 9.25e-3)
    assert ref1 == 0


def test_single_process_is_identity():
    assert bench.job_step_ms(None, 3.5) == 3.5
    assert bench.job_rays_per_s(10, 1, 2.0) == pytest.approx(5000.0)


def test_roofline_object_schema():
    """The bench's roofline object: bound = the L2's random-sector gather rate
    measured live (achieved / peak = frac), the HBM copy peak and the DRAM
    traffic beside it as top-level numbers."""
    import bench

    r = bench.make_roofline(5000.0, 9000.0, 6775.3, "MEASURED_PEAKS.json hbm_gbs (of measured)", 4.47e9, "note",
                            5.8, 3.1e10, 4.2e10)
    assert r["bound"] == "l2_gather" and r["unit"] == "GB/s" and r["peak"] == 9000.0
    assert abs(r["frac"] - 5000.0 / 9000.0) < 1e-12 and r["traffic"] == 4.47e9
    assert abs(r["hbm_frac_of_algorithmic"] - 5000.0 / 6775.3) < 1e-12
    assert abs(r["dram_frac"] - 4.47e9 / 5.8e-3 / 1e9 / 6775.3) < 1e-12
    assert abs(r["l2_over_algorithmic"] - 4.2e10 / 3.1e10) < 1e-12
    for key in ("achieved", "peak", "unit", "frac", "traffic", "bound"):
        assert key in r
    # every value is a scalar, so a flat parse of the line keeps them all
    assert all(not isinstance(v, (dict, list)) for v in r.values())
    r = bench.make_roofline(5000.0, 9000.0, 6775.3, "src", None, "kernel changed", 5.8, 3.1e10)
    assert r["traffic"] is None and r["dram_frac"] is None and r["l2_over_algorithmic"] is None


def test_committed_traffic_summary_is_readable():
    """The committed ncu summary the bench reads for `roofline.traffic` parses:
    its figures come back when the kernel sources hash to the recorded value,
    else the bench says the kernel changed (never that the summary is missing
    or unreadable)."""
    import bench

    traffic, note, l2 = bench.captured_traffic()
    if traffic is None:
        assert note == "kernel changed since the ncu capture"
    else:
        assert traffic > 1e9 and l2 is not None and l2 > traffic and "from" in note
