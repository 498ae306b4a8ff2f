"""The multi-GPU path is replicas only: each rank runs the whole workload on its own GPU and
bench.py reduces the per-step time with a max over ranks behind barriers.  That host logic is
checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(1.5 + rank, world)          # per-rank step times
        args = type("A", (), {"workload": "small", "warmup": 0, "steps": 1, "gpus": world})()
        bench.run_reference(args, rank, world) if rank != 0 else None   # non-zero ranks return at once
        bench.barrier(world)
        out[rank] = m
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        assert out[0] == out[1] == 2.5


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    bench.barrier(1)


def test_serving_child_failure_is_reported():
    """The serving measurement runs in a child interpreter; without a GPU that child exits
    non-zero, and the parent raises with the child's error instead of returning a result."""
    import bench
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the child would run the real measurement")
    with pytest.raises(RuntimeError, match="serving measurement failed"):
        bench.serving_in_child(0)


def test_traffic_is_reported_only_for_its_workload_and_sources():
    """A stored DRAM-traffic figure comes back only for the workload it was captured on and
    while its kernel's source files still hash to the recorded value; otherwise null."""
    import hashlib

    import bench
    assert bench.TRAFFIC, "no stored traffic figures"
    for kernel, t in bench.TRAFFIC.items():
        m = hashlib.sha256()
        for name in t["files"]:
            with open(os.path.join(bench.ROOT, "paper_2608_03778_gb300", "csrc", name), "rb") as f:
                m.update(f.read())
        current = m.hexdigest()[:16] == t["sha"]
        assert bench.kernel_traffic(kernel, t["workload"]) == (t["bytes"] if current else None)
        assert bench.kernel_traffic(kernel, t["workload"] + "_other") is None
    assert bench.kernel_traffic("no_such_kernel", "roofline") is None
