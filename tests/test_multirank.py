"""Host logic of the multi-GPU bench path on CPU: world_size 2 over gloo.  The solver
runs one replica per GPU (independent instances, no data-path collective); the only
exchange is the maximum over the ranks of the timed region, and the reference arm runs
on rank 0 alone.  Also the bench's whole-path roofline arithmetic (host only)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        out.put((rank, bench.rank_max_ms(times[rank], dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_timed_region_is_the_slowest_replica():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [123.5, 456.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 456.25, 1: 456.25}


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max_ms(7.5, None, "cpu") == 7.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_path_roofline_counts():
    import bench
    r = bench.path_roofline(2047, 256, 2048, 4, 29, "tf32", 1947.8, 6789.6, 55.0)
    # (s/2+1)(8/3)m^3 real flops of the 129 complex block LUs at m = 2047
    assert abs(r["setup_flops"] - 2.9506e12) / 2.9506e12 < 1e-4
    # 29 iterations: 20 + 9 Arnoldi steps, each the 4.333 GB factor stream plus its vectors
    vec = sum(4 + 4 * (i % 20 + 1) for i in range(29)) * 8.0 * 2047 * 256
    assert r["iteration_bytes"] == 29 * 129 * (2.0 * 2048 * 2048 * 4 + 4.0 * 2048 * 4) + vec
    assert 0.0 < r["frac"] < 1.0


def test_block_solve_bytes_by_factor_storage():
    """Algorithmic bytes of one block-solve launch: every stored factor entry once (Re and
    Im planes; 4 bytes in FP32, 2 in the bfloat16 copy) plus the FP32 right-hand side in
    and out; the whole-path roofline counts the same bytes per iteration."""
    import bench
    mp, nblk = 2048, 129
    assert bench.trsv_bytes(mp, nblk, 4) == nblk * (2.0 * mp * mp * 4 + 4.0 * mp * 4)
    assert bench.trsv_bytes(mp, nblk, 4, 2) == nblk * (2.0 * mp * mp * 2 + 4.0 * mp * 4)
    assert abs(bench.trsv_bytes(mp, nblk, 4, 2) - 2.168e9) / 2.168e9 < 1e-3
    r4 = bench.path_roofline(2047, 256, mp, 4, 26, "tf32", 1900.0, 6800.0, 35.0, restart=30)
    r2 = bench.path_roofline(2047, 256, mp, 4, 26, "tf32", 1900.0, 6800.0, 35.0, restart=30, fac_esz=2)
    assert r4["iteration_bytes"] - r2["iteration_bytes"] == 26 * nblk * 2.0 * mp * mp * 2
