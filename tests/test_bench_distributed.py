"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas with no data-path
collective) agree on the slowest rank's step time, the whole-job throughput
counts every rank's problems, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks_of(torch, 10.0 + 5.0 * rank, world, "cpu")
        value = bench.whole_job_throughput(world, 64, 600, ms)
        assert bench.dist_env() == (rank, world, rank)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_work():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 64 * 600 / 0.015)


def test_reference_arm_skips_nonzero_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                      "--warmup", "0"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""


def test_traffic_read_from_profile_summary_keyed_to_sources(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu summary only while
    the pass kernels' sources still hash to the value the summary records."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    h = hashlib.sha256()
    for f in ("passes.cuh", "sr_device.cuh", "sr_tma.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2409_05734_gb300", "csrc", f), "rb").read())
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text(f"# summary\n- dram_bytes_per_launch: 1234\n"
                               f"- kernel sources sha256[:16]: {h.hexdigest()[:16]}\n- a note: with a colon\n")
    (prof / "stale.md").write_text("- dram_bytes_per_launch: 1234\n- kernel sources sha256[:16]: 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2409_05734_gb300").symlink_to(os.path.join(ROOT, "paper_2409_05734_gb300"))
    assert bench.traffic_from_profile("k.md") == 1234.0
    assert bench.traffic_from_profile("stale.md") is None
    assert bench.traffic_from_profile("missing.md") is None


def test_only_legs_resolve_to_workload_functions():
    """`bench.py --only NAME` runs the function EXTRA_LEGS names; every name must
    resolve (a CPU check of the dispatch table, no GPU work)."""
    import bench
    for name, fn in bench.EXTRA_LEGS.items():
        assert callable(getattr(bench, fn)), name
    assert {"sweep", "layers", "small", "autograd", "radix3", "two_d", "forward_curve"} <= set(bench.EXTRA_LEGS)


def test_leg_parity_solver_is_the_oracle_protocol():
    """The bench's per-leg oracle solve (problem 0 of a leg, 1D and 2D) is the
    oracle's spectral initialisation plus GD with the bench's step rule on the
    leg's own signal, start vector and phases."""
    import numpy as np
    import bench
    import oracle as O
    import synthetic as S
    n, m, L, seed, sp, gd, B = 16, 64, 2, 5, 3, 4, 2
    got = bench.oracle_leg_solve(("1d", n, m, L, seed, sp, gd, B))
    fwd, adj = O.structured_ops(S.phases(seed, L, m), n, m)
    x = S.signal_gaussian(seed, B, n)[:1]
    y = np.abs(fwd(x)) ** 2
    x0 = O.spectral_init(y, S.start_vector(seed, B, n)[:1], fwd, adj, sp, mode="optimal", lam=-1.0)
    want, _ = O.gradient_descent(x0, y, fwd, adj, gd, mu0=bench.MU0, tau0=bench.TAU0)
    assert np.array_equal(got, want[0])
    h, S_ = 4, 8
    got2 = bench.oracle_leg_solve(("2d", h, S_, 3, seed, sp, gd, B))
    fwd2, adj2 = O.structured_ops_2d(S.phases(seed, 3, S_ * S_), h, h, S_)
    x2 = S.phase_image_ellipses(seed, B, h, h)[:1]
    y2 = np.abs(fwd2(x2)) ** 2
    x02 = O.spectral_init(y2, S.start_vector(seed, B, h * h)[:1], fwd2, adj2, sp, mode="optimal", lam=-1.0)
    want2, _ = O.gradient_descent(x02, y2, fwd2, adj2, gd, mu0=bench.MU0, tau0=bench.TAU0)
    assert np.array_equal(got2, want2[0])
