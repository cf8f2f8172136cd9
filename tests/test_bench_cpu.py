"""Host logic of bench.py that needs no GPU: the oracle's timed window and
the extrapolation of its time per iteration, and the aggregation of
replicas under torchrun."""

import bench


def test_extrapolation_fits_the_growth_exponent():
    small = {"per_iter_s": 1.0, "dofs": 1000}
    large = {"per_iter_s": 8.0 * 2 ** 0.5, "dofs": 8000}      # ~ DOFs^(7/6)
    alpha, t = bench.extrapolate_time(small, large, 64000)
    assert abs(alpha - 7.0 / 6.0) < 1e-12
    assert abs(t - large["per_iter_s"] * 8.0 ** alpha) < 1e-9


def test_extrapolation_never_grows_slower_than_linear():
    alpha, t = bench.extrapolate_time({"per_iter_s": 1.0, "dofs": 1000},
                                      {"per_iter_s": 2.0, "dofs": 8000}, 16000)
    assert alpha == 1.0 and t == 4.0


def test_oracle_window_times_the_requested_iterations():
    w = bench.oracle_window("24x12x12", 1, 2)
    assert w["iterations"] == "2..3" and len(w["seconds"]) == 2
    assert w["dofs"] == 3 * 25 * 13 * 13
    assert sum(w["branches"].values()) == 2 and w["per_iter_s"] > 0.0


# ---------------------------------------------------------------------------
# replicas under torchrun: the slowest rank's time and the whole-job rate,
# exercised with two gloo ranks on the host
# ---------------------------------------------------------------------------

def _replica_rank(rank, world, port, seconds, steps, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        slow = bench.slowest_rank(seconds[rank], world, device="cpu")
        out.put((rank, slow, bench.whole_job_rate(steps, world, slow)))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_report_the_slowest_rank_and_the_summed_rate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    seconds, steps, world = [1.5, 2.5], 10, 2
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank, args=(r, world, port, seconds, steps, out))
             for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate in results:
        assert slow == 2.5
        assert rate == world * steps / 2.5


def test_single_process_uses_its_own_time():
    assert bench.slowest_rank(3.0, 1) == 3.0
    assert bench.whole_job_rate(27, 1, 3.0) == 9.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the CPU reference arm does its work on rank 0; other
    ranks return without timing anything."""
    import argparse
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_window",
                        lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran on rank 1")))
    args = argparse.Namespace(warmup=3, steps=2, precision="mixed")
    assert bench.run_reference(args) is None
