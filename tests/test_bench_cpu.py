"""Host logic of bench.py that needs no GPU: reading the per-launch DRAM
traffic of the dominant kernel from the committed ncu summary."""

import hashlib
import os

import bench


def _fake_tree(tmp_path, source: bytes, record_sha: str, nbytes: str):
    csrc = tmp_path / "paper_2205_00385_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "kernels_pair.cu").write_bytes(source)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "apply_pair_cantilever192.md").write_text(
        "# summary\n\n"
        "- note: a line whose value: has colons\n"
        f"- kernels_pair.cu sha256[:16]: `{record_sha}`\n"
        f"- k_apply3_pair dram bytes per launch: `{nbytes}`\n")


def test_traffic_read_when_the_source_hash_matches(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    sha = hashlib.sha256(src).hexdigest()[:16]
    _fake_tree(tmp_path, src, sha, "30485760")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profiles("k_apply3_pair") == 30485760.0


def test_traffic_dropped_when_the_kernel_changed(tmp_path, monkeypatch):
    _fake_tree(tmp_path, b"new source\n", "0123456789abcdef", "30485760")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_from_profiles("k_apply3_pair") is None


def test_committed_summary_names_the_kernel_source_hash():
    path = os.path.join(bench.ROOT, "profiles", "apply_pair_cantilever192.md")
    text = open(path).read()
    assert "- kernels_pair.cu sha256[:16]: `" in text
    assert "- k_apply3_pair dram bytes per launch: `" in text


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
    monkeypatch.setattr(bench, "cpu_baseline",
                        lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran on rank 1")))
    args = argparse.Namespace(warmup=3, steps=2, precision="mixed")
    assert bench.run_reference(args) is None
