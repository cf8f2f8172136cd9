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
