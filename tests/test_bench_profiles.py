"""bench.py's use of the committed ncu summaries (CPU only).

A bench line's roofline "traffic" comes from a profile summary under
profiles/ only while the kernel's source file still has the hash recorded
beside the capture.  Once the source changes, the figure is stale and the
bench reports null, so an old ncu figure never stands beside a new kernel.
Also checked: every committed summary names an existing source file, and
the hash check reads the file as bytes.
"""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tree(tmp_path, source_text, recorded_sha):
    csrc = tmp_path / "paper_2103_10882_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(source_text.encode())
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text("# k\n\nsource_file: k.cu\nsource_sha256_16: %s\ntraffic_bytes_per_launch: 1234\n"
                               % recorded_sha)
    return tmp_path


def test_traffic_kept_while_the_source_matches(tmp_path, monkeypatch):
    text = "__global__ void k() {}\n"
    sha = hashlib.sha256(text.encode()).hexdigest()[:16]
    monkeypatch.setattr(bench, "ROOT", str(_tree(tmp_path, text, sha)))
    assert bench.profiled_traffic("k.md", "traffic_bytes_per_launch") == 1234


def test_traffic_dropped_once_the_source_changed(tmp_path, monkeypatch):
    text = "__global__ void k() {}\n"
    sha = hashlib.sha256(text.encode()).hexdigest()[:16]
    root = _tree(tmp_path, text, sha)
    (root / "paper_2103_10882_gb300" / "csrc" / "k.cu").write_bytes(b"__global__ void k() { /* changed */ }\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("k.md", "traffic_bytes_per_launch") is None


def test_missing_profile_or_field_gives_null(tmp_path, monkeypatch):
    text = "x\n"
    root = _tree(tmp_path, text, hashlib.sha256(text.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("absent.md", "traffic_bytes_per_launch") is None
    assert bench.profiled_traffic("k.md", "traffic_bytes_per_launch_512") is None


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md")))
def test_committed_summaries_name_a_source_and_a_command(name):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    assert "ncu " in text and "--clock-control none" in text, "the command that made it"
    for line in text.splitlines():
        if line.startswith("source_file:"):
            src = line.split(":", 1)[1].strip()
            assert os.path.exists(os.path.join(ROOT, "paper_2103_10882_gb300", "csrc", src))
