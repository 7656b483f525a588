"""Host logic of bench.py that needs no GPU: a committed ncu summary feeds the
roofline only while its recorded source hash matches the kernel sources.
The committed k_cast summaries are checked for a traffic figure and a
source hash; one captured on other sources is reported as skipped (bench.py
then reports no traffic until the kernel is profiled again)."""
from __future__ import annotations

import hashlib
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _hash(sources):
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1706_07476_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_profiled_field_follows_the_source_hash(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1706_07476_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.CAST_SOURCES:
        (csrc / f).write_text(f"// {f}\n")
    good = hashlib.sha256("".join(f"// {f}\n" for f in bench.CAST_SOURCES).encode()).hexdigest()
    (prof / "k_cast_fp32_wl.md").write_text(
        f"# x\n\ntraffic_bytes_per_launch: 1234\nsource_sha256: {good}\n")
    assert bench.profiled_traffic("k_cast_fp32", "wl") == 1234.0
    assert bench.profiled_field("k_cast_fp32", "wl", "missing_field") is None
    assert bench.profiled_traffic("k_cast_fp32", "other") is None
    (csrc / bench.CAST_SOURCES[0]).write_text("// changed\n")  # the kernel changed since the capture
    assert bench.profiled_traffic("k_cast_fp32", "wl") is None


@pytest.mark.parametrize("name,sources", [
    ("k_cast_fp32_slab256.md", "CAST_SOURCES"),
    ("k_cast_fp32_graded.md", "CAST_SOURCES"),
    ("k_cast_batched_batched.md", "BATCHED_SOURCES"),
])
def test_committed_summaries_match_the_sources(bench, name, sources):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    m = re.search(r"^source_sha256: ([0-9a-f]{64})$", text, re.M)
    assert m, name
    assert re.search(r"^traffic_bytes_per_(launch|step): \d+$", text, re.M)
    if m.group(1) != _hash(getattr(bench, sources)):
        pytest.skip(f"{name} was captured on other kernel sources: profile again")
