"""Host-side bookkeeping of bench.py on the CPU: the dominant kernel's DRAM
traffic is reported from a recorded ncu capture only while the kernel's
sources still hash to the value recorded beside it, and the backward's
algorithmic work counts its hits alone (it reads the forward's hit masks
instead of testing candidate entries)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record(tmp_path, text):
    p = tmp_path / "record.txt"
    p.write_text(text)
    # recorded_traffic joins the record path onto the repository root; an
    # absolute path stays as it is
    return str(p)


def test_traffic_reported_while_sources_match(tmp_path):
    sha = bench.sources_sha1()
    rec = _record(tmp_path, "summary\n\ntraffic: kernel=k_x<3> bytes_per_launch=123456 source_sha1=" + sha + "\n")
    got, note = bench.recorded_traffic("k_x<3>", record=rec)
    assert got == 123456 and "ncu capture" in note


def test_traffic_withheld_after_a_source_change(tmp_path):
    rec = _record(tmp_path, "traffic: kernel=k_x<3> bytes_per_launch=123456 source_sha1=" + "0" * 40 + "\n")
    got, note = bench.recorded_traffic("k_x<3>", record=rec)
    assert got is None and "changed" in note


def test_traffic_of_another_kernel_or_no_record(tmp_path):
    rec = _record(tmp_path, "traffic: kernel=k_y<3> bytes_per_launch=1 source_sha1=" + bench.sources_sha1() + "\n")
    assert bench.recorded_traffic("k_x<3>", record=rec)[0] is None
    assert bench.recorded_traffic("k_x<3>", record=str(tmp_path / "missing.txt"))[0] is None


def test_source_hash_covers_every_kernel_source(tmp_path):
    a, b = tmp_path / "a.cu", tmp_path / "b.cuh"
    a.write_text("x")
    b.write_text("y")
    h0 = bench.sources_sha1((str(a), str(b)))
    b.write_text("z")
    assert bench.sources_sha1((str(a), str(b))) != h0


def test_backward_work_per_hit_includes_its_slab_test():
    # per hit: the segment's slab test plus the forward recompute and the
    # gradient; more than the forward's per-hit work for every K
    for K in (1, 2, 3):
        per_hit = bench.OPS_CAND + bench.OPS_HIT_BWD[K]
        assert per_hit > bench.OPS_CAND + bench.OPS_HIT[K]
    assert bench.OPS_CAND + bench.OPS_HIT_BWD[3] == 226
