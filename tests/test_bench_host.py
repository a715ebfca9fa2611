"""Host-side logic of the benchmark (no GPU): the serving stream's memory
guard, the roofline records keyed to the kernels' sources, and the roofline
arithmetic."""
import json

import pytest

import bench
from paper_2501_02317_gb300 import workloads as wl


def test_serving_prefix_keeps_the_whole_stream_when_it_fits():
    jobs = wl.serving_stream(50, seed=4)
    need = sum((j.ndim + 2) * j.side ** j.ndim * 8 for j in jobs)
    assert bench.serving_prefix(jobs, None) == (50, None)
    assert bench.serving_prefix(jobs, 2 * need) == (50, None)


def test_serving_prefix_cuts_the_stream_to_half_the_free_memory():
    jobs = wl.serving_stream(50, seed=4)
    sizes = [(j.ndim + 2) * j.side ** j.ndim * 8 for j in jobs]
    avail = sum(sizes)  # room for about half of the stream's states, twice over
    keep, note = bench.serving_prefix(jobs, avail)
    assert 0 < keep < 50 and note and ("first %d of 50 jobs" % keep) in note
    assert 2 * sum(sizes[:keep]) <= avail < 2 * sum(sizes[:keep + 1])


def _with_record(monkeypatch, tmp_path, rec):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "stage_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def test_recorded_traffic_is_keyed_to_sources_and_workload(monkeypatch, tmp_path):
    sha = bench.stage_sources_sha256()  # of the real sources, before ROOT moves
    rec = {"workload": "turbulence-3d-256^3-mixed", "stage_sources_sha256": sha,
           "stage1_dram_bytes": 2.0e9, "stage2_dram_bytes": 2.5e9,
           "stage1_warp_inst": 6.0e8, "stage2_warp_inst": 5.0e8}
    _with_record(monkeypatch, tmp_path, rec)
    monkeypatch.setattr(bench, "stage_sources_sha256", lambda *a: sha)
    assert bench._recorded_traffic("turbulence-3d-256^3-mixed") == 4.5e9
    assert bench._recorded_warp_inst("turbulence-3d-256^3-mixed") == 1.1e9
    # another workload, or sources changed since the capture: no number
    assert bench._recorded_traffic("turbulence-3d-128^3-mixed") is None
    monkeypatch.setattr(bench, "stage_sources_sha256", lambda *a: "0" * 64)
    assert bench._recorded_traffic("turbulence-3d-256^3-mixed") is None
    assert bench._recorded_warp_inst("turbulence-3d-256^3-mixed") is None


def test_committed_records_name_their_workloads():
    # the committed records must be keyed (a record without its key would
    # be used for any source tree)
    for name, keys in (("stage_traffic.json", ("workload", "stage_sources_sha256")),
                       ("fp64_stage_ops.json", ("workload", "sources_sha256"))):
        with open("%s/profiles/%s" % (bench.ROOT, name)) as f:
            rec = json.load(f)
        for k in keys:
            assert rec.get(k), (name, k)


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "_recorded_warp_inst", lambda w: 1.0e9)
    r = bench.issue_roofline(1.0, 1 << 20, "w", 152, 2000.0)
    peak = 4 * 152 * 2000.0e6
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(1.0e12)
    assert r["frac"] == pytest.approx(1.0e12 / peak)
    assert r["thread_inst_per_cell_update"] == pytest.approx(32.0e9 / (1 << 20))
    monkeypatch.setattr(bench, "_recorded_warp_inst", lambda w: None)
    assert bench.issue_roofline(1.0, 1 << 20, "w", 152, 2000.0)["frac"] is None


def test_fp64_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "fp64_ops_per_cell_update", lambda w: 2000.0)
    r = bench.fp64_roofline(10.0, 1000, "w", 152, 2000.0)
    peak = bench.FP64_PER_CLK_PER_SM * 152 * 2000.0e6
    assert r["achieved"] == pytest.approx(2000.0 * 1000 / 1e-2 / 1e12)
    assert r["frac"] == pytest.approx(2000.0 * 1000 / 1e-2 / peak)
    monkeypatch.setattr(bench, "fp64_ops_per_cell_update", lambda w: None)
    assert bench.fp64_roofline(10.0, 1000, "w", 152, 2000.0)["frac"] is None
