"""Host logic of bench.py that the GPU runs rely on: an ncu traffic figure is used
only while the kernel sources it was taken from are unchanged and, where the figure
names one, in the loop form it was captured in; whole-job throughput and the
single-rank reduction."""
import json

import bench


def _traffic(tmp_path, monkeypatch, entry):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"w": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda kind="single": "sha-" + kind)


def test_traffic_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    _traffic(tmp_path, monkeypatch, {"dram_bytes_per_iter": 7, "kernel_sha": "sha-single"})
    assert bench.ncu_traffic("w", "single")["dram_bytes_per_iter"] == 7
    assert bench.ncu_traffic("w", "fsai") is None          # taken from other sources
    assert bench.ncu_traffic("other", "single") is None    # no figure for this workload


def test_traffic_needs_the_loop_form_it_was_captured_in(tmp_path, monkeypatch):
    _traffic(tmp_path, monkeypatch, {"dram_bytes_per_iter": 7, "kernel_sha": "sha-fsai", "loop_form": "graph"})
    assert bench.ncu_traffic("w", "fsai", "graph")["dram_bytes_per_iter"] == 7
    assert bench.ncu_traffic("w", "fsai", "persistent") is None
    assert bench.ncu_traffic("w", "fsai") is not None     # no form to compare


def test_throughput_and_single_rank_reduction():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_throughput(4, 10, 2.0) == 20.0


def test_committed_traffic_figures_name_their_sources():
    d = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name, e in d.items():
        # a workload's loop, or one kernel of it ("workload:kernel")
        assert name.split(":")[0] in bench.WORKLOADS
        assert e["sources"] and e["how"] and len(e["kernel_sha"]) == 16


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    import shutil
    src = bench.os.path.join(bench.ROOT, "paper_2608_09647_gb300", "csrc")
    dst = tmp_path / "paper_2608_09647_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = bench.kernel_source_sha("batch")
    f = dst / "cg_batch.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("// Batched solves:", "/* reworded */ // Batched solves:", 1))
    assert bench.kernel_source_sha("batch") == before
    f.write_text(text.replace("constexpr int kNP = 4;", "constexpr int kNP = 5;", 1))
    assert bench.kernel_source_sha("batch") != before
