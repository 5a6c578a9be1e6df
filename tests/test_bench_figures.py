"""The bench's roofline figures from the committed ncu summary of the rollout
kernel (no GPU): the figures block is read only while the rollout sources
hash to the value it records, so a kernel changed since its capture reports
null traffic and executed work instead of a stale number; the committed
summary carries every figure the bench reads, as numbers."""
import os

import bench

KEYS = ("dram_bytes_per_launch", "executed_fp32_gflop", "executed_fp32_frac_of_peak",
        "fma_pipe_active_frac", "alu_pipe_active_frac", "issue_active_frac",
        "warps_active_frac")


def _write(tmp_path, sha):
    p = tmp_path / "summary.md"
    lines = ["# a summary", "", f"    figure source_sha256: {sha}",
             "    figure workload: a test", "    figure dram_bytes_per_launch: 1234"]
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_figures_are_read_only_for_the_sources_they_were_taken_from(tmp_path):
    fig, src = bench.profile_figures(_write(tmp_path, bench.rollout_source_hash()))
    assert fig is not None and fig["dram_bytes_per_launch"] == "1234"
    fig, why = bench.profile_figures(_write(tmp_path, "0" * 16))
    assert fig is None and "changed" in why
    fig, why = bench.profile_figures(str(tmp_path / "missing.md"))
    assert fig is None


def test_the_committed_summary_has_every_figure_the_bench_reads():
    text = open(bench.ROLLOUT_PROFILE).read().splitlines()
    fig = {}
    for ln in text:
        ln = ln.strip()
        if ln.startswith("figure "):
            k, _, v = ln[len("figure "):].partition(":")
            fig[k.strip()] = v.strip()
    assert len(fig.get("source_sha256", "")) == 16
    for k in KEYS:
        float(fig[k])
    assert 0.0 < float(fig["issue_active_frac"]) <= 1.0
    assert os.path.basename(bench.ROLLOUT_PROFILE).startswith("k_rollout_")
