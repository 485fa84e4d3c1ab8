"""Host logic of bench.py's measurement records: the kernel-source hash that
decides whether an ncu traffic record still applies, and the record parser."""
import os
import shutil

import bench


def _copy_sources(tmp_path, edit=None):
    root = tmp_path / "repo"
    for rel in bench.KERNEL_SOURCES:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
        if edit:
            dst.write_text(edit(dst.read_text()))
    return str(root)


def _hash_at(monkeypatch, root):
    monkeypatch.setattr(bench, "ROOT", root)
    return bench.kernel_source_hash()


def test_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    base = _hash_at(monkeypatch, _copy_sources(tmp_path / "a"))
    commented = _copy_sources(
        tmp_path / "b", lambda s: "// a new comment\n/* and a block\n comment */\n" +
        s.replace("\n", "\n\n", 3))
    assert _hash_at(monkeypatch, commented) == base


def test_hash_changes_with_the_code(tmp_path, monkeypatch):
    base = _hash_at(monkeypatch, _copy_sources(tmp_path / "a"))
    changed = _copy_sources(tmp_path / "b", lambda s: s + "\nstatic int changed_code = 1;\n")
    assert _hash_at(monkeypatch, changed) != base


def test_traffic_record_parses_and_names_its_kernel(tmp_path, monkeypatch):
    # a record is used only for its own kernel and workload
    assert bench.recorded_traffic("some other kernel", "scale128", 10) is None
    assert bench.recorded_traffic("k_apply_coef<float> (A p from stored coefficients)",
                                  "another workload", 10) is None
    text = open(bench.TRAFFIC_PROFILE).read()
    for key in ("- kernel:", "- workload:", "- source_sha256:", "- dram_bytes_per_launch:",
                "- samples_per_launch:"):
        assert key in text
    # with the kernel sources of the record, the recorded bytes come back,
    # scaled from the captured case's samples to the asked-for samples
    rec = tmp_path / "rec.md"
    rec.write_text("- kernel: `K`\n- workload: `W`\n"
                   f"- source_sha256: `{bench.kernel_source_hash()}`\n"
                   "- dram_bytes_per_launch: `1234`\n- samples_per_launch: `100`\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(rec))
    assert bench.recorded_traffic("K", "W", 100) == 1234
    assert bench.recorded_traffic("K", "W", 250) == 3085
    rec.write_text(rec.read_text().replace(bench.kernel_source_hash(), "0" * 64))
    assert bench.recorded_traffic("K", "W", 100) is None


def test_cpu_model_is_a_name():
    m = bench.cpu_model()
    assert m is None or (isinstance(m, str) and len(m) > 0)


def test_committed_traffic_record_matches_the_kernel_sources():
    """The DRAM traffic record in profiles/ was taken on the kernel sources in
    the tree (else the bench line would report no traffic): a kernel change
    must come with a new capture."""
    kernel = "k_apply_coef<float> (A p from stored coefficients)"
    rec = bench.recorded_traffic(kernel, "scale128", 4413914798)
    assert rec is not None
    # the capture's bytes are within a few percent of the design bytes
    # (32 B per sample: the coefficient rows read twice)
    assert 0.9 * 32 * 4413914798 < rec < 1.1 * 32 * 4413914798


def test_lpc_summary_ratios():
    gn = {"paper": {"time_to_psnr_s": {"jacobi": 2.0, "learned": 1.0, "block_jacobi": None,
                                       "learned_objective_judge": 0.5}},
          "fixed2": {"time_to_psnr_s": {"jacobi": 4.0, "learned": 5.0}}}
    s = bench.lpc_summary(gn)
    assert s["paper"] == {"learned": 0.5, "block_jacobi": None, "learned_objective_judge": 0.25}
    assert s["fixed2"] == {"learned": 1.25}


def test_grid_option_scales_the_sample_cap():
    """--grid G keeps the workload's cameras and shells and sets the sample
    cap to 2 G, the ratio every grid workload uses (a ray crosses at most
    sqrt(3) G steps of 2/G)."""
    import argparse
    from scenegen import CONFIGS
    for name in ("scale128", "bf16_256", "small32"):
        assert CONFIGS[name].max_samples == 2 * CONFIGS[name].G
    base = bench._scene_config(argparse.Namespace(workload="scale128", grid=None))
    assert base == CONFIGS["scale128"]
    big = bench._scene_config(argparse.Namespace(workload="scale128", grid=512))
    assert (big.G, big.max_samples) == (512, 1024)
    assert (big.n_cams, big.width, big.radii, big.seed) == (base.n_cams, base.width, base.radii,
                                                           base.seed)


def test_traffic_record_scales_by_rows_streamed(tmp_path, monkeypatch):
    """A record taken on a launch that read every row, applied to a launch
    that reads a fraction of them (zero row tails skipped): the bytes scale
    by samples x rows-read over the capture's samples x rows-read."""
    rec = tmp_path / "rec.md"
    rec.write_text("- kernel: `K`\n- workload: `W`\n- source_sha256: `H`\n"
                   "- dram_bytes_per_launch: `1000`\n- samples_per_launch: `10`\n"
                   "- rows_read_fraction: `1.0`\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(rec))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "H")
    assert bench.recorded_traffic("K", "W", 40) == 4000
    assert bench.recorded_traffic("K", "W", 40, 0.5) == 2000
    rec.write_text(rec.read_text().replace("`1.0`", "`0.5`"))
    assert bench.recorded_traffic("K", "W", 40, 0.5) == 4000
    # without the field the capture is taken to have read every row
    rec.write_text(rec.read_text().replace("- rows_read_fraction: `0.5`\n", ""))
    assert bench.recorded_traffic("K", "W", 20) == 2000


class _FakeCtx:
    """Stands in for paper_2112_05598_gb300.Context in the bench's host
    helpers: records the calls and plays back counts."""

    def __init__(self, prefix=None, lanes=0, iters=2):
        self.prefix, self.lanes, self.iters = prefix, lanes, iters
        self.calls = []
        self.counter = None

    def coef_prefix(self):
        from paper_2112_05598_gb300 import PerfError
        if self.prefix is None:
            raise PerfError(2, "coef_prefix: the last Gauss-Newton step did not fill the store")
        return dict(read=self.prefix[0], total=self.prefix[1])

    def set_atomic_counter(self, t):
        self.counter = t
        self.calls.append(("counter", t is not None))

    def set_options(self, **kw):
        self.calls.append(("options", kw))

    def gn_solve(self, x, target, n):
        self.calls.append(("solve", n))
        if self.counter is not None:
            self.counter += self.lanes
        return [dict(pcg_iters=self.iters)]


def test_rows_read_fraction_of_the_last_step():
    assert bench.rows_read_fraction(_FakeCtx(prefix=(30, 40))) == 0.75
    assert bench.rows_read_fraction(_FakeCtx(prefix=(0, 0))) is None
    assert bench.rows_read_fraction(_FakeCtx(prefix=None)) is None


def test_count_lane_ops_per_apply_and_state_restored():
    """Lane operations per A p over one 2-iteration step on a copy of x; the
    counter is detached and the iteration count restored afterwards."""
    import torch
    ctx = _FakeCtx(lanes=600, iters=2)
    x = torch.zeros(8)
    assert bench.count_lane_ops(ctx, x, torch.zeros(3), 50) == 300.0
    assert ctx.calls == [("counter", True), ("options", {"pcg_iters": 2}), ("solve", 1),
                         ("counter", False), ("options", {"pcg_iters": 50})]
