"""The bench's DRAM-traffic lookup (`bench.measured_traffic`): a committed
capture holds only for the kernel sources and the plan variant it was taken
with, and is scaled by the gathers of the launch.  Checked on a synthetic
profile table (not the committed one, whose rows follow the kernels)."""
import bench


def _table(tmp_path, rows):
    text = ["# traffic\n", "\n", "| kernel | gathers per launch | bytes per launch | source hash "
            "| variant | launch |\n", "|---|---|---|---|---|---|\n"]
    text += ["| %s | %s | %s | %s | %s | x |\n" % r for r in rows]
    p = tmp_path / "dram_traffic.md"
    p.write_text("".join(text))
    return str(p)


def test_lookup_scales_and_keys(tmp_path, monkeypatch):
    h = bench.source_hash("stolt_adj_rows")
    path = _table(tmp_path, [
        ("stolt_adj_rows", 8, 800, "0" * 12, "9/16"),        # other sources: ignored
        ("stolt_adj_rows", 8, 1000, h, "4/16"),             # other variant: ignored
        ("stolt_adj_rows", 8, 1600, h, "9/16"),
    ])
    monkeypatch.setattr(bench, "TRAFFIC_FILE", path)
    assert bench.measured_traffic("stolt_adj_rows", 64, (9, 16)) == (1600.0 / 8 * 64, h)
    assert bench.measured_traffic("stolt_adj_rows", 8, (4, 16)) == (1000.0, h)
    assert bench.measured_traffic("stolt_adj_rows", 8, (5, 16)) == (None, h)


def test_lookup_without_a_capture(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.measured_traffic("xfft_r2c", 64) == (None, None)
    path = _table(tmp_path, [("xfft_c2r", 8, "n/a", bench.source_hash("xfft_c2r"), "9/16")])
    monkeypatch.setattr(bench, "TRAFFIC_FILE", path)
    assert bench.measured_traffic("xfft_c2r", 64)[0] is None


def test_source_hash_follows_the_sources():
    # every timed class hashes its own files; the row kernels share some
    hashes = {k: bench.source_hash(k) for k in bench.KERNEL_SOURCES}
    assert all(len(h) == 12 for h in hashes.values())
    assert len(set(hashes.values())) == len(hashes)
