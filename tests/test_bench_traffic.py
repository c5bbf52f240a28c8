"""bench.py's roofline `traffic`: the committed ncu figure is used only for
the workload it was measured on and only while the kernel sources still hash
to the value recorded with it."""
import json

import bench


def _table(tmp_path, monkeypatch, d):
    h = bench.source_hash()  # of the real sources, before ROOT moves
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: h)


def test_traffic_scales_the_per_spectrum_bytes(tmp_path, monkeypatch):
    h = bench.source_hash()
    _table(tmp_path, monkeypatch, {"c2": {"rowfft_detect": {"source_hash": h, "dram_bytes_per_spectrum": 1000.0}}})
    assert bench._traffic("c2", "rowfft_detect", 250) == 250000.0


def test_traffic_is_null_for_another_workload_kernel_or_source(tmp_path, monkeypatch):
    h = bench.source_hash()
    _table(tmp_path, monkeypatch, {"c2": {"fir_colfft": {"source_hash": h, "dram_bytes_per_spectrum": 1.0},
                                          "rowfft_detect": {"source_hash": "0" * 16, "dram_bytes_per_spectrum": 1.0}}})
    assert bench._traffic("c3", "fir_colfft", 10) is None       # measured on another workload
    assert bench._traffic("c2", "reduce", 10) is None           # no capture of this kernel
    assert bench._traffic("c2", "rowfft_detect", 10) is None    # sources changed since the capture


def test_committed_table_names_workloads_and_hashes():
    with open(bench.os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as f:
        d = json.load(f)
    for cfg, kernels in d.items():
        if cfg.startswith("_"):
            continue
        assert cfg in ("c1", "c2", "c3", "c4", "c5")
        for ent in kernels.values():
            assert len(ent["source_hash"]) == 16 and ent["dram_bytes_per_spectrum"] > 0
