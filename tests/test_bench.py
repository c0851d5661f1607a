"""CPU checks of bench.py's measurement plumbing: the algorithmic work each
roofline is measured against (the counts stated for every kernel), the parser
of ncu's CSV logs and the DRAM-traffic table writer."""
import json
import os

import numpy as np
import pytest

import bench
import synth


def test_roofline_models_state_the_algorithmic_counts():
    cfg = synth.make_config("full")
    n_kept = 259_400_000
    models, peak_of = bench.roofline_models(cfg, n_kept, (6798.9, 1904.1, 2070.0, "measured"))
    n_chan = cfg.n_chan_total
    d = (np.arange(cfg.image_size) - cfg.image_size // 2) * cfg.cell
    vox = int(((d[None, :] ** 2 + d[:, None] ** 2) < 1.0).sum()) * n_chan
    # gridding: 2 x 49 taps x 4 flops per gridded visibility, on the FP32 ALU
    assert models["k_grid_tiles"][:3] == ("alu", n_kept * 392, "FLOP")
    # detection kernels per in-horizon voxel: one SNR read for the NMS pass,
    # z' in and SNR + width out for the boxcars, the stream and ranks for the walk
    assert models["k_nms_warp"][1] == vox * 4
    assert models["k_mf"][1] == vox * 9
    assert models["k_walk"][1] == vox * 8
    assert models["k_median_sub"][1] == vox * 12
    # every model is a positive amount against a peak of its own bound
    for k, (bound, amount, unit, units) in models.items():
        assert amount > 0 and units > 0, k
        assert bound in peak_of and peak_of[bound] > 0, k
        assert unit in ("B", "FLOP"), k
    # the derived FP32 peak: 152 SMs x 128 lanes x 2 flops x the max SM clock
    assert peak_of["alu"] == pytest.approx(152 * 128 * 2 * 2070.0e6 / 1e12)


def _csv(path, rows):
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')
    with open(path, "w") as f:
        f.write("==PROF== Connected to process 1\n")
        f.write(head)
        for lid, name, metric, unit, value in rows:
            f.write(f'"{lid}","1","python3","127.0.0.1","{name}","1","7","(1024, 1, 1)","(152, 1, 1)","0","10.3",'
                    f'"Command line profiler metrics","{metric}","{unit}","{value}"\n')


def test_ncu_rows_take_base_names_and_units(tmp_path):
    p = tmp_path / "l.csv"
    _csv(p, [(0, "void ovro::<unnamed>::k_walk<true, 128>(const unsigned int *, int)", "dram__bytes_read.sum",
              "Mbyte", "1.5"),
             (0, "void ovro::<unnamed>::k_walk<true, 128>(const unsigned int *, int)", "gpu__time_duration.sum",
              "us", "2,000.5"),
             (1, "ovro::<unnamed>::k_mf(const float *)", "dram__bytes_write.sum", "byte", "64")])
    rows = bench._ncu_rows(str(p))
    assert rows == [("0", "k_walk", "dram__bytes_read.sum", 1.5e6),
                    ("0", "k_walk", "gpu__time_duration.sum", 2000.5e3),
                    ("1", "k_mf", "dram__bytes_write.sum", 64.0)]


def test_traffic_table_divides_by_the_case_work_and_maps_names(tmp_path, monkeypatch):
    root = tmp_path / "root"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2606_04304_gb300" / "csrc").mkdir(parents=True)
    for src in set(bench.KERNEL_SRC.values()):
        (root / "paper_2606_04304_gb300" / "csrc" / src).write_text("// source\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    p = tmp_path / "t.csv"
    repeats, units, _ = bench.CASE_META["detection"]
    u = repeats * units["k_rank"]
    # the band kernel and the fallback launch both count under the traced name
    _csv(p, [(3, "void ovro::<unnamed>::k_rank_band<8>(const float *)", "dram__bytes_read.sum", "byte", str(3 * u)),
             (3, "void ovro::<unnamed>::k_rank_band<8>(const float *)", "dram__bytes_write.sum", "byte", str(u)),
             (4, "void ovro::<unnamed>::k_rank(const float *)", "dram__bytes_read.sum", "byte", str(u)),
             (5, "void ovro::<unnamed>::k_stats(const float *)", "dram__bytes_read.sum", "byte", str(2 * u))])
    bench.write_traffic_table("detection", str(p), "ncu ... --profile-case detection")
    t = json.load(open(os.path.join(root, "profiles", "dram_traffic.json")))["kernels"]
    assert t["k_rank"]["read_bytes_per_unit"] == pytest.approx(4.0)
    assert t["k_rank"]["write_bytes_per_unit"] == pytest.approx(1.0)
    assert t["k_rank"]["launches"] == 2
    assert t["k_stats"]["dram_bytes_per_unit"] == pytest.approx(2.0)
    # the table is kept only while the kernel's source is unchanged
    assert "k_rank" in bench._traffic_table()
    (root / "paper_2606_04304_gb300" / "csrc" / "detect.cu").write_text("// changed\n")
    assert "k_rank" not in bench._traffic_table()
