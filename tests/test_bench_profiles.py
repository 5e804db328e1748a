"""The committed ncu summaries the benchmark reads (run without a GPU):
the in-chain DRAM ratios and the traffic record parse, and hold values a
capture can produce."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_inchain_ratios_are_present_and_plausible():
    for profile, key in (("inchain_spmv_root_cd2d_1000.md", "dram_to_algorithmic_phi_f64"),
                         ("inchain_spmv_root_cd3d_160.md", "dram_to_algorithmic_phi_f64"),
                         ("inchain_spmv_root_cd3d_160.md", "dram_to_algorithmic_p_f32")):
        r = bench._inchain_ratio(profile, key)
        assert r is not None, (profile, key)
        assert 0.0 < r <= 1.5, (profile, key, r)


def test_traffic_record_has_its_keys():
    path = os.path.join(ROOT, "profiles", "spmv_root_cd2d_1000.txt")
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    assert len(vals["kernel_source_hash"]) == 16
    int(vals["kernel_source_hash"], 16)
    b = float(vals["dram_bytes_per_launch"])
    assert 1e6 < b < 1e9
    # the hash is the one the benchmark computes from the source it reads
    assert len(bench._kernel_source_hash()) == 16
