"""The benchmark's reader of ncu raw-page CSV exports: mean DRAM bytes (read
+ written) per launch and launch counts per kernel function, base units
required (no GPU)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

CSV = '''"==PROF== note"
"ID","Kernel Name","Block Size","dram__bytes_read.sum","dram__bytes_write.sum","gpu__time_duration.sum"
"","","","byte","byte","nsecond"
"0","void hmc::k_cg32_pmdag(hmc::Geo, hmc::Phase<float>, const float2 *)","(512, 1, 1)","26000000","600000","9000"
"1","hmc::k_cg32_m(hmc::Geo, hmc::Phase<float>)","(512, 1, 1)","40000000","8000000","9500"
"2","void hmc::k_cg32_pmdag(hmc::Geo, hmc::Phase<float>, const float2 *)","(512, 1, 1)","26,100,000","700000","9100"
'''


def test_means_and_counts_per_function():
    kernels, launches = bench.traffic_from_csv(CSV)
    assert launches == {"k_cg32_pmdag": 2, "k_cg32_m": 1}
    assert kernels["k_cg32_pmdag"] == pytest.approx((26.6e6 + 26.8e6) / 2)
    assert kernels["k_cg32_m"] == pytest.approx(48e6)


def test_scaled_units_are_refused():
    with pytest.raises(ValueError):
        bench.traffic_from_csv(CSV.replace('"byte","byte"', '"Mbyte","Mbyte"'))


def test_every_traffic_function_has_a_profile_name():
    assert set(bench.TRAFFIC_FUNCS.values()) >= {"k_cg32_pmdag", "k_cg32_m", "k_cg32_fused1", "k_cg32_resident2"}
    for f in bench.PAIR_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, f)), f


def test_write_traffic_merges_reports(tmp_path, monkeypatch):
    a, b = tmp_path / "a.csv", tmp_path / "b.csv"
    a.write_text(CSV)
    b.write_text(CSV.replace("k_cg32_pmdag", "k_cg32_fused1").replace("k_cg32_m(", "k_cg32_m2("))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0123456789abcdef")
    (tmp_path / "profiles").mkdir()
    bench.write_traffic([str(a), str(b)], ["ncu A", "ncu B"])
    import json
    rec = json.loads((tmp_path / "profiles" / "traffic.json").read_text())
    assert set(rec["kernels"]) == {"k_cg32_pmdag", "k_cg32_m", "k_cg32_fused1", "k_cg32_m2"}
    assert rec["source_sha"] == "0123456789abcdef" and rec["capture"] == ["ncu A", "ncu B"]
