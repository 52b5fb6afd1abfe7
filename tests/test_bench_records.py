"""bench.py's JSONL records (host logic): one record per measurement of a
bench line, with throughput, roofline fraction, errors and host cores."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

LINE = {
    "metric": "m", "value": 174.1, "unit": "Gcell/s", "n_gpus": 1, "ms_per_step": 0.771,
    "config": {"workload": "abc512_cec_f32", "launch": {"kernel": "cec_fast", "ctas_per_sm": 2}},
    "roofline": {"achieved": 3480.0, "peak": 6742.6, "frac": 0.516, "traffic": 4.1e9},
    "e2e": {"value": 11.9, "h2d_bytes_per_step": 2 ** 31, "d2h_bytes_per_step": 2 ** 29},
    "cpu_baseline": {"value": 0.17, "cores": 16, "sample": "s"},
    "clocks": {"sm_mhz": 2070.0},
    "schemes": {"CIR": {"gcell_s": 285.5, "ms_per_step": 0.47, "roundtrip_rel_l2_100_100": 0.38, "launch": {}}},
    "batched_c3": {"batched_graph": {"gcell_s": 129.0}, "plain_48_launches": {"gcell_s": 68.0}, "launch": {}},
    "deformation_c5": {"field_gcell_s": 184.0, "rel_l2_at_T": {"u": 3.6e-4}},
    "rotation_c1": {"grid": [128, 128], "CEC": {"rel_l2": 0.0196, "linf": 0.0297, "us_per_step": 13.0}},
}


def test_records_cover_every_measurement(tmp_path):
    recs = bench.jsonl_records(LINE, when="t")
    kinds = [r["record"] for r in recs]
    assert kinds == ["headline", "e2e", "cpu_baseline", "scheme", "batched_c3", "deformation_c5", "rotation_c1"]
    head = recs[0]
    assert head["gcell_s"] == 174.1 and head["roofline_frac"] == 0.516 and head["gb_s"] == 3480.0
    cir = recs[3]
    assert abs(cir["gb_s"] - 285.5 * 20) < 1e-6 and abs(cir["roofline_frac"] - 285.5 * 20 / 6742.6) < 1e-9
    assert recs[2]["host_cores"] == 16
    assert recs[6]["CEC"] == {"rel_l2_vs_exact": 0.0196, "linf_vs_exact": 0.0297}
    p = tmp_path / "m.jsonl"
    bench.write_jsonl(str(p), LINE)
    bench.write_jsonl(str(p), LINE)
    lines = p.read_text().splitlines()
    assert len(lines) == 2 * len(recs)
    assert all(json.loads(x)["record"] for x in lines)


def test_records_of_the_learned_and_rayleigh_benard_measurements():
    line = dict(LINE)
    line["learned_c4"] = {"learned_gcell_s": 20.3, "roofline": {"frac": 0.18}, "fell_back_at_step": 125,
                          "checks": [{"step": 0}],
                          "deformation_c5_learned": {"fell_back_at_step": 0, "rel_l2_at_T": {"u": 3.6e-4}}}
    line["rayleigh_benard_f4"] = {"grid": [50, 50], "device_status": 0,
                                  "CIR": {"us_per_step": 21.5, "top_reached_at_step": 990},
                                  "CEC": {"us_per_step": 29.4, "top_reached_at_step": 970},
                                  "cpu_baseline": {"value": 857.0}}
    recs = bench.jsonl_records(line, when="t")
    kinds = [r["record"] for r in recs]
    i = kinds.index("learned_c4")
    assert kinds[i + 1] == "deformation_c5_learned" and kinds[-1] == "rayleigh_benard_f4"
    assert recs[i + 1]["fell_back_at_step"] == 0 and recs[i + 1]["rel_l2_vs_exact"] == {"u": 3.6e-4}
    rb = recs[-1]
    assert rb["grid"] == [50, 50] and rb["CEC"] == {"us_per_step": 29.4, "top_reached_at_step": 970}
    assert "cpu_baseline" not in rb and "device_status" not in rb
