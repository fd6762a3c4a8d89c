"""The DRAM-traffic record behind the bench line's roofline `traffic`: the
ncu CSV parser (unit column, kernel-name spelling, per-launch averages) and
the lookup, which scales a capture on a smaller box of the same recipe by
the list entry count and refuses a record taken on other device code or
another recipe."""
import json

import pytest

from paper_1211_4406_gb300 import profile_step as ps

HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
       '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
KV = "void <unnamed>::k_vjp_fused<4, 1, 0>(TreeDev, const float *, double *, double *)"
KP = "void <unnamed>::k_pair_packed<2, 0>(TreeDev, float *, int *)"
KO = "<unnamed>::k_keys(const double *, long, unsigned long *, unsigned int *, int *)"


def row(i, kernel, metric, unit, value):
    cells = (i, 1364, "python3.12", "127.0.0.1", kernel, 1, 7, "(256, 1, 1)", "(152, 1, 1)", 0, "10.3",
             "Command line profiler metrics", metric, unit, value)
    return ",".join(f'"{c}"' for c in cells)


def write_csv(path, rows):
    path.write_text("\n".join(["==PROF== Connected to process 1364", HDR] + rows) + "\n")


def test_parser_scales_units_and_averages_launches(tmp_path):
    csv_path, out = tmp_path / "l.csv", tmp_path / "traffic.json"
    write_csv(csv_path, [
        row(0, KO, "dram__bytes_read.sum", "byte", "999"),
        row(3, KV, "dram__bytes_read.sum", "Gbyte", "5.00"),
        row(3, KV, "dram__bytes_write.sum", "Mbyte", "250"),
        row(3, KV, "gpu__time_duration.sum", "msecond", "17.5"),
        row(9, KV, "dram__bytes_read.sum", "byte", "5,100,000,000"),
        row(9, KV, "dram__bytes_write.sum", "byte", "150000000"),
        row(9, KV, "gpu__time_duration.sum", "usecond", "17300"),
        row(4, KP, "dram__bytes_read.sum", "Kbyte", "3000000"),
        row(4, KP, "dram__bytes_write.sum", "byte", "0"),
        row(4, KP, "gpu__time_duration.sum", "ns", "9500000"),
    ])
    rec = ps.record_traffic(str(csv_path), 128 ** 3, out_path=str(out), entries=190000000)
    assert rec["recipe"] == "clustered" and rec["n"] == 128 ** 3 and rec["entries"] == 190000000
    assert rec["digest"] == ps.kernel_source_digest()
    k = rec["kernels"]
    assert set(k) == {"k_vjp_fused<4,1,0>", "k_pair_packed<2,0>"}     # other kernels are ignored
    assert k["k_vjp_fused<4,1,0>"]["bytes_per_launch"] == pytest.approx(5.25e9)
    assert k["k_vjp_fused<4,1,0>"]["ncu_ms_per_launch"] == pytest.approx(17.4)
    assert k["k_pair_packed<2,0>"]["bytes_per_launch"] == pytest.approx(3e9)
    assert k["k_pair_packed<2,0>"]["ncu_ms_per_launch"] == pytest.approx(9.5)
    assert json.loads(out.read_text()) == rec


def test_parser_rejects_an_unknown_unit(tmp_path):
    csv_path = tmp_path / "l.csv"
    write_csv(csv_path, [row(1, KV, "dram__bytes_read.sum", "furlong", "3")])
    with pytest.raises(ValueError):
        ps.record_traffic(str(csv_path), 1024, out_path=str(tmp_path / "t.json"))


def test_lookup_scales_by_entries_and_refuses_other_code_or_recipe(tmp_path):
    rec = {"recipe": "clustered", "n": 2 ** 19, "entries": 30000000, "digest": ps.kernel_source_digest(),
           "kernels": {"k_vjp_fused<4,1,0,0>": {"bytes_per_launch": 8.0e8}}}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(rec))
    name = "k_vjp_fused<4, true, false, false>"          # the bench's spelling
    assert ps.traffic_for(name, 30000000, path=str(p)) == pytest.approx(8.0e8)
    assert ps.traffic_for(name, 190000000, path=str(p)) == pytest.approx(8.0e8 * 19 / 3)
    assert ps.traffic_for(name, 190000000, recipe="uniform", path=str(p)) is None
    assert ps.traffic_for("k_pair_packed<2, 8, false, false>", 190000000, path=str(p)) is None
    rec["digest"] = "0" * 64
    p.write_text(json.dumps(rec))
    assert ps.traffic_for(name, 190000000, path=str(p)) is None
    assert ps.traffic_for(name, 190000000, path=str(tmp_path / "missing.json")) is None
    p.write_text("{not json")
    assert ps.traffic_for(name, 190000000, path=str(p)) is None


def test_committed_record_names_the_bench_kernels():
    """The committed record covers the three pair-kernel launches the bench
    reports, each with a traffic per entry at least the 16-byte record it must
    stream and below 100 bytes."""
    rec = json.load(open(ps.TRAFFIC_JSON))
    assert rec["recipe"] == "clustered" and rec["entries"] > 0
    assert set(rec["kernels"]) == {"k_pair_packed<2,8,0,0>", "k_vjp_fused<4,0,0,0>", "k_vjp_epack<4,1,0,0>"}
    for k in rec["kernels"].values():
        assert 16 <= k["bytes_per_launch"] / rec["entries"] < 100
