"""Host-only checks of the ncu launch-list summariser and of bench.py's
reading of the committed DRAM-traffic summary."""
import os

import bench
from paper_1404_3448_gb300 import ncu_summary as S

CSV = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","p","h","void k_onesweep<unsigned long, unsigned int, 0>(const unsigned long *)","1","7","(256, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","2.00"
"0","1","p","h","void k_onesweep<unsigned long, unsigned int, 0>(const unsigned long *)","1","7","(256, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Kbyte","500.00"
"0","1","p","h","void k_onesweep<unsigned long, unsigned int, 0>(const unsigned long *)","1","7","(256, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","3.00"
"1","1","p","h","unnamed>::k_merge<int>(unnamed>::MergeIn<int>, const long *, int *, int *)","1","7","(512, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","1000"
"1","1","p","h","unnamed>::k_merge<int>(unnamed>::MergeIn<int>, const long *, int *, int *)","1","7","(512, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","24"
"1","1","p","h","unnamed>::k_merge<int>(unnamed>::MergeIn<int>, const long *, int *, int *)","1","7","(512, 1, 1)","(10, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","1000"
'''


def test_summary_units_names_and_kinds(tmp_path):
    p = tmp_path / "l.csv"
    p.write_text(CSV)
    launches = S.read_launches(str(p))
    assert [n for n, _ in launches] == ["k_onesweep<unsigned long, unsigned int, 0>", "k_merge<int>"]
    per_kernel, per_kind = S.summarize(launches)
    assert abs(per_kernel["k_onesweep<unsigned long, unsigned int, 0>"][1] - 0.003) < 1e-12  # ms
    c, t, rd, wr, has = per_kind["radix_pass"]
    assert (c, rd, wr, has) == (1, 2e6, 5e5, True)
    assert per_kind["merge"][2:4] == [1000.0, 24.0]
    md = S.markdown(per_kernel, per_kind)
    assert "| radix_pass | 1 | 0.003 | 0.002 | 0.001 | 2500000 |" in md


def test_every_library_kernel_has_a_kind():
    src = os.path.join(os.path.dirname(S.__file__), "csrc")
    import re
    names = set()
    for f in os.listdir(src):
        names |= set(re.findall(r"__global__ void (?:__launch_bounds__\([^)]*\) )?(k_\w+)", open(os.path.join(src, f)).read()))
    plain = {n for n in names if not n.startswith(("k_pair_", "k_block_", "k_seg_", "k_group_f", "k_group_p",
                                                   "k_encode_group", "k_serve_"))}
    assert plain and all(S.kind_of(n) != "other" for n in plain), sorted(n for n in plain if S.kind_of(n) == "other")


def test_bench_reads_traffic_only_for_current_sources(tmp_path, monkeypatch):
    md = "source hash: `%s`\n\n| kind | launches | total ms | DRAM read GB | DRAM write GB | DRAM bytes per launch |\n|---|---|---|---|---|---|\n| radix_pass | 2 | 1.0 | 0.1 | 0.1 | 12345 |\n"
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    name = bench.TRAFFIC_PROFILES["large"][0]
    (tmp_path / "profiles" / name).write_text(md % "abc123")
    assert bench.ncu_traffic("radix_pass", "large") == 12345.0
    assert bench.ncu_traffic("merge", "large") is None
    assert bench.ncu_traffic("radix_pass", "tiny") is None
    # a kind the first summary lacks is read from the next one
    rmq = md.replace("radix_pass", "rmq_level").replace("12345", "777")
    (tmp_path / "profiles" / bench.TRAFFIC_PROFILES["large"][1]).write_text(rmq % "abc123")
    assert bench.ncu_traffic("rmq_level", "large") == 777.0
    (tmp_path / "profiles" / name).write_text(md % "ffff00")
    assert bench.ncu_traffic("radix_pass", "large") is None


def test_bench_scales_traffic_by_the_dram_to_model_ratio(tmp_path, monkeypatch):
    launches = [("k_onesweep<unsigned long, unsigned int, 0, 12>", {"gpu__time_duration.sum": 1.0,
                 "dram__bytes_read.sum": 3e9, "dram__bytes_write.sum": 1e9})]
    md = S.markdown(*S.summarize(launches), model={"radix_pass": 2e9})
    assert "| radix_pass | 1 | 1.000 | 3.000 | 1.000 | 4000000000 | 2.000 | 2.000 |" in md
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    (tmp_path / "profiles" / bench.TRAFFIC_PROFILES["large"][0]).write_text("source hash: `abc123`\n\n" + md)
    assert bench.ncu_traffic("radix_pass", "large", 5e8) == 1e9
