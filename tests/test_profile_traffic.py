"""The ncu-CSV reader that writes the committed traffic files (no GPU):
both CSV layouts ncu writes, unit scaling, per-kernel grouping."""
import json

from paper_2311_16935_gb300 import profile_traffic as pt

RAW = '''"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","dram__bytes_read.sum","dram__bytes_write.sum"
"","","","","","","","Mbyte","Kbyte"
"0","1","python","h","void osm::(anonymous namespace)::k_mg_fine_rb_fused<float, 16, 16, 0, false, false>(const T1 *, T1 *)","1","7","1,000.5","2000"
"1","1","python","h","void osm::(anonymous namespace)::k_mg_fine_rb_fused<float, 16, 16, 0, false, false>(const T1 *, T1 *)","1","7","999.5","0"
"2","1","python","h","void osm::k_cg_b<float>(float *, const float *)","1","7","12","0.5"
'''

LOG = '''==PROF== Connected to process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","k_residual<float, 3>(const double *)","1","7","(512, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","2.13"
"0","1","python","h","k_residual<float, 3>(const double *)","1","7","(512, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","500"
"0","1","python","h","k_residual<float, 3>(const double *)","1","7","(512, 1, 1)","(608, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","usecond","2800"
'''


def test_raw_page(tmp_path):
    f = tmp_path / "raw.csv"
    f.write_text(RAW)
    d = pt.summarise(str(f), 1000, "cmd")
    k = d["kernels"]["k_mg_fine_rb_fused<float, 16, 16, 0, false, false>"]
    assert k["launches"] == 2
    assert k["dram_bytes_per_launch"] == (1000.5e6 + 2e6 + 999.5e6) / 2
    assert k["dram_bytes_per_cell"] == k["dram_bytes_per_launch"] / 1000
    assert d["kernels"]["k_cg_b<float>"]["dram_bytes_per_launch"] == 12e6 + 500
    assert d["kernel_source_hash"] == pt.kernel_source_hash()
    json.dumps(d)


def test_metrics_log(tmp_path):
    f = tmp_path / "log.csv"
    f.write_text(LOG)
    d = pt.summarise(str(f), 10, "cmd")
    assert d["kernels"]["k_residual<float, 3>"] == {"launches": 1, "idle_launches": 0, "dram_bytes_per_launch": 2.63e9,
                                                    "dram_bytes_per_cell": 2.63e8}


def test_idle_launches_left_out(tmp_path):
    """Launches that returned at once (a captured graph's iterations past
    convergence) do not pull the median down."""
    rows = RAW.splitlines()[:2]
    for i, mb in enumerate(["1000", "1010", "990", "0.01", "0.02"]):
        rows.append(f'"{i}","1","python","h","void osm::k_cg_b<float>(float *)","1","7","{mb}","0"')
    f = tmp_path / "idle.csv"
    f.write_text("\n".join(rows) + "\n")
    k = pt.summarise(str(f), 100, "cmd")["kernels"]["k_cg_b<float>"]
    assert k["launches"] == 5 and k["idle_launches"] == 2
    assert k["dram_bytes_per_launch"] == 1000e6


def test_source_hash_covers_every_included_header():
    """The traffic file is trusted only while the kernel sources hash the
    same: every project header the hashed sources include (transitively)
    must be hashed too, or an edit to it would leave stale counters live."""
    import os
    import re

    csrc = os.path.join(os.path.dirname(pt.__file__), "csrc")
    seen, todo = set(), [n for n in pt.KERNEL_SOURCES if n.endswith(".cu")]
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        seen.add(name)
        with open(os.path.join(csrc, name)) as fh:
            for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), re.M):
                # the kernel headers beside the sources (the public C header,
                # declarations and documentation only, lives elsewhere)
                if "/" not in inc and os.path.exists(os.path.join(csrc, inc)):
                    todo.append(inc)
    missing = sorted(seen - set(pt.KERNEL_SOURCES))
    assert not missing, missing
