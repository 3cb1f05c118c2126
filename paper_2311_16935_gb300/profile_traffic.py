"""DRAM traffic per launch of the solve's kernels, from an ncu capture, as a
machine-written JSON file that bench.py reads for its roofline entry.

    python -m paper_2311_16935_gb300.profile_traffic CSV CELLS OUT.json --command "..."

CSV is either ncu's raw page (``ncu -i rep.ncu-rep --page raw --csv``: one
row per launch, one column per metric, a units row under the header) or the
``--csv`` log of a ``--metrics`` capture (one row per launch and metric).
CELLS is the number of grid cells one launch of each kernel covers in the
captured run.  The file records, per kernel (name up to its template
arguments), the launches, the median DRAM bytes (read + write) per launch of
the launches that did work, and per cell,
and the hash of the kernel sources it was taken on: bench.py reports the
traffic only while the sources still hash the same.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
from collections import defaultdict

HERE = os.path.dirname(os.path.abspath(__file__))
KERNEL_SOURCES = ("solve.cu", "mg.cu", "mg.cuh", "cg_state.cuh", "stencil.cuh", "internal.cuh", "ff.cuh", "fpconv.cuh")
METRICS = ("dram__bytes_read.sum", "dram__bytes_write.sum")


def kernel_source_hash() -> str:
    """Hash of the sources that define the timed solve's kernels."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(HERE, "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def short_name(kernel: str) -> str:
    """`void osm::(anonymous namespace)::k_cg_a<float, 3, 0>(...)` -> `k_cg_a<float, 3, 0>`."""
    m = re.search(r"(k_\w+(?:<[^()]*>)?)", kernel)
    return m.group(1) if m else kernel.strip()


_SCALE = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "b": 1.0, "kb": 1e3, "mb": 1e6, "gb": 1e9}


def _value(v: str, unit: str) -> float:
    return float(v.replace(",", "")) * _SCALE.get(unit.strip().lower(), 1.0)


def read_launches(path: str):
    """[(kernel name, dram bytes)] per launch, in capture order."""
    rows = list(csv.reader(open(path, newline="")))
    head = next((i for i, r in enumerate(rows) if "Kernel Name" in r), None)
    if head is None:
        raise ValueError(f"{path}: no ncu CSV header")
    hdr = rows[head]
    body = rows[head + 1:]
    kn = hdr.index("Kernel Name")
    if "Metric Name" in hdr:  # --metrics log: one row per (launch, metric)
        idc, mn, mu, mv = hdr.index("ID"), hdr.index("Metric Name"), hdr.index("Metric Unit"), hdr.index("Metric Value")
        per = defaultdict(dict)
        names = {}
        for r in body:
            if len(r) <= mv or r[mn] not in METRICS:
                continue
            per[r[idc]][r[mn]] = _value(r[mv], r[mu])
            names[r[idc]] = r[kn]
        return [(names[i], sum(per[i].values())) for i in per if len(per[i]) == len(METRICS)]
    # raw page: a units row follows the header
    units = body[0] if body and not body[0][0].strip().isdigit() else None
    data = body[1:] if units else body
    cols = [hdr.index(m) for m in METRICS]
    out = []
    for r in data:
        if len(r) <= max(cols):
            continue
        out.append((r[kn], sum(_value(r[c], units[c] if units else "byte") for c in cols)))
    return out


def summarise(path: str, cells: int, command: str) -> dict:
    """Per kernel: the median DRAM bytes of the launches that did work.  A
    solve's captured CUDA graphs launch a few iterations past convergence,
    whose kernels return at once; launches below half of the kernel's
    largest are counted as idle and left out of the median."""
    agg = defaultdict(list)
    for name, b in read_launches(path):
        agg[short_name(name)].append(b)
    kernels = {}
    for k, vals in sorted(agg.items()):
        top = max(vals)
        work = sorted(v for v in vals if v >= 0.5 * top)
        n = len(work)
        med = work[n // 2] if n % 2 else 0.5 * (work[n // 2 - 1] + work[n // 2])
        kernels[k] = {"launches": len(vals), "idle_launches": len(vals) - n, "dram_bytes_per_launch": med,
                      "dram_bytes_per_cell": med / cells}
    return {"kernel_source_hash": kernel_source_hash(), "cells_per_launch": cells, "command": command,
            "metrics": list(METRICS), "kernels": kernels}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("cells", type=int)
    ap.add_argument("out")
    ap.add_argument("--command", default="")
    a = ap.parse_args()
    d = summarise(a.csv, a.cells, a.command)
    with open(a.out, "w") as fh:
        json.dump(d, fh, indent=1)
        fh.write("\n")
    print(json.dumps(d, indent=1))


if __name__ == "__main__":
    main()
