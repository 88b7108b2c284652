"""Records per-unit counters of one kernel from an ncu report into
profiles/ncu_traffic.json, which bench.py reads for the `traffic` field of its
rooflines.

  python -m paper_1810_11765_gb300.ncu_record REPORT.ncu-rep --match REGEX \\
      --name KEY --units U1,U2,... [--counter dram|dram_step|l2_atomic|atom_inst|inst] [--scale S]

REPORT is read with `ncu -i REPORT --page raw --csv`; the launches whose kernel
name matches REGEX are taken in order and launch i is divided by Ui (objects
that launch processed).  `dram` records dram__bytes_read.sum +
dram__bytes_write.sum per unit (key dram_bytes_per_unit), from a capture that
flushes the caches before each launch; `dram_step` records the same counters
from a capture without cache control of a run that flushes L2 only between steps
(key dram_bytes_in_step_per_unit: the traffic a kernel causes inside a timed
step, where earlier kernels of the step have already brought shared lines in); `l2_atomic` records
lts__t_requests_op_atom.sum + lts__t_requests_op_red.sum per unit (key
l2_atomic_requests_per_unit); `atom_inst` records
smsp__sass_inst_executed_op_global_atom.sum per unit (key
atomic_instructions_per_unit: warp-level atomic instructions, which for the
allocator's single-lane bitmap atomics equal the atomic operations; --scale 32
turns a full warp's instruction into its 32 operations); `inst` records
smsp__inst_executed.sum per unit (key warp_instructions_per_unit), the issue-slot
work of an issue-bound kernel.  The mean over
launches is stored under KEY together with the library's build fingerprint;
bench.py ignores the record once the fingerprint no longer matches the sources.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import re
import subprocess

from . import build

ROOT = build.ROOT
OUT = os.path.join(ROOT, "profiles", "ncu_traffic.json")

COUNTERS = {
    "dram": ("dram_bytes_per_unit", ("dram__bytes_read.sum", "dram__bytes_write.sum")),
    "dram_step": ("dram_bytes_in_step_per_unit", ("dram__bytes_read.sum", "dram__bytes_write.sum")),
    "l2_atomic": ("l2_atomic_requests_per_unit", ("lts__t_requests_op_atom.sum", "lts__t_requests_op_red.sum")),
    "atom_inst": ("atomic_instructions_per_unit", ("smsp__sass_inst_executed_op_global_atom.sum",)),
    "inst": ("warp_instructions_per_unit", ("smsp__inst_executed.sum",)),
}
SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "request": 1.0, "": 1.0,
         "Krequest": 1e3, "Mrequest": 1e6, "inst": 1.0, "Kinst": 1e3, "Minst": 1e6, "Ginst": 1e9}


def read_rows(report: str):
    out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units = rows[0], rows[1]
    return hdr, units, rows[2:]


def per_launch(report: str, match: str, names):
    hdr, units, rows = read_rows(report)
    ki = hdr.index("Kernel Name")
    idx = [hdr.index(n) for n in names]
    vals = []
    for r in rows:
        if not re.search(match, r[ki]):
            continue
        v = 0.0
        for i in idx:
            v += float(r[i].replace(",", "")) * SCALE.get(units[i], 1.0)
        vals.append(v)
    return vals


def main():
    p = argparse.ArgumentParser()
    p.add_argument("report")
    p.add_argument("--match", required=True)
    p.add_argument("--name", required=True)
    p.add_argument("--units", required=True, help="objects per matched launch, comma-separated")
    p.add_argument("--counter", default="dram", choices=sorted(COUNTERS))
    p.add_argument("--scale", type=float, default=1.0,
                   help="multiply the counters by this (e.g. warp instructions -> thread ops)")
    a = p.parse_args()
    key, names = COUNTERS[a.counter]
    vals = per_launch(a.report, a.match, names)
    units = [float(u) for u in a.units.split(",")]
    if len(vals) != len(units):
        raise SystemExit(f"{len(vals)} matching launches but {len(units)} unit counts")
    vals = [v * a.scale for v in vals]
    per_unit = [v / u for v, u in zip(vals, units)]
    rec = {"fingerprint": build.fingerprint(), "kernels": {}}
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
        if old.get("fingerprint") == rec["fingerprint"]:
            rec = old
    entry = rec["kernels"].setdefault(a.name, {})
    entry[key] = sum(per_unit) / len(per_unit)
    entry[key.replace("_per_unit", "_per_launch")] = vals
    entry["units_per_launch"] = units
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps({a.name: entry}))


if __name__ == "__main__":
    main()
