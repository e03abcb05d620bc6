"""Short markdown summaries of Nsight Compute output for profiles/.

Two inputs, both exported with ncu on or off the GPU machine:

* a raw-page CSV of a capture (``ncu -i rep.ncu-rep --page raw --csv``):
  one table per launch with the figures the roofline and the tuning notes
  use, and per kernel the lines ``dram_bytes_per_launch: <key> <bytes>``,
  ``busiest_pipe_name: <key> <pipe>`` and ``busiest_pipe_pct: <key> <pct>``
  that bench.py reads;
* a launch list (``ncu --metrics gpu__time_duration.sum --csv``): launches,
  total time and share per kernel.

Every summary starts with ``source_digest: <hex>``, the digest of the
library sources that were profiled (paper_1810_00615_gb300._build._digest()
on the machine that ran ncu); bench.py uses a summary's figures only while
that digest is still the current one.

    python -m paper_1810_00615_gb300.ncu_summary capture raw.csv out.md \\
        --title "..." --command "..." --digest HEX --key 'k_matvec_fx<2, 0, 1, double, 0, 1>=matvec_dots1_double'
    python -m paper_1810_00615_gb300.ncu_summary launches launches.csv out.md \\
        --title "..." --command "..." --digest HEX
"""
from __future__ import annotations

import argparse
import collections
import csv
import re
import sys

ROWS = [  # (label, metric, scale, unit)
    ("duration", "gpu__time_duration.sum", 1.0, "us"),
    ("DRAM read", "dram__bytes_read.sum", 1.0, None),
    ("DRAM write", "dram__bytes_write.sum", 1.0, None),
    ("DRAM throughput % of peak", "dram__throughput.avg.pct_of_peak_sustained_elapsed", 1.0, "%"),
    ("SM throughput % of peak", "sm__throughput.avg.pct_of_peak_sustained_elapsed", 1.0, "%"),
    ("issue slots busy %", "smsp__issue_active.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("ALU pipe %", "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("FMA pipe %", "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("FP64 pipe %", "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("LSU pipe %", "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("warp instructions", "smsp__inst_executed.sum", 1.0, None),
    ("warps active % (achieved occupancy)", "sm__warps_active.avg.pct_of_peak_sustained_active", 1.0, "%"),
    ("registers / thread", "launch__registers_per_thread", 1.0, None),
    ("shared memory / block (dynamic)", "launch__shared_mem_per_block_dynamic", 1.0, None),
    ("block size", "launch__block_size", 1.0, None),
    ("grid size", "launch__grid_size", 1.0, None),
    ("L2 hit rate %", "lts__t_sector_hit_rate.pct", 1.0, "%"),
    ("stall: long scoreboard (per issue)",
     "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio", 1.0, None),
    ("stall: barrier (per issue)",
     "smsp__average_warps_issue_stalled_barrier_per_issue_active.ratio", 1.0, None),
    ("stall: short scoreboard (per issue)",
     "smsp__average_warps_issue_stalled_short_scoreboard_per_issue_active.ratio", 1.0, None),
    ("stall: MIO throttle (per issue)",
     "smsp__average_warps_issue_stalled_mio_throttle_per_issue_active.ratio", 1.0, None),
    ("stall: math pipe throttle (per issue)",
     "smsp__average_warps_issue_stalled_math_pipe_throttle_per_issue_active.ratio", 1.0, None),
    ("stall: wait (per issue)", "smsp__average_warps_issue_stalled_wait_per_issue_active.ratio",
     1.0, None),
    ("stall: not selected (per issue)",
     "smsp__average_warps_issue_stalled_not_selected_per_issue_active.ratio", 1.0, None),
]
PIPES = {  # busiest-pipe candidates: name -> metric
    "alu": "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
    "fma": "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "fp64": "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
    "lsu": "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
}
BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}


def _num(v: str):
    try:
        return float(v.replace(",", ""))
    except ValueError:
        return None


def read_raw(path):
    """Rows of a raw-page CSV: list of dicts {metric: (value, unit)}."""
    with open(path, newline="") as f:
        rows = list(csv.reader(f))
    hdr, units, data = rows[0], rows[1], rows[2:]
    out = []
    for d in data:
        if len(d) != len(hdr):
            continue
        out.append({h: (d[i], units[i]) for i, h in enumerate(hdr)})
    return out


def _bytes(rec, metric):
    if metric not in rec:
        return None
    v, u = rec[metric]
    x = _num(v)
    return None if x is None else x * BYTES.get(u, 1.0)


def _strip_params(name: str) -> str:
    """Drop a trailing parameter list '(...)' (balanced, so that template
    arguments such as '(int)-1' stay)."""
    n = name.rstrip()
    if not n.endswith(")"):
        return n
    depth = 0
    for i in range(len(n) - 1, -1, -1):
        depth += {")": 1, "(": -1}.get(n[i], 0)
        if depth == 0:
            return n[:i]
    return n


def short_name(name: str) -> str:
    """'void fft::<unnamed>::k_x<4096, 32>(...)' -> 'k_x<4096, 32>'."""
    n = _strip_params(name)
    n = re.sub(r"^void\s+", "", n).replace("<unnamed>::", "")
    base = n[:n.index("<")] if "<" in n else n
    return base.split("::")[-1] + n[len(base):]


def capture_md(raw, title, command, digest, keys):
    lines = [f"# {title}", "", f"source_digest: {digest}", "",
             "Command (GB300, from the repository root):", "", "```", command, "```", ""]
    seen = collections.Counter()
    for rec in raw:
        name = rec.get("Kernel Name", ("?", ""))[0]
        sn = short_name(name)
        seen[sn] += 1
        lines += [f"## `{sn}` (launch {seen[sn]})", "", "| metric | value |", "|---|---|"]
        for label, metric, _, _u in ROWS:
            if metric in rec and rec[metric][0] not in ("", "n/a"):
                v, u = rec[metric]
                lines.append(f"| {label} | {v} {u} |")
        lines.append("")
        key = None
        for pat, k in keys:
            if re.search(pat, sn) or pat == sn:
                key = k
                break
        rd, wr = _bytes(rec, "dram__bytes_read.sum"), _bytes(rec, "dram__bytes_write.sum")
        if key and rd is not None and wr is not None:
            lines.append(f"dram_bytes_per_launch: {key} {int(rd + wr)}")
        pipes = {p: _num(rec[m][0]) for p, m in PIPES.items() if m in rec and _num(rec[m][0]) is not None}
        if key and pipes:
            p = max(pipes, key=pipes.get)
            lines.append(f"busiest_pipe_name: {key} {p}")
            lines.append(f"busiest_pipe_pct: {key} {pipes[p]:.2f}")
        if key:
            lines.append("")
    return "\n".join(lines) + "\n"


def launches_md(path, title, command, digest):
    with open(path, newline="") as f:
        rows = [r for r in csv.reader(f) if len(r) > 5]
    hdr = rows[0]
    ik, iv, imet = hdr.index("Kernel Name"), hdr.index("Metric Value"), hdr.index("Metric Name")
    iu = hdr.index("Metric Unit") if "Metric Unit" in hdr else None
    agg = collections.OrderedDict()
    for r in rows[1:]:
        if r[imet] != "gpu__time_duration.sum":
            continue
        v = _num(r[iv])
        if v is None:
            continue
        unit = r[iu] if iu is not None else "ns"
        us = v / 1e3 if unit in ("nsecond", "ns") else (v if unit in ("usecond", "us") else v * 1e3)
        a = agg.setdefault(short_name(r[ik]), [0, 0.0])
        a[0] += 1
        a[1] += us
    total = sum(t for _, t in agg.values()) or 1.0
    lines = [f"# {title}", "", f"source_digest: {digest}", "",
             "Command (GB300, from the repository root; the plain run of the same command "
             "line exited 0 first):", "", "```", command, "```", "",
             "Per-launch times under ncu are cold-cache and serialised: compare shares, "
             "not absolutes.", "", "| kernel | launches | total us | mean us | share |",
             "|---|---|---|---|---|"]
    for k, (n, t) in sorted(agg.items(), key=lambda x: -x[1][1]):
        lines.append(f"| `{k}` | {n} | {t:.1f} | {t / n:.1f} | {100 * t / total:.1f}% |")
    lines += ["", f"Total kernel time {total:.1f} us over {sum(n for n, _ in agg.values())} launches.",
              ""]
    return "\n".join(lines) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("kind", choices=["capture", "launches"])
    ap.add_argument("csv")
    ap.add_argument("out")
    ap.add_argument("--title", required=True)
    ap.add_argument("--command", required=True)
    ap.add_argument("--digest", required=True)
    ap.add_argument("--key", action="append", default=[],
                    help="'<kernel name or regex>=<key>' for the bench's lookup lines")
    ap.add_argument("--note", default="")
    a = ap.parse_args(argv)
    if a.kind == "capture":
        keys = [tuple(k.rsplit("=", 1)) for k in a.key]
        text = capture_md(read_raw(a.csv), a.title, a.command, a.digest, keys)
    else:
        text = launches_md(a.csv, a.title, a.command, a.digest)
    if a.note:
        text += "\n" + a.note.strip() + "\n"
    with open(a.out, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
