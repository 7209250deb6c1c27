"""Summaries of ncu launch lists of liblor as the markdown kept under profiles/.

Input: a CSV written by
    ncu --metrics gpu__time_duration.sum[,dram__bytes_read.sum,dram__bytes_write.sum]
        --clock-control none --csv --log-file FILE <command>
Output: per-kernel launches, device time and share, and (when the DRAM
counters are present) DRAM bytes per kernel kind, the kinds being those of
the library's kernel timing (lor_profile_kind_name) so that bench.py can put
the traffic of its dominant kind beside the live roofline.

    python -m paper_1404_3448_gb300.ncu_summary FILE.csv [--skip N] [--take M]
"""
from __future__ import annotations

import argparse
import collections
import csv
import hashlib
import os
import re

# kernel name prefix -> timing kind (the scope each launch is timed under)
KINDS = [
    ("k_encode", "encode"), ("k_mq_encode", "encode"), ("k_mq_rindex", "overlap_scan"),
    ("k_mq_best", "overlap_scan"), ("k_mq_result", "overlap_collect"), ("k_topk_hist", "overlap_scan"),
    ("k_topk_", "overlap_collect"),
    ("k_sample_keys", "sample_keys"), ("k_dense_mark", "sample_keys"), ("k_par_samples", "sample_keys"),
    ("k_par_dups", "sample_keys"), ("k_first_char", "sample_keys"), ("k_dbl_keys", "sample_keys"),
    ("k_radix_hist", "radix_hist"), ("k_radix_offsets", "radix_hist"),
    ("k_onesweep", "radix_pass"), ("k_partition", "radix_pass"), ("k_iota_u32", "radix_pass"),
    ("k_name", "naming"), ("k_par_name", "naming"), ("k_dense_scan", "naming"), ("k_dense_write", "naming"),
    ("k_dbl_", "naming"),
    ("k_rank_scatter", "rank_scatter"), ("k_scatter_pairs<1>", "isa_scatter"), ("k_scatter_pairs", "rank_scatter"),
    ("k_dense_sorted", "rank_scatter"),
    ("k_nonsample", "nonsample"), ("k_first_sym_hist", "nonsample"), ("k_scatter_u64", "nonsample"),
    ("k_ns_", "nonsample"), ("k_par_nonsamples", "nonsample"),
    ("k_par_ns_", "nonsample"), ("k_perm_offsets", "radix_hist"),
    ("k_gather_pri", "nonsample"), ("k_par_dup_writeback", "nonsample"),
    ("k_group_records", "merge"), ("k_merge", "merge"),
    ("k_isa_phi", "isa_scatter"), ("k_scatter_isa_phi", "isa_scatter"), ("k_isa_direct", "isa_scatter"),
    ("k_text_max", "kasai"), ("k_pack_text", "kasai"), ("k_sort_exc", "kasai"), ("k_plcp", "kasai"),
    ("k_lcp_", "kasai"),
    ("k_ov_argmax", "overlap_scan"), ("k_ov_", "overlap_collect"), ("k_copy_u32", "overlap_collect"),
    ("k_sa64_keys0", "sample_keys"), ("k_sa64_round_keys", "sample_keys"), ("k_sa64_names", "naming"),
    ("k_sa64_settle", "rank_scatter"), ("k_narrow_sa64", "isa_scatter"),
    ("k_rmq_query", "rmq_query"), ("k_rmqb_query", "rmq_query"), ("k_rmq_", "rmq_level"),
    ("k_rmqb_", "rmq_level"),
    ("k_pk_count", "sample_keys"), ("k_pk_offsets", "radix_hist"), ("k_pk_partition", "radix_pass"),
    ("k_pk_fixup", "naming"), ("k_pk_name", "naming"),
]


def kind_of(kernel: str) -> str:
    if "SampleKeySrc" in kernel:  # the partition of the level-0 merge keys (Step 2/3)
        return "nonsample"
    for prefix, kind in KINDS:
        if kernel.startswith(prefix):
            return kind
    return "other"


def short_name(name: str) -> str:
    name = re.sub(r"\(.*", "", name.replace("(anonymous namespace)::", ""))
    name = name.replace("<unnamed>::", "").replace("unnamed>::", "").replace("lor::", "").strip()
    return name[5:] if name.startswith("void ") else name


def source_hash(root: str) -> str:
    """Hash of the kernel sources (the same digest bench.py computes)."""
    h = hashlib.sha256()
    csrc = os.path.join(root, "paper_1404_3448_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def read_launches(path: str):
    """[(kernel, {metric: value})] in launch order."""
    with open(path) as fh:
        rows = list(csv.DictReader(line for line in fh if not line.startswith("==")))
    launches = collections.OrderedDict()
    for r in rows:
        key = r["ID"]
        if key not in launches:
            launches[key] = (short_name(r["Kernel Name"]), {})
        val = float(str(r["Metric Value"]).replace(",", ""))
        unit = r.get("Metric Unit", "")
        scale = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
                 "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1.0)
        launches[key][1][r["Metric Name"]] = val * scale
    return list(launches.values())


def summarize(launches):
    per_kernel = collections.OrderedDict()
    per_kind = collections.OrderedDict()
    for name, m in launches:
        t = m.get("gpu__time_duration.sum", 0.0)
        rd = m.get("dram__bytes_read.sum")
        wr = m.get("dram__bytes_write.sum")
        k = per_kernel.setdefault(name, [0, 0.0])
        k[0] += 1
        k[1] += t
        d = per_kind.setdefault(kind_of(name), [0, 0.0, 0.0, 0.0, rd is not None])
        d[0] += 1
        d[1] += t
        d[2] += rd or 0.0
        d[3] += wr or 0.0
    return per_kernel, per_kind


def markdown(per_kernel, per_kind, model=None) -> str:
    """Tables of the launch list; with `model` (algorithmic bytes per kind for
    the same launches, as bench.py's stage_model_bytes) the kind table also
    gives the model bytes and DRAM bytes / model bytes."""
    total = sum(v[1] for v in per_kernel.values()) or 1.0
    out = ["| kernel | launches | total ms | share |", "|---|---|---|---|"]
    for name, (c, t) in sorted(per_kernel.items(), key=lambda x: -x[1][1]):
        out.append(f"| `{name}` | {c} | {t:.3f} | {100 * t / total:.1f} % |")
    if any(v[4] for v in per_kind.values()):
        head = "| kind | launches | total ms | DRAM read GB | DRAM write GB | DRAM bytes per launch |"
        rule = "|---|---|---|---|---|---|"
        if model is not None:
            head += " model GB | DRAM / model |"
            rule += "---|---|"
        out += ["", head, rule]
        for kind, (c, t, rd, wr, _) in sorted(per_kind.items(), key=lambda x: -x[1][1]):
            row = f"| {kind} | {c} | {t:.3f} | {rd / 1e9:.3f} | {wr / 1e9:.3f} | {(rd + wr) / max(c, 1):.0f} |"
            if model is not None:
                mb = model.get(kind)
                row += f" {mb / 1e9:.3f} | {(rd + wr) / mb:.3f} |" if mb else " - | - |"
            out.append(row)
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--skip", type=int, default=0, help="launches to drop from the start")
    ap.add_argument("--take", type=int, default=0, help="launches to keep after --skip (0: all)")
    ap.add_argument("--model-json", help="bench.py output of the same command (one timed step): adds the "
                                         "algorithmic bytes per kind and DRAM / model")
    args = ap.parse_args()
    launches = read_launches(args.csv)[args.skip:]
    if args.take:
        launches = launches[:args.take]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    print(f"source hash: `{source_hash(root)}`\n")
    model = None
    if args.model_json:
        import json
        with open(args.model_json) as fh:
            line = [ln for ln in fh if ln.startswith("{")][-1]
        model = json.loads(line).get("stage_model_bytes")
    print(markdown(*summarize(launches), model=model))


if __name__ == "__main__":
    main()
