"""Writes the golden fixtures ``topk_*.txt`` and ``join_*.txt`` in this folder.

Every stored value comes from the CPU oracle (``oracle/``) run on seeded
inputs from ``paper_2601_19911_gb300.datagen``; nothing here calls the CUDA
library.  Run from the repository root:

    python -m tests.golden.make_golden
"""
import os

import numpy as np

import oracle
from paper_2601_19911_gb300 import datagen

HERE = os.path.dirname(os.path.abspath(__file__))

# The first case is the single-query workload: 2^20 int64 keys uniform over the
# full range (seed 0), K = 100, descending, row-ids 0..N-1.
TOPK_CASES = [
    dict(name="topk_i64_uniform_n1048576_k100_desc", n=1 << 20, dist="uniform", kt="i64",
         seed=0, k=100, order=oracle.DESC),
    dict(name="topk_f32_uniform_n65536_k50_asc", n=1 << 16, dist="uniform", kt="f32",
         seed=1, k=50, order=oracle.ASC),
    dict(name="topk_i64_dup1024_n65536_k300_desc", n=1 << 16, dist="dup1024", kt="i64",
         seed=1, k=300, order=oracle.DESC),
    dict(name="topk_f32_ascending_n65536_k64_desc", n=1 << 16, dist="ascending", kt="f32",
         seed=1, k=64, order=oracle.DESC),
]

JOIN_CASES = [
    dict(name="join_mult14_b200_p500_zipf_h50", nb=200, mult="mult14", np=500, hit=0.5,
         dist="zipf", seed=7),
    dict(name="join_unique_b300_p400_uniform_h90", nb=300, mult="unique", np=400, hit=0.9,
         dist="uniform", seed=8),
]


def topk_input(case):
    return datagen.topk_keys(case["n"], case["dist"], case["kt"], seed=case["seed"])


def join_input(case):
    b = datagen.join_build(case["nb"], case["mult"], seed=case["seed"])
    p = datagen.join_probe(case["np"], b, case["hit"], case["dist"], seed=case["seed"])
    return b, p


def read_topk(name):
    rowids, bits = [], []
    with open(os.path.join(HERE, name + ".txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            r, b = line.split()
            rowids.append(int(r))
            bits.append(int(b, 16))
    return {"rowids": rowids, "key_bits": bits}


def read_join(name):
    with open(os.path.join(HERE, name + ".txt")) as f:
        return [int(line.split()[0]) << 32 | int(line.split()[1])
                for line in f if not line.startswith("#")]


def main():
    for c in TOPK_CASES:
        keys = topk_input(c)
        ok, orow = oracle.topk(keys, c["k"], c["order"])
        bits = ok.view(np.uint64 if ok.dtype == np.int64 else np.uint32)
        with open(os.path.join(HERE, c["name"] + ".txt"), "w") as f:
            f.write(f"# oracle Top-K: {c}\n# rowid key_bits\n")
            for r, b in zip(orow.tolist(), bits.tolist()):
                f.write(f"{r} {b:#x}\n")
    for c in JOIN_CASES:
        b, p = join_input(c)
        pairs = oracle.join(b.keys, p.keys, b.rowids, p.rowids)
        with open(os.path.join(HERE, c["name"] + ".txt"), "w") as f:
            f.write(f"# oracle join pairs: {c}\n# probe_rowid build_rowid\n")
            for v in pairs.tolist():
                f.write(f"{v >> 32} {v & 0xFFFFFFFF}\n")


if __name__ == "__main__":
    main()
