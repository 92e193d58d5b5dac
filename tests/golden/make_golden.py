"""Writes the stored expected values under tests/golden/ from the CPU oracle.

Calls only ``oracle`` (and the seeded input generator); nothing here comes from
the CUDA library.  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1205_2926_gb300.inputs import P_NTT30, uniform_residues  # noqa: E402


def write_single_forward(path, p, L, seed):
    o = oracle.get()
    w = o.root_of_unity(p, L)
    a = uniform_residues(seed, L, p)
    out = o.ntt_ref(p, w, a)
    with open(path, "w") as f:
        f.write("# Forward NTT (Section 1 definition, Algorithm 1 bit-reversed output order)\n")
        f.write("# written by tests/golden/make_golden.py from the CPU oracle\n")
        f.write(f"p {p}\nL {L}\nomega {w}\nseed {seed}\n")
        f.write("input " + " ".join(str(int(v)) for v in a) + "\n")
        f.write("output " + " ".join(str(int(v)) for v in out) + "\n")


if __name__ == "__main__":
    write_single_forward(os.path.join(HERE, "forward_p998244353_L1024_seed1.txt"), P_NTT30, 1024, 1)
