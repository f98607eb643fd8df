"""Writes the stored expected values under tests/golden/ that come from the oracle.

Run from the repository root:  python tests/golden/make_golden.py
It calls only the FP64 CPU oracle (oracle/).  The inputs are chosen so that every
intermediate of the rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2, step 5) is a small
dyadic rational: U = H_4 / 2 (a Hadamard matrix scaled to orthonormal columns, entries
+-1/2) and integer operators O_k.  The stored O'_k are therefore exact in FP64, FP32,
TF32 and BF16 alike, and every precision path must reproduce them bit for bit.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402


def dyadic_case():
    # d = 2 site states, m = 2 block states, m' = m*d = 4 (no truncation)
    H4 = np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], dtype=np.float64)
    U = H4 / 2.0
    O = np.array([[[1, 2], [3, 4]], [[0, -5], [7, 2]], [[9, -1], [-1, -3]]], dtype=np.float64)
    return U, O, 2


def main():
    U, O, d = dyadic_case()
    Op = oracle.rotate_dense(U, O, d)
    path = os.path.join(HERE, "rotate_h4_m2_d2.txt")
    with open(path, "w") as f:
        f.write("# Rotation O'_k = U^T (O_k (x) I_d) U, Sec. 2 step 5 (block index slow, site index fast).\n")
        f.write("# Written by tests/golden/make_golden.py with the FP64 CPU oracle; all values exact.\n")
        f.write("# d m mp K\n%d %d %d %d\n" % (d, O.shape[1], U.shape[1], O.shape[0]))
        f.write("# U (m*d x mp), row-major\n")
        for row in U:
            f.write(" ".join(repr(float(x)) for x in row) + "\n")
        for k in range(O.shape[0]):
            f.write("# O_%d (m x m)\n" % k)
            for row in O[k]:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")
            f.write("# O'_%d (mp x mp)\n" % k)
            for row in Op[k]:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
