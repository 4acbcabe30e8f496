"""Writes the lowest eigenvalues of the config-2 Hamiltonian at one k-point, from the FP64 oracle.

Config 2: cubic cell a = 20 bohr, Ecut = 20 Ha, box 96^3, 64 atoms (seed 1002, minimum separation
2 bohr), 256 s+p projectors, k = (1/4, 1/4, 1/4) (reduced), 34181 plane waves.  The oracle builds
the dense 34181 x 34181 Hamiltonian (18.7 GB) and asks LAPACK (zheevr through SciPy) for its
lowest eigenvalues.  That is the plain definition of what the Chebyshev-filtered solve converges
to; the paper prints no eigenvalues for this path, so the stored file is oracle output.

Slow: an hour on 8 x86 cores (the dense eigensolve took 3568 s there: the tridiagonal reduction
streams the 18.7 GB matrix from memory once per column).  Run from the repository root:

    python tests/golden/make_golden_c2.py [ik] [nvals]
"""
import os
import sys
import time

import numpy as np
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    ik = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    nvals = int(sys.argv[2]) if len(sys.argv) > 2 else 576
    s = W.config2()
    t0 = time.time()
    p = O.build_problem(s, ik)
    H = O.dense_hamiltonian_rowwise(p.basis, p.V, p.beta, p.D, order="F")
    t1 = time.time()
    print(f"built H {H.shape} in {t1 - t0:.0f} s", flush=True)
    w = scipy.linalg.eigh(H, eigvals_only=True, subset_by_index=[0, nvals - 1], driver="evr",
                          overwrite_a=True, check_finite=False)
    t2 = time.time()
    print(f"eigh in {t2 - t1:.0f} s", flush=True)
    k = s.kpts[ik]
    name = f"c2_k{ik}_lowest{nvals}_Ha.txt"
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# config 2 (a=20 bohr, Ecut=20 Ha, box 96^3, 64 atoms seed 1002 min sep 2 bohr,\n")
        f.write(f"# 256 s+p projectors) at reduced k = ({k[0]:g}, {k[1]:g}, {k[2]:g}), "
                f"npw = {p.basis.npw}:\n")
        f.write(f"# the {nvals} lowest eigenvalues (Ha) of the dense plane-wave Hamiltonian, "
                f"oracle (LAPACK evr)\n")
        f.write("# written by tests/golden/make_golden_c2.py\n")
        for v in w:
            f.write(f"{float(v)!r}\n")
    print("wrote", name, flush=True)


if __name__ == "__main__":
    main()
