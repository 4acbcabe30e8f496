"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

The paper prints no worked example for this path (no eigenvalues, counts or tolerances), so every
stored value here comes from the oracle: dense diagonalisation of the plane-wave Hamiltonian of the
seeded configurations.  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, values):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("".join(f"# {line}\n" for line in header))
        for v in values:
            v = int(v) if isinstance(v, (int, np.integer)) else float(v)
            f.write(f"{v!r}\n")


def main():
    s = W.config1()
    w, _ = O.build_problem(s, 0).lowest(16)
    write("c1_lowest16_Ha.txt",
          ["config 1 (a=10 bohr, Ecut=10 Ha, Gamma, box 24^3, 4 atoms seed 1001, 16 projectors):",
           "the 16 lowest eigenvalues (Ha) of the dense plane-wave Hamiltonian, oracle (LAPACK evr)",
           "written by tests/golden/make_golden.py"], list(w))
    s = W.config3()
    w, _ = O.build_problem(s, 0).lowest(1024)
    write("c3_lowest1024_Ha.txt",
          ["config 3 (the config-1 cell: a=10 bohr, Ecut=10 Ha, Gamma, box 24^3, 4 atoms seed 1001):",
           "the 1024 lowest eigenvalues (Ha) of the dense plane-wave Hamiltonian, oracle (LAPACK evr)",
           "written by tests/golden/make_golden.py"], list(w))
    s = W.config1s()
    w, _ = O.build_problem(s, 0).lowest(16)
    write("c1s_lowest16_Ha.txt",
          ["config 1 with the nonlocal overlap q ~ U[0, 0.5] (seed 1001 + 7777):",
           "the 16 lowest generalised eigenvalues H x = lambda S x (Ha), oracle (LAPACK gvx)",
           "written by tests/golden/make_golden.py"], list(w))
    c2 = W.config2()
    counts = [O.enumerate_sphere(c2.lattice, c2.ecut, k).shape[0] for k in c2.kpts]
    c1 = O.enumerate_sphere(W.config1().lattice, 10.0, (0, 0, 0)).shape[0]
    write("sphere_counts.txt",
          ["plane-wave counts 1/2|k+G|^2 <= Ecut by brute-force enumeration (oracle):",
           "config 1 (Gamma), then config 2 at its four shifted k-points",
           "written by tests/golden/make_golden.py"], [c1] + counts)


if __name__ == "__main__":
    main()
