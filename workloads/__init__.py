"""Seeded synthetic inputs for the plane-wave Hamiltonian / Chebyshev-filter workloads.

This module is shared by the CUDA path's tests, the benchmark and the FP64 oracle.  It holds
no arithmetic of the method itself: it only draws cell parameters, atom sites, projector
energies, k-point lists, random wavefunction blocks and request arrival times from seeded
NumPy generators.  Everything that the Kohn-Sham method computes from these inputs (the
G-sphere, V_loc on the grid, projector tables, H, eigenpairs) lives separately on each side.

Units are Hartree atomic units (bohr, Ha).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

# Shifted 2x2x2 Monkhorst-Pack grid: the four time-reversal-irreducible points first, then
# their negatives.  Reduced coordinates.
SHIFTED_222 = np.array(
    [
        [0.25, 0.25, 0.25],
        [0.25, 0.25, -0.25],
        [0.25, -0.25, 0.25],
        [-0.25, 0.25, 0.25],
        [-0.25, -0.25, -0.25],
        [-0.25, -0.25, 0.25],
        [-0.25, 0.25, -0.25],
        [0.25, -0.25, -0.25],
    ],
    dtype=np.float64,
)


@dataclass
class System:
    """One Kohn-Sham system: cell, cutoff, k-points, atoms and the requested band count."""

    name: str
    lattice: np.ndarray  # (3,3) rows a1, a2, a3 in bohr
    ecut: float  # Ha
    kpts: np.ndarray  # (nk,3) reduced coordinates
    pos: np.ndarray  # (natom,3) Cartesian, bohr
    D: np.ndarray  # (natom*nproj_per_atom,) Ha, diagonal projector energies
    nband: int
    fft_box: Optional[Tuple[int, int, int]] = None  # None: default size rule
    vloc_amp: float = -2.0  # Ha
    vloc_sigma: float = 1.0  # bohr
    nproj_per_atom: int = 4  # 4 = s, px, py, pz ; 1 = s only ; 0 = none
    proj_alpha: float = 0.25  # form factor exp(-alpha |q|^2)
    seed: int = 0
    Q: Optional[np.ndarray] = None  # (nproj,) overlap coefficients q_i; None: S = 1

    @property
    def natom(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nproj(self) -> int:
        return self.natom * self.nproj_per_atom


def cubic(a: float) -> np.ndarray:
    return np.diag([float(a), float(a), float(a)])


def _uniform_sites(rng: np.random.Generator, lattice: np.ndarray, natom: int,
                   min_sep: float = 0.0, max_tries: int = 100000) -> np.ndarray:
    """Uniform sites in the cell (reduced draws mapped to Cartesian), optional rejection on a
    minimum Cartesian separation measured between the raw draws (no periodic images)."""
    pos: List[np.ndarray] = []
    tries = 0
    while len(pos) < natom:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("site rejection did not finish")
        r = rng.random(3) @ lattice
        if min_sep > 0 and any(np.linalg.norm(r - p) < min_sep for p in pos):
            continue
        pos.append(r)
    return np.array(pos, dtype=np.float64).reshape(natom, 3)


def make_system(name: str, a: float, ecut: float, natom: int, nband: int, seed: int,
                kpts=None, fft_box=None, min_sep: float = 0.0, nproj_per_atom: int = 4,
                vloc_amp: float = -2.0, vloc_sigma: float = 1.0,
                proj_alpha: float = 0.25) -> System:
    rng = np.random.default_rng(seed)
    lat = cubic(a)
    pos = _uniform_sites(rng, lat, natom, min_sep)
    D = rng.uniform(-1.0, 1.0, size=natom * nproj_per_atom)
    if kpts is None:
        kpts = np.zeros((1, 3))
    return System(name=name, lattice=lat, ecut=float(ecut), kpts=np.asarray(kpts, np.float64),
                  pos=pos, D=D, nband=int(nband), fft_box=fft_box, vloc_amp=vloc_amp,
                  vloc_sigma=vloc_sigma, nproj_per_atom=nproj_per_atom,
                  proj_alpha=proj_alpha, seed=seed)


def config1() -> System:
    """Gamma, a=10 bohr, Ecut=10 Ha, box 24^3, 4 atoms x (s,p), 16 bands, complex128."""
    return make_system("C1", 10.0, 10.0, 4, 16, seed=1001, fft_box=(24, 24, 24))


def config2() -> System:
    """a=20 bohr, Ecut=20 Ha, box 96^3, 64 atoms (min sep 2 bohr), 512 bands, 4 shifted k."""
    return make_system("C2", 20.0, 20.0, 64, 512, seed=1002, kpts=SHIFTED_222[:4],
                       fft_box=(96, 96, 96), min_sep=2.0)


def config3() -> System:
    """The config-1 cell with 1024 bands (mixed-precision form)."""
    s = make_system("C3", 10.0, 10.0, 4, 1024, seed=1001, fft_box=(24, 24, 24))
    return s


def config4(nsys: int = 48) -> List[System]:
    """Uneven batch: a~U[8,16], Ecut~U[12,20], natom~U{8..64}, bands=2*natom, nk~U{1..8}."""
    out = []
    for j in range(nsys):
        rng = np.random.default_rng(4000 + j)
        a = float(rng.uniform(8.0, 16.0))
        ecut = float(rng.uniform(12.0, 20.0))
        natom = int(rng.integers(8, 65))
        nk = int(rng.integers(1, 9))
        out.append(make_system(f"C4.{j}", a, ecut, natom, 2 * natom, seed=4000 + 100000 + j,
                               kpts=SHIFTED_222[:nk]))
    return out


@dataclass
class Request:
    t_arrival: float  # seconds from start
    system: System
    repeat_of: Optional[int] = None  # index of an earlier request with the same cell


def config5(nreq: int = 200, rate: float = 200.0) -> List[Request]:
    """Poisson arrivals; 90% config-4-distribution systems, 10% config-1-size systems;
    25% of requests repeat an earlier cell (warm start)."""
    rng = np.random.default_rng(1005)
    t = 0.0
    reqs: List[Request] = []
    for i in range(nreq):
        t += float(rng.exponential(1.0 / rate))
        if reqs and rng.random() < 0.25:
            j = int(rng.integers(0, len(reqs)))
            reqs.append(Request(t, reqs[j].system, repeat_of=j))
            continue
        if rng.random() < 0.1:
            s = make_system(f"C5.{i}", 10.0, 10.0, 4, 16, seed=5000 + i, fft_box=(24, 24, 24))
        else:
            sub = np.random.default_rng(5000 + i)
            a = float(sub.uniform(8.0, 16.0))
            ecut = float(sub.uniform(12.0, 20.0))
            natom = int(sub.integers(8, 65))
            nk = int(sub.integers(1, 9))
            s = make_system(f"C5.{i}", a, ecut, natom, 2 * natom, seed=5000 + 100000 + i,
                            kpts=SHIFTED_222[:nk])
        reqs.append(Request(t, s))
    return reqs


def with_overlap(s: System, qmax: float = 0.5, qmin: float = 0.0, seed: Optional[int] = None) -> System:
    """The same system with overlap coefficients q_i ~ U[qmin, qmax] (one per projector), drawn
    from their own generator (seed + 7777 unless given) so that the other inputs are unchanged."""
    rng = np.random.default_rng((s.seed + 7777) if seed is None else seed)
    return replace(s, Q=rng.uniform(qmin, qmax, size=s.nproj))


def config1s() -> System:
    """Config 1 with a nonlocal overlap S = 1 + sum_i |beta_i> q_i <beta_i|, q_i ~ U[0, 0.5]."""
    return with_overlap(replace(config1(), name="C1S"))


def config2s(nk: int = 1) -> System:
    """The config-2 cell (96^3, 64 atoms, 256 projectors, 512 bands) with the overlap of
    config1s, on the first nk shifted k-points."""
    s = config2()
    return with_overlap(replace(s, name="C2S", kpts=s.kpts[:nk]))


def tiny_system(a: float = 6.0, ecut: float = 2.0, natom: int = 2, nband: int = 8,
                seed: int = 7, kpts=None, fft_box=None, nproj_per_atom: int = 4,
                vloc_amp: float = -2.0) -> System:
    """Small cells for exhaustive checks (N_pw of a few dozen to a few hundred)."""
    return make_system("tiny", a, ecut, natom, nband, seed=seed, kpts=kpts, fft_box=fft_box,
                       nproj_per_atom=nproj_per_atom, vloc_amp=vloc_amp)


def random_block(npw: int, nb: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex Gaussian block, band-major: shape (nb, npw) (one row per band)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))
    return x.astype(dtype)


def with_(s: System, **kw) -> System:
    return replace(s, **kw)
