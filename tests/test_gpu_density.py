"""Electron density n(r) = sum w |psi(r)|^2 (Eq. nandtau, §2) on the GPU through the C ABI,
against the oracle's naive-DFT density.

Bars: FP64 within 1e-12 of max n (element by element); mixed (complex64 transforms, FP64
accumulation) within 2e-6 of max n; accumulation over calls (k-points) exact up to the same bars;
the integral sum_j n_j Omega / N^3 equals sum w |c|^2 (Parseval).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_destroy(c)


def gpu_density(ctx, sysh, blocks, occs, prec, box):
    import torch
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    rho = torch.zeros(tuple(reversed(box)), dtype=torch.float64, device="cuda")
    for ik, (c, w) in enumerate(zip(blocks, occs)):
        psi = torch.from_numpy(c).to(cdt).cuda()
        K.kss_density_accumulate(sysh, ik, psi, w, rho, prec)
    torch.cuda.synchronize()
    return rho.cpu().numpy()


CASES = [
    ("C1", lambda: W.config1(), K.KSS_PREC_FP64, 1e-12, 20),
    ("C1_mixed", lambda: W.config1(), K.KSS_PREC_MIXED, 2e-6, 20),
    ("shifted_2k", lambda: W.make_system("d2", 7.0, 6.0, 3, 8, seed=51, kpts=W.SHIFTED_222[:2]), K.KSS_PREC_FP64, 1e-12, 9),
    ("C4_box", lambda: W.config4(1)[0], K.KSS_PREC_FP64, 1e-12, 7),
]


@pytest.mark.parametrize("name,mk,prec,tol,nb", CASES, ids=[c[0] for c in CASES])
def test_density_matches_oracle(ctx, name, mk, prec, tol, nb):
    s = mk()
    sysh = setup(ctx, s)
    try:
        box = O.system_box(s)
        _, vol = O.reciprocal_lattice(s.lattice)
        rng = np.random.default_rng(5)
        blocks, occs, ref = [], [], np.zeros(tuple(reversed(box)))
        for ik in range(len(s.kpts)):
            b = O.make_basis(s.lattice, s.ecut, s.kpts[ik], box)
            c = W.random_block(b.npw, nb, seed=60 + ik) / np.sqrt(b.npw)
            w = rng.uniform(0.0, 2.0, nb) / len(s.kpts)
            blocks.append(c)
            occs.append(w)
            ref += O.density(c, b, w, vol)
        rho = gpu_density(ctx, sysh, blocks, occs, prec, box)
        assert np.max(np.abs(rho - ref)) < tol * np.max(ref), np.max(np.abs(rho - ref)) / np.max(ref)
        integral = rho.sum() * vol / np.prod(box)
        expect = sum(float(w @ (np.abs(c) ** 2).sum(axis=1)) for c, w in zip(blocks, occs))
        assert abs(integral - expect) < (1e-11 if prec == K.KSS_PREC_FP64 else 1e-5) * expect
    finally:
        K.kss_sys_destroy(sysh)


def test_density_c2_sampled_bands(ctx):
    """The 96^3 box of config 2 (k-point 0), two bands against the oracle."""
    s = W.config2()
    sysh = setup(ctx, s)
    try:
        box = O.system_box(s)
        _, vol = O.reciprocal_lattice(s.lattice)
        b = O.make_basis(s.lattice, s.ecut, s.kpts[0], box)
        c = W.random_block(b.npw, 2, seed=70) / np.sqrt(b.npw)
        w = np.array([2.0, 0.5])
        rho = gpu_density(ctx, sysh, [c], [w], K.KSS_PREC_FP64, box)
        ref = O.density(c, b, w, vol)
        assert np.max(np.abs(rho - ref)) < 1e-12 * np.max(ref)
    finally:
        K.kss_sys_destroy(sysh)


def test_density_is_reproducible_and_rejects(ctx):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        b = O.make_basis(s.lattice, s.ecut, s.kpts[0], (24, 24, 24))
        c = W.random_block(b.npw, 11, seed=71)
        w = np.linspace(0.1, 2.0, 11)
        r1 = gpu_density(ctx, sysh, [c], [w], K.KSS_PREC_FP64, (24, 24, 24))
        r2 = gpu_density(ctx, sysh, [c], [w], K.KSS_PREC_FP64, (24, 24, 24))
        assert np.array_equal(r1, r2)  # fixed-order accumulation
        rho = torch.zeros((24, 24, 24), dtype=torch.float64, device="cuda")
        psi = torch.from_numpy(c).cuda()
        with pytest.raises(K.KssError):
            K.kss_density_accumulate(sysh, 0, psi, np.full(11, np.nan), rho)
        with pytest.raises(ValueError):
            K.kss_density_accumulate(sysh, 0, psi, np.ones(3), rho)
    finally:
        K.kss_sys_destroy(sysh)
    t = W.tiny_system(a=5.0, ecut=2.5, natom=2, fft_box=(16, 20, 18))
    th = setup(ctx, t)
    try:
        b = O.make_basis(t.lattice, t.ecut, t.kpts[0], (16, 20, 18))
        psi = torch.from_numpy(W.random_block(b.npw, 2, seed=1)).cuda()
        rho = torch.zeros((18, 20, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(K.KssError) as e:
            K.kss_density_accumulate(th, 0, psi, np.ones(2), rho)
        assert e.value.status == K.KSS_ENOTSUP
    finally:
        K.kss_sys_destroy(th)
