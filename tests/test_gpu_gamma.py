"""The Gamma-point path (real-space-real bands, two bands per complex FFT) on the GPU through the
C ABI: the same eigenvalues as the unpacked path and as the oracle, eigenvectors with
psi(-G) = conj psi(G).

Bars: FP64 eigenvalues within 1e-8 Ha of the oracle and 1e-10 Ha of the unpacked solve; mixed
within 1e-6 Ha of the oracle; symmetry of the returned vectors to 1e-12 (FP64).
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


def mirror_index(basis):
    at = {tuple(m): i for i, m in enumerate(basis.miller)}
    return np.array([at[tuple(-m)] for m in basis.miller])


@pytest.mark.parametrize("nband,nbuffer", [(16, -1), (15, 4)])  # even and odd block sizes
def test_gamma_fp64_matches_unpacked_and_oracle(ctx, nband, nbuffer):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        npw = p.basis.npw
        X = torch.zeros((nband, npw), dtype=torch.complex128, device="cuda")
        ev, rs, st, _ = K.kss_chebfi_solve(sysh, 0, nband, K.make_opts(tol=1e-9, seed=3, nbuffer=nbuffer), evecs=X)
        ev0 = K.kss_chebfi_solve(sysh, 0, nband, K.make_opts(tol=1e-9, seed=3, nbuffer=nbuffer,
                                                             flags=K.KSS_SOLVE_NO_GAMMA_REAL))[0]
        w, _ = p.lowest(nband)
        assert np.max(np.abs(ev - w)) < 1e-8
        assert np.max(np.abs(ev - ev0)) < 1e-10
        assert rs.max() <= 1e-9
        x = X.cpu().numpy()
        mir = mirror_index(p.basis)
        assert np.max(np.abs(x[:, mir] - x.conj())) < 1e-12
    finally:
        K.kss_sys_destroy(sysh)


def test_gamma_mixed(ctx):
    s = W.with_(W.config1(), nband=64)
    sysh = setup(ctx, s)
    try:
        ev = K.kss_chebfi_solve(sysh, 0, s.nband, K.make_opts(prec=K.KSS_PREC_MIXED, seed=8))[0]
        w, _ = O.build_problem(s, 0).lowest(s.nband)
        assert np.max(np.abs(ev - w)) < 1e-6, np.max(np.abs(ev - w))
    finally:
        K.kss_sys_destroy(sysh)


def test_gamma_other_box_and_warm_start(ctx):
    """A default-box Gamma cell (36^3 class) and a warm start from non-symmetric vectors."""
    import torch
    s = W.make_system("g2", 8.0, 9.0, 5, 20, seed=91)
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        npw = p.basis.npw
        w, _ = p.lowest(s.nband)
        ev, rs, st, _ = K.kss_chebfi_solve(sysh, 0, s.nband, K.make_opts(tol=1e-9, seed=1))
        assert np.max(np.abs(ev - w)) < 1e-8
        x0 = torch.from_numpy(W.random_block(npw, s.nband, seed=5)).cuda()  # no symmetry
        ev2 = K.kss_chebfi_solve(sysh, 0, s.nband, K.make_opts(tol=1e-9, x0=x0, x0_nb=s.nband, x0_ld=npw))[0]
        assert np.max(np.abs(ev2 - w)) < 1e-8
    finally:
        K.kss_sys_destroy(sysh)


def symmetric_block(basis, nb, seed):
    c = W.random_block(basis.npw, nb, seed=seed)
    mir = mirror_index(basis)
    c = 0.5 * (c + c[:, mir].conj())
    return c


GAMMA_APPLY_SYSTEMS = {
    "C1": lambda: W.config1(),
    # x edge 96: band pairs through the CTA-wide x passes
    "box_96_48_48": lambda: W.tiny_system(a=10.0, ecut=6.0, natom=3, fft_box=(96, 48, 48)),
}


@pytest.mark.parametrize("prec,tol", [(K.KSS_PREC_FP64, 1e-10), (K.KSS_PREC_MIXED, 2e-5)])
@pytest.mark.parametrize("nb", [6, 5])
@pytest.mark.parametrize("system", list(GAMMA_APPLY_SYSTEMS))
def test_apply_gamma_matches_oracle(ctx, prec, tol, nb, system):
    import torch
    from tests.kss_helpers import rel_err_rows
    s = GAMMA_APPLY_SYSTEMS[system]()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        c = symmetric_block(p.basis, nb, 17)
        cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
        psi = torch.from_numpy(c).to(cdt).cuda()
        out = torch.zeros_like(psi)
        K.kss_apply_H_gamma(sysh, 0, psi, out, prec)
        torch.cuda.synchronize()
        assert rel_err_rows(out.cpu().numpy(), p.apply(c)) < tol
    finally:
        K.kss_sys_destroy(sysh)
