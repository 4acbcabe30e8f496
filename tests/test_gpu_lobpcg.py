"""LOBPCG (the paper's second GPU eigensolver, §5.1) on the GPU through the C ABI, against the
oracle's dense diagonalisation and against ChebFi.

Bars: eigenvalues within 1e-8 Ha of the oracle, residuals <= tol, eigenvectors orthonormal to
1e-10, agreement with ChebFi within 1e-8 Ha; warm start from converged vectors converges at once.
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


CASES = {
    "C1": lambda: W.config1(),
    "shifted_2k": lambda: W.make_system("l2", 7.5, 6.0, 4, 12, seed=81, kpts=W.SHIFTED_222[1:3]),
    "C4.1": lambda: W.config4(3)[1],
}


@pytest.mark.parametrize("name", list(CASES))
def test_lobpcg_matches_oracle_and_chebfi(ctx, name):
    import torch
    s = CASES[name]()
    sysh = setup(ctx, s)
    try:
        for ik in range(min(2, len(s.kpts))):
            p = O.build_problem(s, ik)
            npw = p.basis.npw
            X = torch.zeros((s.nband, npw), dtype=torch.complex128, device="cuda")
            ev, rs, st, _ = K.kss_lobpcg_solve(sysh, ik, s.nband, K.make_opts(tol=1e-8, seed=4), evecs=X)
            w, _ = p.lowest(s.nband)
            assert np.max(np.abs(ev - w)) < 1e-8, np.max(np.abs(ev - w))
            assert rs.max() <= 1e-8 and st["iters"] >= 1 and st["napply"] > 0
            x = X.cpu().numpy()
            assert np.max(np.abs(x.conj() @ x.T - np.eye(s.nband))) < 1e-10
            ev2 = K.kss_chebfi_solve(sysh, ik, s.nband, K.make_opts(tol=1e-8, seed=4))[0]
            assert np.max(np.abs(ev - ev2)) < 1e-8
    finally:
        K.kss_sys_destroy(sysh)


def test_lobpcg_warm_start_and_statuses(ctx):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, 0).shape[0]
        X = torch.zeros((s.nband, npw), dtype=torch.complex128, device="cuda")
        ev, _, st, _ = K.kss_lobpcg_solve(sysh, 0, s.nband, K.make_opts(tol=1e-9, seed=2), evecs=X)
        ev2, _, st2, _ = K.kss_lobpcg_solve(sysh, 0, s.nband, K.make_opts(tol=1e-8, x0=X, x0_nb=s.nband, x0_ld=npw))
        assert st2["iters"] <= 2 and np.max(np.abs(ev2 - ev)) < 1e-8
        ev3, rs3, st3, status = K.kss_lobpcg_solve(sysh, 0, s.nband, K.make_opts(tol=1e-13, max_iter=2),
                                                   allow_noconv=True)
        assert status == K.KSS_ENOCONV and st3["iters"] == 2 and np.all(np.isfinite(ev3))
        with pytest.raises(K.KssError) as e:
            K.kss_lobpcg_solve(sysh, 0, s.nband, K.make_opts(prec=K.KSS_PREC_MIXED))
        assert e.value.status == K.KSS_ENOTSUP
    finally:
        K.kss_sys_destroy(sysh)
    sysS = setup(ctx, W.config1s())
    try:
        with pytest.raises(K.KssError) as e:
            K.kss_lobpcg_solve(sysS, 0, 16, K.make_opts())
        assert e.value.status == K.KSS_ENOTSUP
    finally:
        K.kss_sys_destroy(sysS)


@pytest.mark.parametrize("name", ["C1", "C4.1"])
def test_rmmdiis_refines_a_loose_solve(ctx, name):
    """RMM-DIIS from the vectors of a loose ChebFi solve (residual 1e-3, the whole block of nband +
    nbuffer bands) reaches 1e-8 and the oracle's eigenvalues."""
    import torch
    s = CASES[name]()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        npw = p.basis.npw
        nbuf = max(4, (s.nband + 9) // 10)
        m = s.nband + nbuf
        X0 = torch.zeros((m, npw), dtype=torch.complex128, device="cuda")  # trial vectors for the whole block
        K.kss_chebfi_solve(sysh, 0, m, K.make_opts(tol=1e-3, seed=6), evecs=X0)
        X = torch.zeros((s.nband, npw), dtype=torch.complex128, device="cuda")
        ev, rs, st, _ = K.kss_rmmdiis_solve(sysh, 0, s.nband, K.make_opts(tol=1e-8, nbuffer=nbuf, x0=X0, x0_nb=m,
                                                                          x0_ld=npw), evecs=X)
        w, _ = p.lowest(s.nband)
        assert np.max(np.abs(ev - w)) < 1e-8, np.max(np.abs(ev - w))
        assert rs.max() <= 1e-8 and st["iters"] >= 1
        x = X.cpu().numpy()
        assert np.max(np.abs(x.conj() @ x.T - np.eye(s.nband))) < 1e-10
    finally:
        K.kss_sys_destroy(sysh)


def test_rmmdiis_statuses(ctx):
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        with pytest.raises(K.KssError) as e:
            K.kss_rmmdiis_solve(sysh, 0, s.nband, K.make_opts())  # no trial vectors
        assert e.value.status == K.KSS_EINVAL
    finally:
        K.kss_sys_destroy(sysh)
