"""The hand-written FP64 dense generalised Hermitian eigensolver (the Rayleigh-Ritz subspace problem,
§5.1) through the C ABI, against the oracle's dense LAPACK eigensolve.

Bars: eigenvalues within 1e-11 of the largest |eigenvalue| of the oracle's (a backward-stable
solver's error on these well-conditioned B); eigenvectors checked by their own invariants, since
degenerate and clustered eigenvalues make individual vectors gauge-dependent: the residual
|A X - B X diag(w)| <= 1e-11 |A| and B-orthonormality |X^H B X - I| <= 1e-11.  Real symmetric
pencils run in real arithmetic and are checked the same way (and for exactly real outputs); the
returned Cholesky factor is checked against LAPACK's.
"""
import numpy as np
import pytest

import oracle as O
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_destroy(c)


def pencil(n, seed, real=False, cond=1e3):
    rng = np.random.default_rng(seed)
    def rnd():
        m = rng.standard_normal((n, n))
        return m if real else m + 1j * rng.standard_normal((n, n))
    a = rnd()
    A = (a + a.conj().T) / 2
    m = rnd()
    B = m @ m.conj().T / n + np.eye(n) / cond
    return A.astype(np.complex128), B.astype(np.complex128)


def to_dev(M, ld=None):
    """Column-major device copy: a (ncols, ld) tensor whose row j holds column j (rows past n are
    filled with a marker value that must stay untouched by the lower-triangle reads)."""
    import torch
    n = M.shape[0]
    ld = ld or n
    T = np.full((n, ld), 5.0 + 5.0j)
    T[:, :n] = M.T
    # poison the strictly upper triangle: the solver reads the lower triangles only
    for j in range(n):
        T[j, :j] = np.nan + 1j * np.nan
    return torch.from_numpy(T).cuda()


def check(A, B, w, X, tol=1e-11):
    wr, _ = O.lowest_generalized_eigenpairs(A, B, A.shape[0])
    scale = max(1.0, np.max(np.abs(wr)))
    assert np.max(np.abs(w - wr)) <= tol * scale, np.max(np.abs(w - wr))
    R = A @ X - (B @ X) * w[None, :]
    assert np.max(np.abs(R)) <= tol * max(1.0, np.max(np.abs(A))) * max(1.0, np.max(np.abs(X))), np.max(np.abs(R))
    G = X.conj().T @ B @ X
    assert np.max(np.abs(G - np.eye(A.shape[0]))) <= tol * max(1.0, np.linalg.norm(B, 2))


def run(ctx, pencils, real=False, lds=None):
    import torch
    As = [to_dev(A, None if lds is None else lds[i]) for i, (A, _) in enumerate(pencils)]
    Bs = [to_dev(B) for _, B in pencils]
    ws = [torch.zeros(max(1, A.shape[0]), dtype=torch.float64, device="cuda") for A, _ in pencils]
    info = K.kss_dense_hegv(ctx, As, Bs, ws, real=real)
    out = []
    for i, (A, B) in enumerate(pencils):
        n = A.shape[0]
        T = As[i].cpu().numpy()
        if lds is not None:
            assert np.all(T[:, n:] == 5.0 + 5.0j)  # rows past n untouched
        out.append((ws[i].cpu().numpy()[:n], T[:, :n].T.copy()))
    return info, out


@pytest.mark.parametrize("n", [1, 2, 3, 17, 31, 32, 64, 159, 160, 301, 564])
def test_single_pencil(ctx, n):
    A, B = pencil(n, seed=n)
    info, [(w, X)] = run(ctx, [(A, B)])
    assert info[0] == 0
    check(A, B, w, X)


def test_batched_pencils_of_uneven_order_with_padding(ctx):
    ps = [pencil(n, seed=100 + n) for n in (5, 33, 96, 141, 7, 120)]
    lds = [p[0].shape[0] + 3 for p in ps]
    info, out = run(ctx, ps, lds=lds)
    assert np.all(info == 0)
    for (A, B), (w, X) in zip(ps, out):
        check(A, B, w, X)


@pytest.mark.parametrize("n", [40, 200])
def test_degenerate_clusters(ctx, n):
    """Exactly degenerate eigenvalues (shells of 1, 6, 12 and the rest, as in the free-electron
    spectrum) in a random unitary frame, B = I: the cluster's vectors must come out orthonormal."""
    rng = np.random.default_rng(7)
    lam = np.concatenate([np.zeros(1), np.full(6, 0.2), np.full(12, 0.4), np.linspace(0.5, 2.0, n - 19)])
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    A = (q * lam[None, :]) @ q.conj().T
    A = (A + A.conj().T) / 2
    B = np.eye(n, dtype=np.complex128)
    info, [(w, X)] = run(ctx, [(A, B)])
    assert info[0] == 0
    check(A, B, w, X)


@pytest.mark.parametrize("n", [1, 2, 24, 31, 32, 159, 300, 700])
def test_real_symmetric(ctx, n):
    """Real symmetric pencils (solved in real arithmetic): a single pencil runs on one CTA below
    order 32 and on the cooperative grid from 32; imaginary parts planted in the inputs are
    ignored."""
    A, B = pencil(n, seed=3 * n, real=True)
    rng = np.random.default_rng(n)
    junk = 1j * rng.standard_normal((n, n))
    info, [(w, X)] = run(ctx, [(A + junk, B + junk.T)], real=True)
    assert info[0] == 0
    assert np.all(X.imag == 0)
    check(A.real.astype(np.complex128), B.real.astype(np.complex128), w, X)


def test_real_batched_pencils_of_uneven_order_with_padding(ctx):
    ps = [pencil(n, seed=200 + n, real=True) for n in (3, 40, 97, 150, 8)]
    lds = [p[0].shape[0] + 5 for p in ps]
    info, out = run(ctx, ps, real=True, lds=lds)
    assert np.all(info == 0)
    for (A, B), (w, X) in zip(ps, out):
        assert np.all(X.imag == 0)
        check(A, B, w, X)


@pytest.mark.parametrize("n", [40, 200])
def test_real_degenerate_clusters(ctx, n):
    """Exactly degenerate shells in a random orthogonal frame, B = I, in real arithmetic."""
    rng = np.random.default_rng(9)
    lam = np.concatenate([np.zeros(1), np.full(6, 0.2), np.full(12, 0.4), np.linspace(0.5, 2.0, n - 19)])
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (q * lam[None, :]) @ q.T
    A = ((A + A.T) / 2).astype(np.complex128)
    B = np.eye(n, dtype=np.complex128)
    info, [(w, X)] = run(ctx, [(A, B)], real=True)
    assert info[0] == 0
    check(A, B, w, X)


@pytest.mark.parametrize("n,real", [(50, False), (50, True), (260, False), (260, True)])
def test_cholesky_factor_returned(ctx, n, real):
    """On return the lower triangle of B holds L with B = L L^H (LAPACK's factor: positive real
    diagonal), the strictly upper triangle is untouched."""
    import torch
    A, B = pencil(n, seed=11 * n, real=real)
    Bd = to_dev(B)
    Ad = to_dev(A)
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = K.kss_dense_hegv(ctx, [Ad], [Bd], [w], real=real)
    assert info[0] == 0
    T = Bd.cpu().numpy().T  # column-major back to (row, col)
    L = np.tril(T)
    ref = np.linalg.cholesky(B)
    assert np.max(np.abs(L - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.all(np.isnan(T[np.triu_indices(n, 1)]))
    if real:
        assert np.all(L.imag == 0)


@pytest.mark.parametrize("n", [12, 200])
def test_not_positive_definite(ctx, n):
    """B with a negative eigenvalue: the Cholesky stops with info = j + 1 > 0 (LAPACK convention)."""
    A, B = pencil(n, seed=5)
    B = B - 2.0 * np.linalg.norm(B, 2) * np.outer(np.eye(n)[n // 2], np.eye(n)[n // 2])
    info, _ = run(ctx, [(A, B)])
    assert 0 < info[0] <= n
