"""GPU parity of the path's complex GEMMs (kss_gemm) against numpy complex128 products.

FP64 engine (FP64-accurate digit products on the tensor cores): within 1e-12 relative.  Tensor-core engine (complex64 data, BF16 hi/lo split,
FP32 accumulation): the dropped lo*lo term and the BF16 rounding of the split leave a relative
error of order 2^-16 per product, so max|dC| / max|C| < 1e-4 is the bar.
"""
import numpy as np
import pytest

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


def crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


SHAPES = [  # (op, M, N, K)
    (0, 16, 20, 1503),      # C1 projector coefficients
    (0, 37, 150, 3001),     # ragged
    (0, 256, 90, 34181),    # C2-like projector coefficients, long K
    (0, 130, 130, 777),     # Gram-like, ragged tile edges
    (1, 1503, 20, 16),      # C1 nonlocal accumulation
    (1, 3001, 70, 37),      # ragged
    (1, 2000, 140, 140),    # rotation-like
    (1, 100, 30, 4000),     # A B form with a K-split (partial sums + combine)
    (0, 1300, 1300, 64),    # more output tiles than SMs (several waves, no K-split)
]


@pytest.mark.parametrize("op,M,N,Kd", SHAPES)
@pytest.mark.parametrize("prec", [K.KSS_PREC_FP64, K.KSS_PREC_MIXED])
def test_gemm(ctx, op, M, N, Kd, prec):
    import torch
    rng = np.random.default_rng(M * 7 + N * 13 + Kd)
    # column-major matrices stored as (ncols, ld) arrays
    if op == 0:
        A = crand(rng, (M, Kd))      # A: Kd x M, columns along axis 0
    else:
        A = crand(rng, (Kd, M))      # A: M x Kd
    B = crand(rng, (N, Kd))          # B: Kd x N
    C0 = crand(rng, (N, M))
    alpha, beta = 0.7 - 0.2j, 0.5 + 0.25j
    Am = A.T if op == 0 else A.T     # numpy (rows, cols) view of the column-major matrix
    Bm = B.T
    ref = alpha * ((Am.conj().T if op == 0 else Am) @ Bm) + beta * C0.T
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    tA = torch.from_numpy(A).to(cdt).cuda()
    tB = torch.from_numpy(B).to(cdt).cuda()
    tC = torch.from_numpy(C0).to(cdt).cuda()
    K.kss_gemm(ctx, op, tA, tB, tC, alpha, beta, prec)
    torch.cuda.synchronize()
    got = tC.cpu().numpy().T
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    tol = 1e-12 if prec == K.KSS_PREC_FP64 else 1e-4
    assert err < tol, err


@pytest.mark.parametrize("op", [0, 1])
def test_gemm_fp64_badly_scaled_rows(ctx, op):
    """FP64 products with rows and columns spanning 30 orders of magnitude (the filtered block's
    columns and the projector table's decaying entries differ in scale): every row and column
    of the digit form carries its own exponent, so each entry of C keeps the accuracy of the
    49-bit digit form (about 1e-13 of its own row and column scales times sqrt(K)) instead of losing
    it to the largest scale in the matrix."""
    import torch
    rng = np.random.default_rng(11 + op)
    M, N, Kd = 150, 70, 3000
    ra = 10.0 ** rng.uniform(-15, 15, M)
    rb = 10.0 ** rng.uniform(-15, 15, N)
    if op == 0:
        A = crand(rng, (M, Kd)) * ra[:, None]
    else:
        A = crand(rng, (Kd, M)) * ra[None, :]
    B = crand(rng, (N, Kd)) * rb[:, None]
    C0 = np.zeros((N, M), dtype=np.complex128)
    Am, Bm = A.T, B.T
    ref = (Am.conj().T if op == 0 else Am) @ Bm
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    K.kss_gemm(ctx, op, tA, tB, tC, 1.0, 0.0, K.KSS_PREC_FP64)
    torch.cuda.synchronize()
    got = tC.cpu().numpy().T
    scale = np.abs(ra)[:, None] * np.abs(rb)[None, :] * np.sqrt(Kd)
    assert np.max(np.abs(got - ref) / scale) < 1e-12


def test_gemm_rejects_bad_sizes(ctx):
    import torch
    a = torch.zeros((4, 8), dtype=torch.complex64, device="cuda")
    L = K.lib()
    st = L.kss_gemm(ctx, 0, 4, 4, 8, a.data_ptr(), 7, a.data_ptr(), 8, a.data_ptr(), 8,
                    1.0, 0.0, 0.0, 0.0, K.KSS_PREC_MIXED)
    assert st == K.KSS_EINVAL
    st = L.kss_gemm(ctx, 2, 4, 4, 8, a.data_ptr(), 8, a.data_ptr(), 8, a.data_ptr(), 8,
                    1.0, 0.0, 0.0, 0.0, K.KSS_PREC_MIXED)
    assert st == K.KSS_EINVAL


def test_bounded_wait_gives_up_and_context_stays_usable(ctx):
    """The failure path of the bounded device waits, without a fault: a wait on a word that nothing
    writes gives up after its limit, the host reads KSS_ETIMEOUT and a message, the flag is
    cleared, and the context goes on computing correct products."""
    import time
    import torch
    L = K.lib()
    t0 = time.perf_counter()
    st = K.kss_selftest_bounded_wait(ctx, 50.0)
    dt = time.perf_counter() - t0
    assert st == K.KSS_ETIMEOUT
    assert b"gave up" in L.kss_last_error(ctx)
    assert 0.045 < dt < 5.0
    assert K.kss_selftest_bounded_wait(ctx, 0.0) == K.KSS_EINVAL
    assert K.kss_selftest_bounded_wait(ctx, 2000.0) == K.KSS_EINVAL
    rng = np.random.default_rng(3)
    A, B = crand(rng, (40, 300)), crand(rng, (24, 300))
    C = np.zeros((24, 40), dtype=np.complex128)
    tA, tB = (torch.from_numpy(x).to(torch.complex64).cuda() for x in (A, B))
    tC = torch.from_numpy(C).to(torch.complex64).cuda()
    K.kss_gemm(ctx, 0, tA, tB, tC, 1.0, 0.0, K.KSS_PREC_MIXED)   # raises if the flag were still set
    torch.cuda.synchronize()
    ref = A.conj() @ B.T
    got = tC.cpu().numpy().T
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-4


@pytest.mark.parametrize("prec", [K.KSS_PREC_FP64, K.KSS_PREC_MIXED], ids=["fp64", "mixed"])
def test_gemm_split_autotuner_and_every_candidate(ctx, prec):
    """The K-split of the tensor-core products is tuned at first use of a shape (table entry with
    several candidates timed), and every split computes the same product: each one pinned in turn
    gives the numpy product within the precision's bar."""
    import torch
    K.kss_autotune_clear()
    rng = np.random.default_rng(21)
    M, N, Kd = 150, 130, 9000                 # few output tiles, long K: the split matters
    A = crand(rng, (M, Kd))
    B = crand(rng, (N, Kd))
    ref = A.conj() @ B.T                     # (M x N)
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    tol = 1e-12 if prec == K.KSS_PREC_FP64 else 1e-4
    tA, tB = (torch.from_numpy(x).to(cdt).cuda() for x in (A, B))

    def run():
        tC = torch.zeros((N, M), dtype=cdt, device="cuda")
        K.kss_gemm(ctx, 0, tA, tB, tC, 1.0, 0.0, prec)
        torch.cuda.synchronize()
        got = tC.cpu().numpy().T
        return np.max(np.abs(got - ref)) / np.max(np.abs(ref))

    assert run() < tol
    kind = 1 if prec == K.KSS_PREC_FP64 else 0
    entries = [e for e in K.kss_autotune_gemm_table() if e["kind"] == kind and e["Nr"] == N]
    assert len(entries) == 1 and entries[0]["ncand"] >= 2 and entries[0]["ms"] > 0
    e = entries[0]
    assert e["Mr"] == 2 * M
    forms = (0, 1, 2) if kind == 0 else (0,)
    if kind == 0:
        assert e["ncand"] >= 6 and e["form"] in forms
    for form in forms:
        for sp in sorted({1, 2, 3, 5, e["splits"], max(1, e["kblocks"] // 24)}):
            K.kss_autotune_gemm_put(e["device"], kind, e["Mr"], e["Nr"], e["kblocks"], sp, form)
            assert run() < tol, (form, sp)
    with pytest.raises(K.KssError):
        K.kss_autotune_gemm_put(e["device"], kind, e["Mr"], e["Nr"], e["kblocks"], 1, 3)
    K.kss_autotune_clear()
    assert K.kss_autotune_gemm_table() == []


@pytest.mark.parametrize("op,M,N,Kd", SHAPES)
def test_split_bf16_every_form(ctx, op, M, N, Kd):
    """Every kernel form of the split-BF16 products (one CTA per 128 x 128 tile; persistent CTAs
    with two TMEM accumulators on 128- and 64-column tiles), with and without a K-split, pinned in
    turn, gives the numpy product within 1e-4 (alpha and beta complex, ragged edges)."""
    import torch
    rng = np.random.default_rng(M * 5 + N * 11 + Kd + op)
    A = crand(rng, (M, Kd)) if op == 0 else crand(rng, (Kd, M))
    B = crand(rng, (N, Kd))
    C0 = crand(rng, (N, M))
    alpha, beta = 0.6 + 0.3j, -0.4 + 0.2j
    Am = A.T
    ref = alpha * ((Am.conj().T if op == 0 else Am) @ B.T) + beta * C0.T
    tA, tB = (torch.from_numpy(x).to(torch.complex64).cuda() for x in (A, B))
    kblocks = (2 * Kd + 63) // 64
    K.kss_autotune_clear()
    try:
        for form in (0, 1, 2):
            for sp in (1, 4):
                sp = min(sp, max(1, kblocks // (8 if form == 0 else 4)))
                K.kss_autotune_gemm_put(0, 0, 2 * M, N, kblocks, sp, form)
                tC = torch.from_numpy(C0).to(torch.complex64).cuda()
                K.kss_gemm(ctx, op, tA, tB, tC, alpha, beta, K.KSS_PREC_MIXED)
                torch.cuda.synchronize()
                got = tC.cpu().numpy().T
                err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
                assert err < 1e-4, (form, sp, err)
    finally:
        K.kss_autotune_clear()
