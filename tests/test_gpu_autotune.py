"""The autotuner of the FFT pass-B schedule, on the GPU through the C ABI.

* Every schedule the tuner can pick for a box length (the CTA-wide form with each compile-time
  split N = A * B at 256 and 384 threads, 128 too in single precision, and the per-warp form),
  pinned with kss_autotune_put, gives H psi within 1e-10 relative (FP64) / 2e-5 (mixed) of the
  oracle, for the config-1 cell (on a 25 x 24 x 24 box), config-4 lengths (30^3, 36^3, 40^3) and
  the config-2 box (96^3, whose splits run pruned stages).
* With tuning on, the first apply of a configuration adds one table entry whose choice was timed
  against every candidate; its result agrees with the built-in choice to rounding.
* The batch engine follows the table: the same batch with every entry pinned to the per-warp
  form gives the same eigenvalues.
"""
import dataclasses
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, rel_err_rows, setup

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def wide_splits():
    """(A, B) pairs of the KSS_WIDE_SPLITS instance list, read from the kernel source."""
    src = open(os.path.join(ROOT, "paper_2507_08578_gb300", "csrc", "local_kernels.cuh")).read()
    m = re.search(r"#define KSS_WIDE_SPLITS\(X\)(.*?)\n\n", src, flags=re.S)
    return [(int(a), int(b)) for a, b in re.findall(r"X\((\d+),\s*(\d+)\)", m.group(1))]


def candidates(N, prec=K.KSS_PREC_FP64):
    nts = (128, 256, 384) if prec == K.KSS_PREC_MIXED else (256, 384)
    c = [(a, b, nt) for a, b in wide_splits() if a * b == N for nt in nts]
    return c + [(0, 0, 0)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_autotune_clear()
    K.kss_autotune_set(c, 1)
    K.kss_destroy(c)


def _apply(sysh, c, prec, npw):
    import torch
    cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
    psi = torch.from_numpy(c).to(cdt).cuda()
    hpsi = torch.zeros_like(psi)
    K.kss_apply_H(sysh, 0, psi, hpsi, prec)
    torch.cuda.synchronize()
    return hpsi.cpu().numpy()


CASES = [
    ("C1_24", lambda: W.config1(), K.KSS_PREC_FP64, 1e-10),
    # a cubic single-precision box of edge <= 25 takes the fused single-kernel local part, which has
    # no pass-B schedule; the config-1 cell on a 25 x 24 x 24 box keeps the three-pass form
    ("C1_25x24_mixed", lambda: dataclasses.replace(W.config1(), fft_box=(25, 24, 24)), K.KSS_PREC_MIXED, 2e-5),
    ("box30", lambda: W.tiny_system(a=8.0, ecut=6.0, natom=3, fft_box=(30, 30, 30)), K.KSS_PREC_FP64, 1e-10),
    ("box36_mixed", lambda: W.tiny_system(a=9.0, ecut=7.0, natom=3, fft_box=(36, 36, 36)), K.KSS_PREC_MIXED, 2e-5),
    ("box40", lambda: W.tiny_system(a=9.0, ecut=8.0, natom=2, fft_box=(40, 40, 40)), K.KSS_PREC_FP64, 1e-10),
    # the config-2 box (96^3, sphere |m| <= 20): every 96-point split has a pruned instance that
    # skips the zero inputs and discarded outputs of its strided stages
    ("C2_96", lambda: W.config2(), K.KSS_PREC_FP64, 1e-10),
    ("C2_96_mixed", lambda: W.config2(), K.KSS_PREC_MIXED, 2e-5),
]


@pytest.mark.parametrize("name,mk,prec,tol", CASES, ids=[c[0] for c in CASES])
def test_every_schedule_matches_oracle(ctx, name, mk, prec, tol):
    s = mk()
    sysh = setup(ctx, s)
    try:
        box = O.system_box(s)
        p = O.build_problem(s, 0, box=box)
        c = W.random_block(p.basis.npw, 5, seed=3)
        ref = p.apply(c)
        # one tuned apply: the table gets this configuration's entry (its key as the library sees it)
        K.kss_autotune_clear()
        K.kss_autotune_set(ctx, 1)
        tuned = _apply(sysh, c, prec, p.basis.npw)
        tab = K.kss_autotune_table()
        assert len(tab) == 1
        e = tab[0]
        N = box[1]
        cand = candidates(N, prec)
        assert e["N1"] == box[0] and e["N"] == N and e["ncand"] == len(cand)
        assert (e["A"], e["B"], e["threads"]) in [(a, b, t) for a, b, t in cand if t] or e["threads"] == 0
        assert rel_err_rows(tuned, ref) < tol
        outs = []
        for a, b, nt in cand:
            if nt == 0:  # per-warp form: its split is the library's cost-model choice
                a, b = e["A"], e["B"]
                if e["threads"]:
                    a, b = [(x, y) for x, y in wide_splits() if x * y == N][0]
            K.kss_autotune_put(0, prec, e["N1"], N, e["W3"], a, b, nt)
            out = _apply(sysh, c, prec, p.basis.npw)
            err = rel_err_rows(out, ref)
            assert err < tol, (a, b, nt, err)
            outs.append(out)
        # all schedules agree with each other to rounding
        for o in outs[1:]:
            assert rel_err_rows(o, outs[0]) < (1e-13 if prec == K.KSS_PREC_FP64 else 1e-5)
    finally:
        K.kss_sys_destroy(sysh)
        K.kss_autotune_clear()


def test_fused_box_consults_no_schedule(ctx):
    """The config-1 box (24^3) in single precision runs the fused local kernel: a tuned apply adds
    no table entry and still matches the oracle."""
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        c = W.random_block(p.basis.npw, 5, seed=3)
        K.kss_autotune_clear()
        K.kss_autotune_set(ctx, 1)
        out = _apply(sysh, c, K.KSS_PREC_MIXED, p.basis.npw)
        assert K.kss_autotune_table() == []
        assert rel_err_rows(out, p.apply(c)) < 2e-5
    finally:
        K.kss_sys_destroy(sysh)
        K.kss_autotune_clear()


def test_tuned_matches_builtin_and_table_reports(ctx):
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        c = W.random_block(p.basis.npw, 8, seed=4)
        K.kss_autotune_clear()
        K.kss_autotune_set(ctx, 0)
        r0 = _apply(sysh, c, K.KSS_PREC_FP64, p.basis.npw)
        assert K.kss_autotune_table() == []  # mode 0 adds nothing
        K.kss_autotune_set(ctx, 1)
        r1 = _apply(sysh, c, K.KSS_PREC_FP64, p.basis.npw)
        tab = K.kss_autotune_table()
        assert len(tab) == 1 and tab[0]["ms"] > 0 and tab[0]["precision"] == K.KSS_PREC_FP64
        assert rel_err_rows(r1, r0) < 1e-13
        # a second apply reuses the entry
        _apply(sysh, c, K.KSS_PREC_FP64, p.basis.npw)
        assert len(K.kss_autotune_table()) == 1
    finally:
        K.kss_sys_destroy(sysh)
        K.kss_autotune_clear()


def test_put_rejects_inconsistent_entries(ctx):
    with pytest.raises(K.KssError):
        K.kss_autotune_put(0, K.KSS_PREC_FP64, 24, 24, 15, 5, 5, 256)   # 5 * 5 != 24
    with pytest.raises(K.KssError):
        K.kss_autotune_put(0, K.KSS_PREC_FP64, 24, 24, 15, 4, 6, 64)    # threads
    with pytest.raises(K.KssError):
        K.kss_autotune_put(0, 7, 24, 24, 15, 4, 6, 256)                 # precision
    with pytest.raises(K.KssError):
        K.kss_autotune_put(0, K.KSS_PREC_FP64, 24, 24, 25, 4, 6, 256)   # W3 > N


def test_batch_follows_table(ctx):
    systems = [
        W.make_system("t1", 7.0, 6.0, 3, 6, seed=31, kpts=W.SHIFTED_222[:1]),
        W.make_system("t2", 8.0, 7.0, 4, 8, seed=32),
    ]
    handles = [setup(ctx, s) for s in systems]
    try:
        opts = K.make_opts(tol=1e-9, seed=9)
        args = ([h for h in handles], [0, 0], [s.nband for s in systems], opts)
        K.kss_autotune_clear()
        K.kss_autotune_set(ctx, 1)
        ev1 = K.kss_solve_batch(ctx, *args)[0]
        tab = K.kss_autotune_table()
        assert len(tab) >= 1
        for e in tab:  # pin every configuration to the per-warp form
            K.kss_autotune_put(e["device"], e["precision"], e["N1"], e["N"], e["W3"], e["A"], e["B"], 0)
        ev2 = K.kss_solve_batch(ctx, *args)[0]
        for a, b, s in zip(ev1, ev2, systems):
            assert np.max(np.abs(a - b)) < 1e-8
            assert np.max(np.abs(a - O.lowest_eigenpairs(O.build_problem(s, 0).dense(), s.nband)[0])) < 1e-8
    finally:
        for h in handles:
            K.kss_sys_destroy(h)
        K.kss_autotune_clear()
