"""Several solvers stepped together (kss_solver_step_many) against the same solvers stepped one
at a time, and against the oracle.

The pipelined call runs each solver's Rayleigh-Ritz on a helper stream while the next solver's
filter runs on the context stream; the kernels and their launch shapes are the same, so the
iterates must agree with the one-at-a-time path to rounding (here: bit for bit is expected, the
bar is 1e-12 Ha) and the eigenvalues with the oracle's dense diagonalisation.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, setup

pytestmark = pytest.mark.gpu

KPTS = [(0.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.25, 0.25, -0.25)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_destroy(c)


def run(ctx, s, nband, prec, tol, many, max_steps=40):
    sysh = setup(ctx, s)
    svs = [K.kss_solver_create(sysh, ik, nband, K.make_opts(tol=tol, prec=prec, seed=31 + ik))
           for ik in range(len(s.kpts))]
    try:
        steps = 0
        conv = [False] * len(svs)
        while not all(conv) and steps < max_steps:
            if many:
                conv = K.kss_solver_step_many(svs)
            else:
                conv = [K.kss_solver_step(sv) for sv in svs]
            steps += 1
        out = [K.kss_solver_results(sv) for sv in svs]
        return steps, conv, out
    finally:
        for sv in svs:
            K.kss_solver_destroy(sv)
        K.kss_sys_destroy(sysh)


@pytest.mark.parametrize("prec,tol,bar", [(K.KSS_PREC_FP64, 1e-9, 1e-8), (K.KSS_PREC_MIXED, 1e-6, 1e-6)])
def test_step_many_matches_sequential(ctx, prec, tol, bar):
    s = W.tiny_system(a=7.0, ecut=3.0, natom=3, kpts=KPTS)
    nband = 10
    n1, c1, seq = run(ctx, s, nband, prec, tol, many=False)
    n2, c2, par = run(ctx, s, nband, prec, tol, many=True)
    # a mixed solve ends with an FP64 refinement and is done even when that leaves a residual
    # above tol; its bar is the eigenvalue error
    if prec == K.KSS_PREC_FP64:
        assert all(c1)
    assert c1 == c2 and n1 == n2
    for ik, ((e1, r1, st1), (e2, r2, st2)) in enumerate(zip(seq, par)):
        assert np.max(np.abs(e1 - e2)) <= 1e-12, (ik, e1 - e2)
        assert np.max(np.abs(r1 - r2)) <= 1e-12, (ik, r1 - r2)
        assert st1["iters"] == st2["iters"] and st1["napply"] == st2["napply"]
        p = O.build_problem(s, ik)
        ref, _ = O.lowest_eigenpairs(p.dense(), nband)
        assert np.max(np.abs(np.sort(e2) - ref)) < bar, (ik, np.sort(e2) - ref)


def test_step_many_edge_cases(ctx):
    s = W.tiny_system(a=6.5, ecut=2.5, natom=2, kpts=KPTS[1:])
    sysh = setup(ctx, s)
    a = K.kss_solver_create(sysh, 0, 6, K.make_opts(tol=1e-9, seed=3))
    b = K.kss_solver_create(sysh, 1, 6, K.make_opts(tol=1e-9, seed=4))
    try:
        assert K.kss_solver_step_many([]) == []
        # first call: the initial Rayleigh-Ritz of each (one step each, a listed twice steps once)
        K.kss_solver_step_many([a, a, b])
        assert K.kss_solver_results(a)[2]["iters"] == 0
        K.kss_solver_step_many([a, a, b])
        assert K.kss_solver_results(a)[2]["iters"] == 1
        assert K.kss_solver_results(b)[2]["iters"] == 1
        # run a to convergence alone, then a done solver is skipped
        while not K.kss_solver_step(a):
            pass
        it_a = K.kss_solver_results(a)[2]["iters"]
        K.kss_solver_step_many([a, b])
        assert K.kss_solver_results(a)[2]["iters"] == it_a
        assert K.kss_solver_results(b)[2]["iters"] == 2
    finally:
        K.kss_solver_destroy(a)
        K.kss_solver_destroy(b)
        K.kss_sys_destroy(sysh)


def test_step_many_profile_counts_helper_launches(ctx):
    s = W.tiny_system(a=6.5, ecut=2.5, natom=2, kpts=KPTS[:2])
    sysh = setup(ctx, s)
    svs = [K.kss_solver_create(sysh, ik, 6, K.make_opts(tol=1e-9, seed=9 + ik)) for ik in range(2)]
    try:
        K.kss_solver_step_many(svs)
        K.kss_profile_enable(ctx, True)
        K.kss_solver_step_many(svs)
        names = {}
        nk, launches = K.kss_profile_count(ctx)
        for i in range(nk):
            name, cnt, ms = K.kss_profile_entry(ctx, i)
            names[name] = cnt
        K.kss_profile_enable(ctx, False)
        # the Gram products and rotations ran on the helper streams and are counted
        assert sum(c for n, c in names.items() if n.endswith(":gram")) >= 4
        assert sum(c for n, c in names.items() if n.endswith(":rotate")) >= 4
        assert launches >= sum(names.values())
    finally:
        for sv in svs:
            K.kss_solver_destroy(sv)
        K.kss_sys_destroy(sysh)
