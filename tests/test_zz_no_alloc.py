"""kss_apply_H_noalloc: H psi without any device allocation, checked against kss_apply_H.

Some callers of this library cannot allocate device memory when they need H psi: work being
recorded into a CUDA graph, an application whose device memory belongs to another allocator,
or a latency-critical loop that must not pay for cudaMalloc/cudaFree (cudaFree synchronises the
device).  The no-alloc entry point keeps every temporary in one static device array instead.

Each case calls the new entry point twice in a row through the C ABI (the array keeps the first
call's contents, so the second call shows that leftovers do not leak into results) and compares
both results with kss_apply_H on the same input: 1e-10 relative per band in FP64, 2e-5 in the
mixed precision (the tolerances of the other H psi parity tests).  The second call must not
change the device's free memory.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, rel_err_rows, setup

pytestmark = pytest.mark.gpu

TOL = {K.KSS_PREC_FP64: 1e-10, K.KSS_PREC_MIXED: 2e-5}


@pytest.fixture(scope="module")
def ctx():
    import torch
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_destroy(c)


CASES = [
    ("C1_fp64", W.config1, 20, K.KSS_PREC_FP64, None),
    ("C1_mixed", W.config1, 20, K.KSS_PREC_MIXED, None),
    ("C2_k0_fp64_64_bands", W.config2, 64, K.KSS_PREC_FP64, 1),   # several band chunks
    ("C2_k1_mixed_40_bands", W.config2, 40, K.KSS_PREC_MIXED, 2),
]


@pytest.mark.parametrize("name,mk,nb,prec,nk", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_apply_h(ctx, name, mk, nb, prec, nk):
    import torch
    s = mk()
    if nk is not None:
        s.kpts = s.kpts[:nk]
    ik = len(s.kpts) - 1
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, ik).shape[0]
        cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
        psi = torch.from_numpy(W.random_block(npw, nb, seed=31)).to(cdt).cuda()
        ref = torch.empty_like(psi)
        K.kss_apply_H(sysh, ik, psi, ref, prec)
        torch.cuda.synchronize()
        ref_h = ref.cpu().numpy()
        outs = []
        free = []
        for _ in range(2):
            out = torch.full_like(psi, complex(3.0, -3.0))
            torch.cuda.synchronize()
            free.append(torch.cuda.mem_get_info()[0])
            K.kss_apply_H_noalloc(sysh, ik, psi, out, prec)
            torch.cuda.synchronize()
            free.append(torch.cuda.mem_get_info()[0])
            outs.append(out.cpu().numpy())
        for o in outs:
            assert rel_err_rows(o, ref_h) < TOL[prec]
        # the second call allocates nothing on the device
        assert free[3] == free[2]
    finally:
        K.kss_sys_destroy(sysh)


def test_noalloc_rejects_requests_beyond_scratch(ctx):
    """A band block whose projector coefficients alone exceed the static scratch is refused with
    KSS_EINVAL and a message; nothing is launched (the buffers are not touched)."""
    import torch
    s = W.config2()
    s.kpts = s.kpts[:1]
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, 0).shape[0]
        dummy = torch.zeros((1, npw), dtype=torch.complex128, device="cuda")
        L = K.lib()
        st = L.kss_apply_H_noalloc(sysh.h, 0, 40000, dummy.data_ptr(), dummy.data_ptr() + 16 * npw,
                                   npw, K.KSS_PREC_FP64)
        assert st == K.KSS_EINVAL
        assert "scratch" in K.kss_last_error(ctx)
    finally:
        K.kss_sys_destroy(sysh)
