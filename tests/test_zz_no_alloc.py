"""kss_apply_H_noalloc: H psi without any device allocation, checked against kss_apply_H.

Some callers of this library cannot allocate device memory when they need H psi: work being
recorded into a CUDA graph, an application whose device memory belongs to another allocator,
or a latency-critical loop that must not pay for cudaMalloc/cudaFree (cudaFree synchronises the
device).  The no-alloc entry point keeps every temporary in one static device array instead.

Each case calls the new entry point twice in a row through the C ABI (the array keeps the first
call's contents, so the second call shows that leftovers do not leak into results) and compares
both results with kss_apply_H on the same input: 1e-10 relative per band in FP64, 2e-5 in the
mixed precision (the tolerances of the other H psi parity tests).  The second call must not
change the device's free memory; the first call in the process may commit the static array
itself (CUDA loads the module that holds it lazily), and no more than that.  This file is named
so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, rel_err_rows, setup

pytestmark = pytest.mark.gpu

TOL = {K.KSS_PREC_FP64: 1e-10, K.KSS_PREC_MIXED: 2e-5}
MIB = 1024 * 1024
SCRATCH = 64 * MIB  # KSS_NOALLOC_SCRATCH_BYTES


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


def _two_calls(sysh, ik, psi, prec):
    """Two kss_apply_H_noalloc calls in a row; results and free device memory around each."""
    import torch
    outs, free = [], []
    for _ in range(2):
        out = torch.full_like(psi, complex(3.0, -3.0))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        K.kss_apply_H_noalloc(sysh, ik, psi, out, prec)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        outs.append(out.cpu().numpy())
    return outs, free


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
        outs, free = _two_calls(sysh, ik, psi, prec)
        for o in outs:
            assert rel_err_rows(o, ref_h) < TOL[prec]
        # at most the static array (plus module overhead) is committed by the first call ...
        assert free[0] - free[1] <= SCRATCH + 16 * MIB
        # ... and the second call allocates nothing on the device
        assert free[3] == free[2]
    finally:
        K.kss_sys_destroy(sysh)


def test_noalloc_after_context_rebuilt():
    """A context destroyed and made again looks the scratch address up again and gives the same
    results as kss_apply_H, two calls in a row, with no allocation in the second."""
    import torch
    ensure_built()
    s = W.config1()
    for _ in range(2):
        c = make_ctx()
        sysh = setup(c, s)
        try:
            npw = K.kss_sphere(sysh, 0).shape[0]
            psi = torch.from_numpy(W.random_block(npw, 12, seed=32)).cuda()
            ref = torch.empty_like(psi)
            K.kss_apply_H(sysh, 0, psi, ref, K.KSS_PREC_FP64)
            torch.cuda.synchronize()
            outs, free = _two_calls(sysh, 0, psi, K.KSS_PREC_FP64)
            for o in outs:
                assert rel_err_rows(o, ref.cpu().numpy()) < TOL[K.KSS_PREC_FP64]
            assert free[3] == free[2]
        finally:
            K.kss_sys_destroy(sysh)
            torch.cuda.synchronize()
            K.kss_destroy(c)


def test_noalloc_rejects_requests_beyond_scratch(ctx):
    """A band block whose projector coefficients alone exceed the static scratch (C2: 256
    projectors x 8400 bands x 16 B = 34 MB, twice with the partial sums, plus one FFT slab) is
    refused with KSS_EINVAL and a message.  The buffers are really sized for the request (2 x 4.6
    GB), so the call never holds a pointer past an allocation, refused or not."""
    import torch
    s = W.config2()
    s.kpts = s.kpts[:1]
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, 0).shape[0]
        nb = 8400
        psi = torch.zeros((nb, npw), dtype=torch.complex128, device="cuda")
        hpsi = torch.zeros_like(psi)
        with pytest.raises(K.KssError) as e:
            K.kss_apply_H_noalloc(sysh, 0, psi, hpsi, K.KSS_PREC_FP64)
        assert e.value.status == K.KSS_EINVAL
        assert "scratch" in K.kss_last_error(ctx)
        torch.cuda.synchronize()
        assert not torch.any(hpsi != 0)  # nothing was launched
        del psi, hpsi
        torch.cuda.empty_cache()
    finally:
        K.kss_sys_destroy(sysh)
