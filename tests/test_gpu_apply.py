"""GPU parity of the setup tables and of H psi against the FP64 oracle, through the C ABI.

Bars: index maps bit-exact; V(r), kinetic energies and projector table to rounding; H psi in
FP64 within 1e-10 relative (per band, both as a row norm and element by element against the
largest coefficient of the row); H psi in mixed precision (complex64 FFTs and products) within
2e-5 relative, the single-precision rounding of the FFT and product path.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx, rel_err_elem, rel_err_rows, setup

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    c = make_ctx()
    yield c
    torch.cuda.synchronize()
    K.kss_destroy(c)


def triclinic_system(kpts=((0.25, -0.25, 0.25),), box=(15, 18, 20)):
    lat = np.array([[6.0, 0.0, 0.0], [1.1, 6.3, 0.0], [-0.7, 0.9, 6.6]])
    rng = np.random.default_rng(99)
    pos = rng.random((3, 3)) @ lat
    D = rng.uniform(-1, 1, 12)
    return W.System(name="tri", lattice=lat, ecut=2.5, kpts=np.array(kpts, float), pos=pos, D=D,
                    nband=6, fft_box=box)


MAP_CASES = {
    "C1": lambda: W.config1(),
    "C2": lambda: W.config2(),
    "tiny_k": lambda: W.tiny_system(a=6.5, ecut=3.0, natom=2, kpts=[(0.25, 0.25, -0.25), (0.5, 0, 0.25)]),
    "triclinic": lambda: triclinic_system(),
    "C4.0": lambda: W.config4(3)[0],
    "C4.1": lambda: W.config4(3)[1],
}


@pytest.mark.parametrize("name", list(MAP_CASES))
def test_maps_bit_exact(ctx, name):
    s = MAP_CASES[name]()
    sysh = setup(ctx, s)
    try:
        info = K.kss_sys_info_get(sysh)
        box = O.system_box(s)
        assert tuple(info["fft_box"]) == tuple(box)
        for ik in range(len(s.kpts)):
            b = O.make_basis(s.lattice, s.ecut, s.kpts[ik], box)
            miller, off = K.kss_get_maps(sysh, ik)
            assert np.array_equal(miller, b.miller)
            assert np.array_equal(off.astype(np.int64), b.offset)
            assert np.array_equal(K.kss_sphere(sysh, ik), b.miller)
    finally:
        K.kss_sys_destroy(sysh)


@pytest.mark.parametrize("name", ["C1", "triclinic", "tiny_k"])
def test_tables(ctx, name):
    s = MAP_CASES[name]()
    sysh = setup(ctx, s)
    try:
        box = O.system_box(s)
        for ik in range(len(s.kpts)):
            p = O.build_problem(s, ik, box=box)
            V, kin, beta = K.kss_get_tables(sysh, ik)
            assert np.max(np.abs(V - p.V)) < 1e-13
            assert np.max(np.abs(kin - p.basis.kinetic)) < 1e-13 * max(1.0, kin.max())
            assert np.max(np.abs(beta.T - p.beta)) < 1e-13 * max(1.0, np.abs(p.beta).max())
        # rigorous bound >= largest eigenvalue
        H = O.build_problem(s, 0, box=box).dense()
        assert K.kss_upper_bound(sysh, 0) >= O.all_eigenvalues(H)[-1]
    finally:
        K.kss_sys_destroy(sysh)


def _apply_case(ctx, s, nb, pad, prec, ik=0, box=None, seed=5):
    import torch
    sysh = setup(ctx, s)
    try:
        box = box or O.system_box(s)
        p = O.build_problem(s, ik, box=box)
        npw = p.basis.npw
        c = W.random_block(npw, nb, seed=seed)
        cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
        ld = npw + pad
        psi = torch.zeros((nb, ld), dtype=cdt, device="cuda")
        psi[:, :npw] = torch.from_numpy(c).to(cdt)
        hpsi = torch.full((nb, ld), complex(7, 7), dtype=cdt, device="cuda")
        K.kss_apply_H(sysh, ik, psi, hpsi, prec)
        torch.cuda.synchronize()
        out = hpsi.cpu().numpy()
        ref = p.apply(c)
        # padding untouched
        if pad:
            assert np.all(out[:, npw:] == complex(7, 7))
        return max(rel_err_rows(out[:, :npw], ref), rel_err_elem(out[:, :npw], ref))
    finally:
        K.kss_sys_destroy(sysh)


APPLY_CASES = [
    ("C1", lambda: W.config1(), 20, 5),
    ("C1_one_band", lambda: W.config1(), 1, 0),
    ("triclinic_k", lambda: triclinic_system(), 3, 1),
    ("odd_box_25_27_30", lambda: W.tiny_system(a=6.0, ecut=3.0, natom=2, fft_box=(25, 27, 30),
                                               kpts=[(0.25, 0, -0.25)]), 17, 0),
    ("box_45_48_36", lambda: W.tiny_system(a=9.0, ecut=4.0, natom=3, fft_box=(45, 48, 36)), 5, 3),
    ("box_16_20_18_s_only", lambda: W.tiny_system(a=5.0, ecut=2.5, natom=2, fft_box=(16, 20, 18),
                                                  nproj_per_atom=1), 4, 0),
    ("no_projectors", lambda: W.tiny_system(a=5.0, ecut=2.5, natom=2, nproj_per_atom=0), 4, 0),
    ("C4.0_default_box", lambda: W.config4(1)[0], 9, 2),
    # power-of-two and 2^3*3^2 box edges (the CTA-wide middle pass needs N2 == N3)
    ("box_32_cubic", lambda: W.tiny_system(a=8.0, ecut=5.0, natom=3, fft_box=(32, 32, 32)), 5, 0),
    ("box_64_cubic_k", lambda: W.tiny_system(a=10.0, ecut=6.0, natom=3, fft_box=(64, 64, 64),
                                             kpts=[(0.25, 0.25, 0.25)]), 7, 2),
    ("box_72_cubic", lambda: W.tiny_system(a=10.0, ecut=6.0, natom=3, fft_box=(72, 72, 72)), 3, 0),
    ("box_32_64_72_k", lambda: W.tiny_system(a=10.0, ecut=6.0, natom=3, fft_box=(32, 64, 72),
                                             kpts=[(0.25, 0.0, -0.25)]), 6, 1),
    # x edge 96: the CTA-wide x passes, pruned to a small sphere's x window here ...
    ("box_96_48_48_k", lambda: W.tiny_system(a=10.0, ecut=6.0, natom=3, fft_box=(96, 48, 48),
                                             kpts=[(0.25, 0.0, -0.25)]), 5, 1),
    # ... and unpruned (|m| up to 28 along each axis: wider than the pruned instances cover)
    ("box_96_wide_sphere", lambda: W.tiny_system(a=20.0, ecut=40.0, natom=3, fft_box=(96, 96, 96)), 3, 0),
]


@pytest.mark.parametrize("name,mk,nb,pad", APPLY_CASES, ids=[c[0] for c in APPLY_CASES])
def test_apply_fp64(ctx, name, mk, nb, pad):
    err = _apply_case(ctx, mk(), nb, pad, K.KSS_PREC_FP64)
    assert err < FP64_TOL, err


MIXED_CASES = APPLY_CASES[:5] + APPLY_CASES[-6:]


@pytest.mark.parametrize("name,mk,nb,pad", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_apply_mixed(ctx, name, mk, nb, pad):
    err = _apply_case(ctx, mk(), nb, pad, K.KSS_PREC_MIXED)
    assert err < MIXED_TOL, err


# Cubic boxes of every length the fused single-kernel local path has an instance for (single
# precision: the whole box and V in one SM's shared memory), at shifted k-points (unpacked), with
# ragged band counts, padded rows, and more bands than CTAs (the persistent loop over bands).
FUSED_CASES = [
    ("fused_10_k_310_bands", lambda: W.tiny_system(a=5.0, ecut=2.0, natom=2, fft_box=(10, 10, 10),
                                                   kpts=[(0.25, 0.0, 0.0)]), 310, 3),
    ("fused_12_k", lambda: W.tiny_system(a=5.5, ecut=2.5, natom=2, fft_box=(12, 12, 12),
                                         kpts=[(0.1, 0.2, 0.3)]), 7, 0),
    ("fused_15_k", lambda: W.tiny_system(a=6.0, ecut=3.0, natom=2, fft_box=(15, 15, 15),
                                         kpts=[(0.25, 0.25, -0.25)]), 5, 2),
    ("fused_16_k", lambda: W.tiny_system(a=6.0, ecut=3.0, natom=3, fft_box=(16, 16, 16),
                                         kpts=[(0.5, 0.0, 0.25)]), 9, 1),
    ("fused_18_k", lambda: W.tiny_system(a=7.0, ecut=3.5, natom=3, fft_box=(18, 18, 18),
                                         kpts=[(0.0, 0.25, 0.0)]), 4, 0),
    ("fused_20_k", lambda: W.tiny_system(a=7.5, ecut=4.0, natom=3, fft_box=(20, 20, 20),
                                         kpts=[(0.125, -0.25, 0.375)]), 11, 4),
    ("fused_24_gamma", lambda: W.tiny_system(a=8.0, ecut=5.0, natom=3, fft_box=(24, 24, 24)), 6, 1),
    ("fused_25_k", lambda: W.tiny_system(a=9.0, ecut=5.0, natom=3, fft_box=(25, 25, 25),
                                         kpts=[(0.25, 0.25, 0.25)]), 3, 0),
]


@pytest.mark.parametrize("name,mk,nb,pad", FUSED_CASES, ids=[c[0] for c in FUSED_CASES])
def test_apply_mixed_fused_boxes(ctx, name, mk, nb, pad):
    """Against the oracle, element by element and per band, at the mixed-form tolerance; the
    profile shows the fused kernel ran (and none of the three slab passes)."""
    K.kss_profile_enable(ctx, True)
    err = _apply_case(ctx, mk(), nb, pad, K.KSS_PREC_MIXED)
    prof = K.profile_table(ctx)
    K.kss_profile_enable(ctx, False)
    assert err < MIXED_TOL, err
    assert prof.get("local_fused<f32>", (0, 0))[0] >= 1, prof
    assert not any(k.startswith("local_pass") for k in prof), prof


def test_apply_c2_sampled_bands(ctx):
    """Full-size C2 cell (96^3 box, 256 projectors): 4 bands per k-point against the oracle."""
    import torch
    s = W.config2()
    sysh = setup(ctx, s)
    try:
        box = tuple(s.fft_box)
        V = O.vloc_for(s, box)
        for ik in range(4):
            p = O.build_problem(s, ik, box=box, V=V)
            npw = p.basis.npw
            assert npw == 34181
            c = W.random_block(npw, 4, seed=40 + ik)
            psi = torch.from_numpy(c).cuda()
            hpsi = torch.empty_like(psi)
            K.kss_apply_H(sysh, ik, psi, hpsi, K.KSS_PREC_FP64)
            torch.cuda.synchronize()
            out, ref = hpsi.cpu().numpy(), p.apply(c)
            err = max(rel_err_rows(out, ref), rel_err_elem(out, ref))
            assert err < FP64_TOL, (ik, err)
    finally:
        K.kss_sys_destroy(sysh)


# Bands sampled from a full 564-band block (512 wanted + 52 buffer): the first and last band and
# bands on both sides of the 64-, 128- and 256-band tile edges of the projector products.
C2_SAMPLE = [0, 63, 64, 127, 128, 255, 256, 383, 511, 563]


@pytest.mark.parametrize("prec", [K.KSS_PREC_FP64, K.KSS_PREC_MIXED], ids=["fp64", "mixed"])
def test_apply_c2_full_block_sampled(ctx, prec):
    """H on the full C2 band block (96^3 box, 256 projectors, 564 bands: the shapes of a C2 solve,
    including the tensor-core projector products of the mixed form with their production tiling
    and K-split), at the first and last k-point; sampled bands against the oracle."""
    import torch
    s = W.config2()
    sysh = setup(ctx, s)
    try:
        box = tuple(s.fft_box)
        V = O.vloc_for(s, box)
        cdt = torch.complex128 if prec == K.KSS_PREC_FP64 else torch.complex64
        tol = FP64_TOL if prec == K.KSS_PREC_FP64 else MIXED_TOL
        for ik in (0, 3):
            p = O.build_problem(s, ik, box=box, V=V)
            npw = p.basis.npw
            c = W.random_block(npw, 564, seed=60 + ik)
            psi = torch.from_numpy(c).to(cdt).cuda()
            hpsi = torch.empty_like(psi)
            K.kss_apply_H(sysh, ik, psi, hpsi, prec)
            torch.cuda.synchronize()
            out = hpsi.cpu().numpy()[C2_SAMPLE].astype(np.complex128)
            cin = psi.cpu().numpy()[C2_SAMPLE].astype(np.complex128)  # the rounded input in mixed
            ref = p.apply(cin)
            err = max(rel_err_rows(out, ref), rel_err_elem(out, ref))
            assert err < tol, (ik, err)
    finally:
        K.kss_sys_destroy(sysh)


def test_cheb_step_epilogue(ctx):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        p = O.build_problem(s, 0)
        npw = p.basis.npw
        c = W.random_block(npw, 6, seed=1)
        cp = W.random_block(npw, 6, seed=2)
        al, be, ga = 0.37, -1.25, -0.81
        ref = al * p.apply(c) + be * c + ga * cp
        psi = torch.from_numpy(c).cuda()
        prev = torch.from_numpy(cp).cuda()
        out = torch.empty_like(psi)
        K.kss_cheb_step(sysh, 0, psi, prev, out, al, be, ga)
        torch.cuda.synchronize()
        assert rel_err_rows(out.cpu().numpy(), ref) < FP64_TOL
        # out aliasing psi_prev (the in-place form the filter uses)
        K.kss_cheb_step(sysh, 0, psi, prev, prev, al, be, ga)
        torch.cuda.synchronize()
        assert rel_err_rows(prev.cpu().numpy(), ref) < FP64_TOL
    finally:
        K.kss_sys_destroy(sysh)


def test_apply_host_entry_point(ctx):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, 0).shape[0]
        c = W.random_block(npw, 5, seed=3)
        out = np.zeros_like(c)
        K.kss_apply_H_host(sysh, 0, c, out)
        psi = torch.from_numpy(c).cuda()
        h = torch.empty_like(psi)
        K.kss_apply_H(sysh, 0, psi, h)
        torch.cuda.synchronize()
        assert np.array_equal(out, h.cpu().numpy())
    finally:
        K.kss_sys_destroy(sysh)


def test_apply_edge_cases(ctx):
    import torch
    s = W.config1()
    sysh = setup(ctx, s)
    try:
        npw = K.kss_sphere(sysh, 0).shape[0]
        psi = torch.zeros((2, npw), dtype=torch.complex128, device="cuda")
        L = K.lib()
        assert L.kss_apply_H(sysh.h, 0, 0, None, None, npw, 0) == K.KSS_OK  # nb = 0: no-op
        assert L.kss_apply_H(sysh.h, 0, 2, psi.data_ptr(), psi.data_ptr(), npw, 0) == K.KSS_EINVAL
        assert L.kss_apply_H(sysh.h, 0, 2, psi.data_ptr(), psi.data_ptr(), npw - 1, 0) == K.KSS_EINVAL
        assert L.kss_apply_H(sysh.h, 3, 2, psi.data_ptr(), psi.data_ptr(), npw, 0) == K.KSS_EINVAL
        assert L.kss_apply_H(sysh.h, 0, -1, psi.data_ptr(), psi.data_ptr(), npw, 0) == K.KSS_EINVAL
        assert "out of range" in K.kss_last_error(ctx) or K.kss_last_error(ctx)
        # deterministic: two applications are bitwise identical
        c = torch.from_numpy(W.random_block(npw, 2, seed=8)).cuda()
        h1, h2 = torch.empty_like(c), torch.empty_like(c)
        K.kss_apply_H(sysh, 0, c, h1)
        K.kss_apply_H(sysh, 0, c, h2)
        torch.cuda.synchronize()
        assert torch.equal(h1, h2)
    finally:
        K.kss_sys_destroy(sysh)


def test_setup_rejects_bad_input(ctx):
    s = W.config1()
    with pytest.raises(K.KssError) as e:
        K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=(14, 24, 24))
    assert e.value.status == K.KSS_EINVAL  # box cannot hold the sphere (needs >= 15)
    with pytest.raises(K.KssError):
        K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D, fft_box=(29, 29, 29))  # not 2,3,5-smooth
    with pytest.raises(K.KssError):
        K.kss_setup(ctx, s.lattice, -1.0, s.kpts, s.pos, s.D)
    # non-finite host inputs are refused at setup, before anything reaches the device
    pos = np.array(s.pos, dtype=np.float64)
    pos[1, 2] = np.nan
    D = np.array(s.D, dtype=np.float64)
    D[3] = np.inf
    kp = np.array(s.kpts, dtype=np.float64)
    kp[0, 0] = np.nan
    for args in ((s.lattice, s.ecut, s.kpts, pos, s.D), (s.lattice, s.ecut, s.kpts, s.pos, D),
                 (s.lattice, s.ecut, kp, s.pos, s.D)):
        with pytest.raises(K.KssError) as e:
            K.kss_setup(ctx, *args)
        assert e.value.status == K.KSS_EINVAL and "non-finite" in str(e.value)


def test_stream_ordering_with_torch(ctx):
    """Work queued by torch and by the library on the same stream is ordered: an asynchronous
    pinned-host upload followed at once by kss_apply_H (no synchronisation in between), on the
    default stream and on a user stream."""
    import torch
    s = W.config1()
    p = O.build_problem(s, 0)
    c = W.random_block(p.basis.npw, 8, seed=21)
    ref = p.apply(c)
    host = torch.from_numpy(c).pin_memory()
    # default stream (the context's stream)
    sysh = setup(ctx, s)
    try:
        for _ in range(3):
            psi = torch.empty(host.shape, dtype=host.dtype, device="cuda")
            psi.copy_(host, non_blocking=True)
            out = torch.empty_like(psi)
            K.kss_apply_H(sysh, 0, psi, out)
            res = torch.empty(out.shape, dtype=out.dtype).pin_memory()
            res.copy_(out, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            assert rel_err_rows(res.numpy(), ref) < FP64_TOL
    finally:
        K.kss_sys_destroy(sysh)
    # a separate user stream with its own context
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        c2 = K.kss_create(0, st.cuda_stream)
        sys2 = setup(c2, s)
        try:
            psi = torch.empty(host.shape, dtype=host.dtype, device="cuda")
            psi.copy_(host, non_blocking=True)
            out = torch.empty_like(psi)
            K.kss_apply_H(sys2, 0, psi, out)
            res = torch.empty(out.shape, dtype=out.dtype).pin_memory()
            res.copy_(out, non_blocking=True)
            st.synchronize()
            assert rel_err_rows(res.numpy(), ref) < FP64_TOL
        finally:
            K.kss_sys_destroy(sys2)
            K.kss_destroy(c2)
