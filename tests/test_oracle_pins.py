"""Pins of the FP64 oracle against facts fixed by the mathematics, not by the oracle itself.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
index, a conjugated or transposed operand) fails at least one of them:

* sphere counts from exact integer arithmetic (basis, inclusion test, k shift);
* free-electron spectrum 0.5|k+G|^2 (kinetic term, no spurious V or projector part);
* constant potential shifts every eigenvalue by exactly v0 (V_N(0) normalisation);
* one s projector: eigenvalues are the roots of the rank-one secular equation (nonlocal sign,
  D placement, |beta|^2 weights);
* Hermiticity of the naive-DFT apply and agreement with the dense matrix (DFT signs, V_N index
  direction, beta vs conj(beta));
* naive DFT round trip and Parseval (normalisation of the two transforms);
* translation of all atoms by a grid vector leaves the spectrum unchanged (relative sign of the
  V_loc centres and the projector phase e^{-iq.R});
* axis permutation of the atom sites in a cubic cell leaves the Gamma spectrum unchanged
  (p-channel axis assignment);
* V_N at low |G| equals the analytic Fourier series of the periodic Gaussian (amplitude, width,
  image sum, structure-factor sign);
* projector norms tend to 1 and s/p channels are orthogonal (normalisation constants);
* Sylvester inertia count equals the number of eigenvalues below a shift.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def exact_count(a, ecut, kred):
    """Number of Miller triples with |m+kappa|^2 <= 2 Ecut (a/2pi)^2 for a cubic cell, using
    integer arithmetic on 4(m+kappa) (kappa is a multiple of 1/4 in every config here)."""
    R2 = 2.0 * ecut * (a / (2 * math.pi)) ** 2
    lim16 = math.floor(16 * R2)
    assert abs(16 * R2 - round(16 * R2)) > 1e-6  # not on a boundary
    k4 = [int(round(4 * k)) for k in kred]
    M = int(math.isqrt(int(R2))) + 2
    n = 0
    for m1 in range(-M, M + 1):
        for m2 in range(-M, M + 1):
            s12 = (4 * m1 + k4[0]) ** 2 + (4 * m2 + k4[1]) ** 2
            if s12 > lim16:
                continue
            for m3 in range(-M, M + 1):
                if s12 + (4 * m3 + k4[2]) ** 2 <= lim16:
                    n += 1
    return n


def test_reciprocal_lattice_general():
    rng = np.random.default_rng(3)
    lat = np.eye(3) * 7 + rng.uniform(-1, 1, (3, 3))
    B, vol = O.reciprocal_lattice(lat)
    assert np.allclose(lat @ B.T, 2 * math.pi * np.eye(3), atol=1e-13)
    assert abs(vol - np.linalg.det(lat)) < 1e-10


@pytest.mark.parametrize("a,ecut,kred,expect", [
    (10.0, 10.0, (0, 0, 0), 1503),
    (20.0, 20.0, (0.25, 0.25, 0.25), 34181),
    (20.0, 20.0, (0.25, -0.25, 0.25), 34181),
    (8.0, 12.0, (0.25, 0.25, -0.25), None),
    (16.0, 20.0, (0, 0, 0), None),
])
def test_sphere_count_exact(a, ecut, kred, expect):
    miller = O.enumerate_sphere(W.cubic(a), ecut, kred)
    n = exact_count(a, ecut, kred)
    assert miller.shape[0] == n
    if expect is not None:
        assert n == expect


def test_sphere_order_and_offsets():
    s = W.config1()
    b = O.make_basis(s.lattice, s.ecut, s.kpts[0], (24, 24, 24))
    m = b.miller
    key = (m[:, 2].astype(np.int64) * 1000 + m[:, 1]) * 1000 + m[:, 0]
    assert np.all(np.diff(key) > 0)  # strictly ascending (m3, m2, m1)
    assert np.unique(b.offset).size == b.npw
    assert b.offset.min() >= 0 and b.offset.max() < 24 ** 3
    # offsets decode back to the Miller triples modulo N
    o = b.offset
    assert np.array_equal(o % 24, m[:, 0] % 24)
    assert np.array_equal((o // 24) % 24, m[:, 1] % 24)
    assert np.array_equal(o // 576, m[:, 2] % 24)


def test_default_box_rule():
    assert O.is_smooth235(96) and O.is_smooth235(25) and not O.is_smooth235(29)
    s = W.make_system("x", 10.0, 10.0, 1, 4, seed=1)  # max |m| = 7 -> 29 -> 30
    assert O.system_box(s) == (30, 30, 30)


def free_electron_levels(a, ecut, kred):
    """Sorted 0.5 (2pi/a)^2 |m+kappa|^2 over the exact-integer sphere (cubic cell)."""
    R2 = 2.0 * ecut * (a / (2 * math.pi)) ** 2
    M = int(math.isqrt(int(R2))) + 2
    r = np.arange(-M, M + 1)
    m1, m2, m3 = np.meshgrid(r, r, r, indexing="ij")
    s = (m1 + kred[0]) ** 2 + (m2 + kred[1]) ** 2 + (m3 + kred[2]) ** 2
    s = np.sort(s[s <= R2].ravel())
    return 0.5 * (2 * math.pi / a) ** 2 * s


@pytest.mark.parametrize("kred", [(0, 0, 0), (0.25, -0.25, 0.25)])
def test_free_electron(kred):
    s = W.tiny_system(a=7.0, ecut=3.0, natom=2, kpts=[kred], vloc_amp=0.0, nproj_per_atom=0)
    p = O.build_problem(s, 0, box=(16, 16, 16))
    assert np.all(p.V == 0.0)
    w = O.all_eigenvalues(p.dense())
    ref = free_electron_levels(7.0, 3.0, kred)
    assert w.size == ref.size
    assert np.max(np.abs(w - ref)) < 1e-12
    c = W.random_block(p.basis.npw, 3, seed=11)
    assert np.allclose(p.apply(c), c * ref_order_kinetic(p), atol=1e-12)


def ref_order_kinetic(p):
    k = p.basis.kred
    m = p.basis.miller + k
    return 0.5 * (2 * math.pi / 7.0) ** 2 * (m ** 2).sum(1)


def test_constant_potential_shift():
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2)
    p = O.build_problem(s, 0, box=(15, 15, 15))
    v0 = -0.8125
    p0 = O.Problem(p.basis, np.zeros_like(p.V), p.beta, p.D)
    p1 = O.Problem(p.basis, np.full_like(p.V, v0), p.beta, p.D)
    w0 = O.all_eigenvalues(p0.dense())
    w1 = O.all_eigenvalues(p1.dense())
    assert np.max(np.abs(w1 - w0 - v0)) < 1e-12


def secular_roots(t, w, D):
    """All eigenvalues of diag(t) + D b b^H from the rank-one secular equation
    1 + D sum_s w_s/(t_s - e) = 0 over distinct shells t_s with weights w_s = sum |b|^2
    (Golub 1973), plus the g_s - 1 unperturbed copies in every shell of multiplicity g_s."""
    order = np.argsort(t)
    t = t[order]
    w = w[order]
    shells, mult, wt = [], [], []
    for ti, wi in zip(t, w):
        if shells and abs(ti - shells[-1]) < 1e-10:
            mult[-1] += 1
            wt[-1] += wi
        else:
            shells.append(ti)
            mult.append(1)
            wt.append(wi)
    ts = np.array(shells)
    ws = np.array(wt)

    def f(e):
        return 1.0 + D * np.sum(ws / (ts - e))

    def bisect(lo, hi):
        flo = f(lo)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if (fm > 0) == (flo > 0):
                lo, flo = mid, fm
            else:
                hi = mid
        return 0.5 * (lo + hi)

    roots = []
    tot = float(ws.sum())
    eps = 1e-13
    if D > 0:
        for i in range(len(ts) - 1):
            roots.append(bisect(ts[i] + eps, ts[i + 1] - eps))
        roots.append(bisect(ts[-1] + eps, ts[-1] + D * tot + 1.0))
    else:
        roots.append(bisect(ts[0] + D * tot - 1.0, ts[0] - eps))
        for i in range(len(ts) - 1):
            roots.append(bisect(ts[i] + eps, ts[i + 1] - eps))
    for ti, g in zip(ts, mult):
        roots.extend([ti] * (g - 1))
    return np.sort(np.array(roots))


@pytest.mark.parametrize("D", [0.7, -0.45])
def test_rank_one_secular_equation(D):
    s = W.tiny_system(a=6.0, ecut=2.0, natom=1, vloc_amp=0.0, nproj_per_atom=1)
    s.D[:] = D
    p = O.build_problem(s, 0, box=(15, 15, 15))
    b = p.beta[:, 0]
    w_dense = O.all_eigenvalues(p.dense())
    roots = secular_roots(p.basis.kinetic.copy(), np.abs(b) ** 2, D)
    assert roots.size == w_dense.size
    assert np.max(np.abs(roots - w_dense)) < 1e-10


@pytest.fixture(scope="module")
def tiny_problem():
    s = W.tiny_system(a=6.5, ecut=2.5, natom=3, kpts=[(0.25, 0.25, -0.25)])
    return O.build_problem(s, 0, box=(16, 15, 18))


def test_hermiticity_naive_apply(tiny_problem):
    p = tiny_problem
    phi = W.random_block(p.basis.npw, 1, seed=1)[0]
    psi = W.random_block(p.basis.npw, 1, seed=2)[0]
    hpsi = p.apply(psi[None])[0]
    hphi = p.apply(phi[None])[0]
    lhs = np.vdot(phi, hpsi)
    rhs = np.conj(np.vdot(psi, hphi))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_naive_apply_matches_dense(tiny_problem):
    p = tiny_problem
    c = W.random_block(p.basis.npw, 4, seed=5)
    a = p.apply(c)
    b = O.apply_h_dense(c, p.dense())
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
    H = p.dense()
    assert np.max(np.abs(H - H.conj().T)) < 1e-14


def test_dft_roundtrip_and_parseval(tiny_problem):
    p = tiny_problem
    c = W.random_block(p.basis.npw, 2, seed=9)
    box = O.scatter_to_box(c, p.basis)
    r = O.naive_inverse_dft(box)
    back = O.gather_from_box(O.naive_forward_dft(r), p.basis)
    assert np.max(np.abs(back - c)) < 1e-13
    n = np.prod(p.basis.box)
    assert np.allclose((np.abs(r) ** 2).sum(axis=(1, 2, 3)) / n, (np.abs(c) ** 2).sum(1), rtol=1e-13)
    # the inverse transform is the library inverse FFT up to the N^3 normalisation
    assert np.allclose(r, np.fft.ifftn(box, axes=(1, 2, 3)) * n, atol=1e-12)


def test_time_reversal():
    k = (0.25, -0.25, 0.25)
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2, kpts=[k, tuple(-x for x in k)])
    w = [O.all_eigenvalues(O.build_problem(s, ik, box=(15, 15, 15)).dense()) for ik in (0, 1)]
    assert np.max(np.abs(w[0] - w[1])) < 1e-11


def test_translation_by_grid_vector():
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2, kpts=[(0.25, 0.25, 0.25)])
    box = (15, 15, 15)
    w0 = O.all_eigenvalues(O.build_problem(s, 0, box=box).dense())
    t = np.array([2 * 6.0 / 15, -3 * 6.0 / 15, 6.0 / 15])
    s2 = W.with_(s, pos=s.pos + t)
    w1 = O.all_eigenvalues(O.build_problem(s2, 0, box=box).dense())
    assert np.max(np.abs(w0 - w1)) < 1e-11

    # Power of this pin: plant a flipped projector phase (centres at -R while V sits at +R);
    # the planted operator is not translation invariant.
    def planted(sys_):
        p = O.build_problem(sys_, 0, box=box)
        beta = O.projectors(sys_.lattice, p.basis, -sys_.pos, 4, sys_.proj_alpha)
        return O.all_eigenvalues(O.Problem(p.basis, p.V, beta, p.D).dense())

    assert np.max(np.abs(planted(s) - planted(s2))) > 1e-6


def test_axis_permutation_cubic_gamma():
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2)
    box = (15, 15, 15)
    w0 = O.all_eigenvalues(O.build_problem(s, 0, box=box).dense())
    perm = [1, 2, 0]
    D2 = s.D.reshape(-1, 4)[:, [0, 1 + perm[0], 1 + perm[1], 1 + perm[2]]].ravel()
    s2 = W.with_(s, pos=s.pos[:, perm], D=D2)
    w1 = O.all_eigenvalues(O.build_problem(s2, 0, box=box).dense())
    assert np.max(np.abs(w0 - w1)) < 1e-11


def test_vloc_continuum_fourier_series():
    a = 8.0
    s = W.make_system("v", a, 4.0, 3, 4, seed=21)
    box = (48, 48, 48)
    V = O.vloc_for(s, box)
    VN = O.vloc_fourier_grid(V)
    _, vol = O.reciprocal_lattice(s.lattice)
    sig = s.vloc_sigma
    for m in [(0, 0, 0), (1, 0, 0), (0, -2, 1), (3, 1, -2), (-4, 2, 2)]:
        G = 2 * math.pi / a * np.array(m, float)
        ana = (s.vloc_amp * (2 * math.pi * sig ** 2) ** 1.5 / vol
               * math.exp(-0.5 * sig ** 2 * G @ G) * np.exp(-1j * (s.pos @ G)).sum())
        got = VN[m[2] % 48, m[1] % 48, m[0] % 48]
        assert abs(got - ana) < 1e-12, (m, got, ana)


def test_vloc_two_forms_agree():
    s = W.make_system("v", 7.0, 4.0, 3, 4, seed=22)
    box = (12, 14, 15)
    a = O.vloc_grid(s.lattice, s.pos, s.vloc_amp, s.vloc_sigma, box)
    b = O.vloc_grid_orthorhombic(s.lattice, s.pos, s.vloc_amp, s.vloc_sigma, box)
    assert np.max(np.abs(a - b)) < 1e-13


def test_projector_norms_and_orthogonality():
    s = W.make_system("p", 8.0, 40.0, 1, 4, seed=23)
    b = O.make_basis(s.lattice, s.ecut, (0, 0, 0), (64, 64, 64))
    beta = O.projectors(s.lattice, b, s.pos, 4, s.proj_alpha)
    S = beta.conj().T @ beta
    assert np.allclose(np.diag(S).real, 1.0, atol=1e-10)
    assert np.max(np.abs(S - np.diag(np.diag(S)))) < 1e-12


def test_inertia_count():
    s = W.tiny_system(a=6.0, ecut=2.0, natom=2)
    H = O.build_problem(s, 0, box=(15, 15, 15)).dense()
    w = O.all_eigenvalues(H)
    for k in (0, 5, 17, w.size - 3):
        sigma = 0.5 * (w[k] + w[k + 1]) if k + 1 < w.size else w[-1] + 1
        assert O.count_below(H, sigma) == k + 1


# ---------------------------------------------------------------------------------------------
# Generalised form: H x = lambda S x with S = 1 + sum_i |beta_i> q_i <beta_i| (§5.2: the overlap's
# nonlocal part has the structure of Eq. ham-nl)
# ---------------------------------------------------------------------------------------------

def gen_secular_roots(t, w, q):
    """All eigenvalues of diag(t) x = lambda (1 + q b b^H) x (t > 0, 1 + q |b|^2 > 0).  With
    s = b^H x != 0: (t - lambda) x = lambda q b s gives the secular equation
    1 = lambda q sum_s w_s / (t_s - lambda) over distinct shells t_s (weights w_s = sum |b|^2);
    a shell of multiplicity g_s keeps g_s - 1 eigenvalues at t_s.  For q > 0 one root lies in
    (0, t_1) and one in each (t_i, t_i+1); for q < 0 one in each (t_i, t_i+1) and one above the
    last shell."""
    order = np.argsort(t)
    t, w = t[order], w[order]
    shells, mult, wt = [], [], []
    for ti, wi in zip(t, w):
        if shells and abs(ti - shells[-1]) < 1e-10:
            mult[-1] += 1
            wt[-1] += wi
        else:
            shells.append(ti)
            mult.append(1)
            wt.append(wi)
    ts, ws = np.array(shells), np.array(wt)

    def f(e):
        return 1.0 - e * q * np.sum(ws / (ts - e))

    def bisect(lo, hi):
        flo = f(lo)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if (fm > 0) == (flo > 0):
                lo, flo = mid, fm
            else:
                hi = mid
        return 0.5 * (lo + hi)

    eps = 1e-13
    roots = [bisect(ts[i] + eps, ts[i + 1] - eps) for i in range(len(ts) - 1)]
    if q > 0:
        roots.append(bisect(eps, ts[0] - eps))
    else:
        hi = ts[-1] + 1.0
        while f(hi) < 0:  # f -> 1 + q sum w > 0 as e -> infinity
            hi = ts[-1] + 2.0 * (hi - ts[-1])
        roots.append(bisect(ts[-1] + eps, hi))
    for ti, g in zip(ts, mult):
        roots.extend([ti] * (g - 1))
    return np.sort(np.array(roots))


@pytest.mark.parametrize("q", [0.8, -0.3])
def test_generalized_rank_one_secular_equation(q):
    s = W.tiny_system(a=6.0, ecut=2.0, natom=1, vloc_amp=0.0, nproj_per_atom=1,
                      kpts=[(0.25, 0.25, 0.25)])
    s.D[:] = 0.0
    s = W.with_(s, Q=np.array([q]))
    p = O.build_problem(s, 0, box=(15, 15, 15))
    b = p.beta[:, 0]
    assert 1.0 + q * np.sum(np.abs(b) ** 2) > 0.1
    w_gen = O.lowest_generalized_eigenpairs(p.dense(), p.dense_S(), p.basis.npw)[0]
    roots = gen_secular_roots(p.basis.kinetic.copy(), np.abs(b) ** 2, q)
    assert roots.size == w_gen.size
    assert np.max(np.abs(roots - w_gen)) < 1e-10
    # the pin discriminates: a flipped overlap sign (a plausible slip) is far off
    wrong = O.lowest_generalized_eigenpairs(p.dense(), O.dense_overlap(p.beta, -p.Q), p.basis.npw)[0]
    assert np.max(np.abs(roots - wrong)) > 1e-3


@pytest.fixture(scope="module")
def tiny_overlap_problem():
    s = W.with_overlap(W.tiny_system(a=6.5, ecut=2.5, natom=3, kpts=[(0.25, 0.25, -0.25)]), qmax=0.6)
    return O.build_problem(s, 0, box=(16, 15, 18))


def test_overlap_apply_matches_dense_and_is_spd(tiny_overlap_problem):
    p = tiny_overlap_problem
    S = p.dense_S()
    assert np.max(np.abs(S - S.conj().T)) < 1e-15
    np.linalg.cholesky(S)  # positive definite
    c = W.random_block(p.basis.npw, 3, seed=12)
    assert np.max(np.abs(p.apply_S(c) - c @ S.T)) < 1e-13
    # q = 0 gives S = 1, and no overlap gives the standard problem
    p0 = O.Problem(p.basis, p.V, p.beta, p.D, None)
    assert np.array_equal(p0.dense_S(), np.eye(p.basis.npw))
    assert np.array_equal(p0.apply_S(c), c)


def test_generalized_eigenpairs_invariants(tiny_overlap_problem):
    p = tiny_overlap_problem
    n = 12
    w, v = p.lowest(n)
    H, S = p.dense(), p.dense_S()
    assert np.max(np.abs(H @ v - (S @ v) * w[None, :])) < 1e-11
    assert np.max(np.abs(v.conj().T @ S @ v - np.eye(n))) < 1e-12
    # textbook reduction with the Cholesky factor S = L L^H: eig(L^-1 H L^-H) are the same values
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    w_red = np.linalg.eigvalsh(Li @ H @ Li.conj().T)[:n]
    assert np.max(np.abs(w_red - w)) < 1e-11
    # S >= 1 (q >= 0) only shrinks Rayleigh quotients towards 0, so by Courant-Fischer
    # min(l_k, 0) <= l_k(gen) <= max(l_k, 0) for the standard eigenvalue l_k of the same index
    ws = O.lowest_eigenpairs(H, n)[0]
    assert np.all(w <= np.maximum(ws, 0.0) + 1e-12) and np.all(w >= np.minimum(ws, 0.0) - 1e-12)
    assert np.any(np.abs(w - ws) > 1e-3)  # and the overlap does change them


# ---------------------------------------------------------------------------------------------
# Density after the solve: n(r) = sum w |psi(r)|^2 (Eq. nandtau, §2)
# ---------------------------------------------------------------------------------------------

def test_density_integral_is_the_occupation(tiny_problem):
    p = tiny_problem
    c = W.random_block(p.basis.npw, 3, seed=31)
    occ = np.array([2.0, 1.0, 0.5])
    _, vol = O.reciprocal_lattice(W.tiny_system(a=6.5, ecut=2.5, natom=3).lattice)
    n = O.density(c, p.basis, occ, vol)
    assert np.all(n >= 0)
    integral = n.sum() * vol / np.prod(p.basis.box)
    assert abs(integral - float(occ @ (np.abs(c) ** 2).sum(axis=1))) < 1e-11 * integral


def test_density_plane_waves_closed_form(tiny_problem):
    p = tiny_problem
    npw = p.basis.npw
    lat = W.tiny_system(a=6.5, ecut=2.5, natom=3).lattice
    _, vol = O.reciprocal_lattice(lat)
    # one plane wave: uniform density w / Omega
    c1 = np.zeros((1, npw), np.complex128)
    c1[0, 7] = 1.0
    n1 = O.density(c1, p.basis, [3.0], vol)
    assert np.max(np.abs(n1 - 3.0 / vol)) < 1e-13
    # two plane waves a e^{iG1.r} + b e^{iG2.r}: (|a|^2 + |b|^2 + 2 Re(a conj(b) e^{i(G1-G2).r})) / Omega
    i1, i2 = 3, 40
    a, b = 0.6 - 0.2j, -0.3 + 0.7j
    c2 = np.zeros((1, npw), np.complex128)
    c2[0, i1], c2[0, i2] = a, b
    N1, N2, N3 = p.basis.box
    j3, j2, j1 = np.meshgrid(np.arange(N3), np.arange(N2), np.arange(N1), indexing="ij")
    dm = p.basis.miller[i1].astype(float) - p.basis.miller[i2].astype(float)
    phase = 2 * np.pi * (dm[0] * j1 / N1 + dm[1] * j2 / N2 + dm[2] * j3 / N3)
    expect = (abs(a) ** 2 + abs(b) ** 2 + 2 * np.real(a * np.conj(b) * np.exp(1j * phase))) / vol
    n2 = O.density(c2, p.basis, [1.0], vol)
    assert np.max(np.abs(n2 - expect)) < 1e-13
    # discriminates a sign slip in the transform direction: conj(phase) differs
    wrong = (abs(a) ** 2 + abs(b) ** 2 + 2 * np.real(a * np.conj(b) * np.exp(-1j * phase))) / vol
    assert np.max(np.abs(n2 - wrong)) > 1e-3


def test_density_time_reversal():
    """k -> -k with c(-G) = conj(c(G)) gives the same density (psi_-k = conj(psi_k))."""
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2, kpts=[(0.25, 0.25, -0.25), (-0.25, -0.25, 0.25)])
    box = (15, 15, 15)
    b0 = O.make_basis(s.lattice, s.ecut, s.kpts[0], box)
    b1 = O.make_basis(s.lattice, s.ecut, s.kpts[1], box)
    c0 = W.random_block(b0.npw, 2, seed=33)
    idx = {tuple(m): i for i, m in enumerate(b1.miller)}
    c1 = np.zeros((2, b1.npw), np.complex128)
    for i, m in enumerate(b0.miller):
        c1[:, idx[tuple(-m)]] = np.conj(c0[:, i])
    _, vol = O.reciprocal_lattice(s.lattice)
    n0 = O.density(c0, b0, [1.0, 2.0], vol)
    n1 = O.density(c1, b1, [1.0, 2.0], vol)
    assert np.max(np.abs(n0 - n1)) < 1e-13 * np.max(n0)


# ---------------------------------------------------------------------------------------------
# Stored values (tests/golden/, written by tests/golden/make_golden.py from the oracle only)
# ---------------------------------------------------------------------------------------------

def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    return np.array([float(l) for l in open(path) if l.strip() and not l.startswith("#")])


def test_golden_values_reproduce():
    w, _ = O.build_problem(W.config1(), 0).lowest(16)
    assert np.max(np.abs(w - _golden("c1_lowest16_Ha.txt"))) < 1e-12
    w3, _ = O.build_problem(W.config3(), 0).lowest(1024)
    assert np.max(np.abs(w3 - _golden("c3_lowest1024_Ha.txt"))) < 1e-12
    ws, _ = O.build_problem(W.config1s(), 0).lowest(16)
    assert np.max(np.abs(ws - _golden("c1s_lowest16_Ha.txt"))) < 1e-12
    counts = _golden("sphere_counts.txt").astype(int)
    assert counts[0] == 1503 and np.all(counts[1:] == 34181)


def test_pins_catch_planted_mistakes():
    """The power of the pins above, shown on the CPU: each plausible slip, planted in a copy of an
    oracle problem, moves the quantity its pin fixes far outside that pin's tolerance."""
    from dataclasses import replace

    # (1) kinetic energy at -k instead of +k: the free-electron levels at a shifted k move
    kred = (0.25, -0.25, 0.25)
    s = W.tiny_system(a=7.0, ecut=3.0, natom=2, kpts=[kred], vloc_amp=0.0, nproj_per_atom=0)
    p = O.build_problem(s, 0, box=(16, 16, 16))
    m = p.basis.miller - np.asarray(kred)
    wrong_t = 0.5 * (2 * math.pi / 7.0) ** 2 * (m ** 2).sum(1)
    bad = replace(p, basis=replace(p.basis, kinetic=wrong_t))
    ref = free_electron_levels(7.0, 3.0, kred)
    assert np.max(np.abs(O.all_eigenvalues(bad.dense()) - ref)) > 1e-2

    # (2) nonlocal sign flipped: the rank-one secular roots no longer match
    s = W.tiny_system(a=6.0, ecut=2.0, natom=1, vloc_amp=0.0, nproj_per_atom=1)
    s.D[:] = 0.7
    p = O.build_problem(s, 0, box=(15, 15, 15))
    roots = secular_roots(p.basis.kinetic.copy(), np.abs(p.beta[:, 0]) ** 2, 0.7)
    bad = replace(p, D=-p.D)
    assert np.max(np.abs(O.all_eigenvalues(bad.dense()) - roots)) > 1e-3

    # (3) potential offset by the mean (a dropped V_N(0) term): the constant-shift pin fails
    s = W.tiny_system(a=6.0, ecut=2.5, natom=2)
    p = O.build_problem(s, 0, box=(15, 15, 15))
    v0 = -0.8125
    w0 = O.all_eigenvalues(replace(p, V=np.zeros_like(p.V)).dense())
    w1 = O.all_eigenvalues(replace(p, V=np.full_like(p.V, v0) - v0).dense())
    assert np.max(np.abs(w1 - w0 - v0)) > 0.5

    # (4) projector table conjugated in the dense matrix only: the naive apply and the dense
    # matrix (the two independent forms) disagree
    s = W.tiny_system(a=6.5, ecut=2.5, natom=3, kpts=[(0.25, 0.25, -0.25)])
    p = O.build_problem(s, 0, box=(16, 15, 18))
    c = W.random_block(p.basis.npw, 2, seed=4)
    good = p.apply(c)
    bad_dense = replace(p, beta=np.conj(p.beta)).dense()
    assert np.max(np.abs(c @ bad_dense.T - good)) > 1e-3 * np.max(np.abs(good))


# ---------------------------------------------------------------------------------------------
# Sheared (triclinic) cells: the general image sum of V and the projector phases, pinned by
# closed forms that hold on any lattice
# ---------------------------------------------------------------------------------------------

TRICLINIC = np.array([[9.0, 0.0, 0.0], [1.65, 9.45, 0.0], [-1.05, 1.35, 9.9]])
FLAT_SHEAR = np.array([[6.0, 0.0, 0.0], [5.5, 1.5, 0.0], [0.0, 0.0, 6.0]])


def _vloc_series(lat, pos, amp, sig, m):
    """Continuum Fourier coefficient of the periodic Gaussian sum at G = m . B:
    A (2 pi sigma^2)^{3/2} / Omega exp(-sigma^2 |G|^2 / 2) sum_a exp(-i G . R_a)."""
    B, vol = O.reciprocal_lattice(lat)
    G = np.asarray(m, float) @ B
    return (amp * (2 * math.pi * sig ** 2) ** 1.5 / vol * math.exp(-0.5 * sig ** 2 * G @ G)
            * np.exp(-1j * (pos @ G)).sum())


@pytest.mark.parametrize("lat", [TRICLINIC, FLAT_SHEAR], ids=["triclinic", "flat_shear"])
def test_vloc_continuum_series_sheared_cell(lat):
    """On a sheared cell the grid DFT of V equals the continuum Fourier series of the periodic
    Gaussian sum (aliasing below 1e-14 on these boxes): fixes the grid points r_j = sum (j_i/N_i) a_i,
    the image sum and G . R for a non-diagonal lattice."""
    rng = np.random.default_rng(31)
    pos = rng.random((3, 3)) @ lat
    box = (36, 36, 40) if lat is TRICLINIC else (32, 12, 32)
    V = O.vloc_grid(lat, pos, -2.0, 1.0, box)
    VN = O.vloc_fourier_grid(V)
    for m in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, -1), (1, -1, 2), (-2, 1, 1), (3, 0, -1)]:
        got = VN[m[2] % box[2], m[1] % box[1], m[0] % box[0]]
        ana = _vloc_series(lat, pos, -2.0, 1.0, m)
        assert abs(got - ana) < 1e-12, (m, got, ana)


@pytest.mark.parametrize("lat", [TRICLINIC, FLAT_SHEAR], ids=["triclinic", "flat_shear"])
def test_vloc_translation_by_grid_vector_sheared_cell(lat):
    """Moving every atom by a grid vector t = sum (s_i/N_i) a_i rolls V on the grid by s exactly
    (to rounding): the full periodic image sum is translation covariant, a truncated one is not."""
    rng = np.random.default_rng(32)
    pos = rng.random((2, 3)) @ lat
    box = (20, 18, 24)
    s = np.array([7, -5, 11])
    t = (s / np.array(box)) @ lat
    V0 = O.vloc_grid(lat, pos, -2.0, 1.0, box)
    V1 = O.vloc_grid(lat, pos + t, -2.0, 1.0, box)
    assert np.max(np.abs(V1 - np.roll(V0, shift=(s[2], s[1], s[0]), axis=(0, 1, 2)))) < 1e-13


def _images_covering(lat, reach):
    """Image counts n_i such that every lattice vector within `reach` of the origin has
    |n_i| <= n_i: the spacing of the lattice planes is 1/|column i of lat^-1|."""
    inv = np.linalg.inv(lat)
    return [int(math.ceil(reach * float(np.linalg.norm(inv[:, i])))) + 1 for i in range(3)]


def _projector_overlap_closed_form(lat, d, alpha):
    """sum_G c_s^2 exp(-2 alpha |G|^2) exp(i G . d) = sum_L exp(-|d + L|^2 / (8 alpha)) (Poisson
    summation at Gamma with the continuum unit-norm constant c_s)."""
    reach = math.sqrt(8 * alpha * 50.0) + float(np.linalg.norm(d))
    n = _images_covering(lat, reach)
    tot = 0.0
    for n1 in range(-n[0], n[0] + 1):
        for n2 in range(-n[1], n[1] + 1):
            for n3 in range(-n[2], n[2] + 1):
                L = n1 * lat[0] + n2 * lat[1] + n3 * lat[2]
                x = d + L
                tot += math.exp(-(x @ x) / (8 * alpha))
    return tot


@pytest.mark.parametrize("lat", [TRICLINIC, FLAT_SHEAR], ids=["triclinic", "flat_shear"])
def test_projectors_sheared_cell_closed_form(lat):
    """s-projectors of two atoms on a sheared cell at Gamma: <beta_a|beta_b> and |beta_a|^2 equal
    the periodic Gaussian of the separation in closed form (cutoff tail e^-40).  On the large
    triclinic cell the image terms are negligible and the norm is the continuum value 1; on the
    flat cell (lattice planes 1.5 bohr apart) the images carry O(1) weight, so the pin also fixes
    the reciprocal vectors, the phases e^{-iq.R} and c_s on a skew lattice."""
    pos = np.array([[1.0, 2.0, 0.5], [3.1, 0.4, 2.2]]) @ np.diag([1.0, 0.5 if lat is FLAT_SHEAR else 1.0, 1.0])
    spheres = [O.enumerate_sphere(lat, 40.0, (0, 0, 0))]
    b = O.make_basis(lat, 40.0, (0, 0, 0), O.default_box(spheres))
    beta = O.projectors(lat, b, pos, 4, 0.25)
    S = beta.conj().T @ beta
    norm = _projector_overlap_closed_form(lat, np.zeros(3), 0.25)
    if lat is TRICLINIC:
        assert abs(norm - 1.0) < 1e-12
    for i in (0, 4):
        assert abs(S[i, i] - norm) < 1e-10
    ana = _projector_overlap_closed_form(lat, pos[0] - pos[1], 0.25)
    assert 1e-3 < ana
    assert abs(S[0, 4] - ana) < 1e-10, (S[0, 4], ana)


def test_sheared_cell_pins_catch_planted_mistakes():
    """Each plausible skew-lattice slip, planted in a copy of the oracle's arithmetic, fails the
    pin above that covers it by a wide margin."""
    # (5) grid points built with the transposed lattice: the continuum series pin fails
    lat = TRICLINIC
    rng = np.random.default_rng(31)
    pos = rng.random((3, 3)) @ lat
    box = (36, 36, 40)

    def vloc_transposed(lat_, pos_, box_):
        N1, N2, N3 = box_
        j3, j2, j1 = np.meshgrid(np.arange(N3), np.arange(N2), np.arange(N1), indexing="ij")
        f = np.stack([j1 / N1, j2 / N2, j3 / N3], axis=-1)
        r = (f @ lat_.T).reshape(-1, 3)
        n = _images_covering(lat_, O.GAUSS_CUT_SIGMAS + float(np.abs(lat_).sum()))
        V = np.zeros(r.shape[0])
        for R in pos_:
            for n1 in range(-n[0], n[0] + 1):
                for n2 in range(-n[1], n[1] + 1):
                    for n3 in range(-n[2], n[2] + 1):
                        d = r - (R + n1 * lat_[0] + n2 * lat_[1] + n3 * lat_[2])
                        V += np.exp(-(d * d).sum(axis=1) * 0.5)
        return (-2.0 * V).reshape(N3, N2, N1)

    VN = O.vloc_fourier_grid(vloc_transposed(lat, pos, box))
    m = (1, -1, 2)
    got = VN[m[2] % box[2], m[1] % box[1], m[0] % box[0]]
    assert abs(got - _vloc_series(lat, pos, -2.0, 1.0, m)) > 1e-4

    # (6) image range from the lengths of the lattice vectors instead of the spacing of the
    # lattice planes: on a flat sheared cell images are missing and translation covariance fails
    lat = FLAT_SHEAR

    def vloc_short_images(lat_, pos_, box_):
        r = O.grid_points(lat_, box_).reshape(-1, 3)
        n = [int(math.ceil(O.GAUSS_CUT_SIGMAS / float(np.linalg.norm(lat_[i])))) + 1 for i in range(3)]
        V = np.zeros(r.shape[0])
        for R in pos_:
            for n1 in range(-n[0], n[0] + 1):
                for n2 in range(-n[1], n[1] + 1):
                    for n3 in range(-n[2], n[2] + 1):
                        d = r - (R + n1 * lat_[0] + n2 * lat_[1] + n3 * lat_[2])
                        V += np.exp(-(d * d).sum(axis=1) * 0.5)
        N1, N2, N3 = box_
        return (-2.0 * V).reshape(N3, N2, N1)

    rng = np.random.default_rng(32)
    pos = rng.random((2, 3)) @ lat
    box = (20, 18, 24)
    s = np.array([7, -5, 11])
    t = (s / np.array(box)) @ lat
    V0 = vloc_short_images(lat, pos, box)
    V1 = vloc_short_images(lat, pos + t, box)
    assert np.max(np.abs(V1 - np.roll(V0, shift=(s[2], s[1], s[0]), axis=(0, 1, 2)))) > 1e-7  # pin: 1e-13

    # (7) projector phases with the transposed reciprocal lattice: the two-atom closed form on the
    # flat sheared cell fails
    lat = FLAT_SHEAR
    pos = np.array([[1.0, 1.0, 0.5], [3.1, 0.2, 2.2]])
    b = O.make_basis(lat, 40.0, (0, 0, 0), O.default_box([O.enumerate_sphere(lat, 40.0, (0, 0, 0))]))
    B, _ = O.reciprocal_lattice(lat)
    qbad = b.miller.astype(float) @ B.T
    bad = replace_basis_q(b, qbad)
    beta = O.projectors(lat, bad, pos, 1, 0.25)
    S = beta.conj().T @ beta
    assert abs(S[0, 1] - _projector_overlap_closed_form(lat, pos[0] - pos[1], 0.25)) > 1e-3


def replace_basis_q(b, q):
    from dataclasses import replace
    return replace(b, q=q)


def test_stored_c2_spectrum_against_lanczos_on_the_naive_apply():
    """The stored config-2 spectrum (LAPACK on the dense 34181^2 matrix, an hour of CPU) against an
    independent route through the oracle: Lanczos (ARPACK) on the naive-DFT H-apply, which never
    forms the matrix, for the lowest two eigenvalues."""
    import scipy.sparse.linalg as sla
    p = O.build_problem(W.config2(), 0)
    n = p.basis.npw
    op = sla.LinearOperator((n, n), matvec=lambda x: p.apply(np.asarray(x).reshape(1, -1))[0],
                            dtype=np.complex128)
    w = np.sort(sla.eigsh(op, k=2, which="SA", tol=1e-11, return_eigenvectors=False,
                          v0=np.ones(n, complex)))
    ref = _golden("c2_k0_lowest576_Ha.txt")
    assert ref.size == 576 and np.all(np.diff(ref) >= 0)
    assert np.max(np.abs(w - ref[:2])) < 1e-10
