"""FP64 oracle: basis, local potential, projectors, dense H, naive-DFT H-apply, eigenpairs.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain NumPy/SciPy in float64 /
complex128; no blocking, fusion or reordering beyond the definitions written below.

Conventions (readings of the paper's plane-wave statement, §1 and §5.2):

* Lattice rows a1, a2, a3 (bohr).  Reciprocal rows b_i with a_i . b_j = 2 pi delta_ij,
  computed from the cross products in the fixed scalar order of ``reciprocal_lattice``.
* Basis at reduced k = kappa: Miller triples m with 0.5*|q|^2 <= Ecut, q = sum_i (m_i+kappa_i) b_i,
  each Cartesian component summed left to right and |q|^2 = (qx*qx + qy*qy) + qz*qz.  This
  inclusion test is the one piece of arithmetic both implementations must evaluate the same
  way, so that the G-sphere is reproduced bit for bit.
* Canonical order: ascending (m3, m2, m1), m1 fastest.  Box offset of m on an N1 x N2 x N3
  grid: (m1 mod N1) + N1*((m2 mod N2) + N2*(m3 mod N3)).
* Wavefunction blocks are band-major: array (nb, npw); row n holds the plane-wave
  coefficients of band n.
* Local potential: V(r) = A * sum_a sum_L exp(-|r - R_a - L|^2 / (2 sigma^2)) sampled at the
  grid points r_j = sum_i (j_i/N_i) a_i.  The operator is the grid operator
  <G|V|G'> = V_N(G - G'), V_N(dm) = N^-3 sum_j V(r_j) exp(-2 pi i sum_i dm_i j_i / N_i).
* Projectors: beta_{a,s}(G) = c_s exp(-alpha |q|^2) exp(-i q.R_a),
  beta_{a,x}(G) = c_p q_x exp(-alpha |q|^2) exp(-i q.R_a) (likewise y, z), with c_s, c_p the
  continuum unit-norm constants; H_nl = sum_i |beta_i> D_i <beta_i| (Eq. ham-nl, §5.2, with
  the diagonal h of norm-conserving pseudopotentials).
* Overlap (the generalised form, §5.2: the nonlocal part of the overlap operator has the same
  structure as Eq. ham-nl): S = 1 + sum_i |beta_i> q_i <beta_i| with diagonal q, and the
  eigenproblem H psi = lambda S psi, eigenvectors S-orthonormal.  q = None means S = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

TWO_PI = 2.0 * math.pi

# Terms of the periodic Gaussian sum farther than this many sigma are below 1e-20 * |A|.
GAUSS_CUT_SIGMAS = math.sqrt(2.0 * math.log(1e20))


# ---------------------------------------------------------------------------------------------
# Basis (plane-wave sphere), §1 / §5.2
# ---------------------------------------------------------------------------------------------

def reciprocal_lattice(lat: np.ndarray) -> Tuple[np.ndarray, float]:
    """Reciprocal rows b1, b2, b3 (a_i . b_j = 2 pi delta_ij) and the cell volume.

    Scalar formula in a fixed evaluation order: b_i = (2 pi / vol) * (a_j x a_k)."""
    a1x, a1y, a1z = (float(v) for v in lat[0])
    a2x, a2y, a2z = (float(v) for v in lat[1])
    a3x, a3y, a3z = (float(v) for v in lat[2])
    c23 = (a2y * a3z - a2z * a3y, a2z * a3x - a2x * a3z, a2x * a3y - a2y * a3x)
    c31 = (a3y * a1z - a3z * a1y, a3z * a1x - a3x * a1z, a3x * a1y - a3y * a1x)
    c12 = (a1y * a2z - a1z * a2y, a1z * a2x - a1x * a2z, a1x * a2y - a1y * a2x)
    vol = a1x * c23[0] + a1y * c23[1] + a1z * c23[2]
    f = TWO_PI / vol
    B = np.array([[f * c23[0], f * c23[1], f * c23[2]],
                  [f * c31[0], f * c31[1], f * c31[2]],
                  [f * c12[0], f * c12[1], f * c12[2]]], dtype=np.float64)
    return B, vol


def q_components(miller: np.ndarray, kred, B: np.ndarray):
    """Cartesian q = k + G for integer Miller rows, summed left to right without contraction."""
    m = miller.astype(np.float64)
    u1 = m[:, 0] + float(kred[0])
    u2 = m[:, 1] + float(kred[1])
    u3 = m[:, 2] + float(kred[2])
    qx = u1 * B[0, 0] + u2 * B[1, 0] + u3 * B[2, 0]
    qy = u1 * B[0, 1] + u2 * B[1, 1] + u3 * B[2, 1]
    qz = u1 * B[0, 2] + u2 * B[1, 2] + u3 * B[2, 2]
    return qx, qy, qz


def half_q2(qx, qy, qz):
    """0.5 * ((qx*qx + qy*qy) + qz*qz): the kinetic energy and the inclusion measure."""
    return 0.5 * ((qx * qx + qy * qy) + qz * qz)


@dataclass
class Basis:
    miller: np.ndarray  # (npw,3) int32 in canonical order
    kred: np.ndarray  # (3,)
    box: Tuple[int, int, int]
    offset: np.ndarray  # (npw,) int64 box offsets
    kinetic: np.ndarray  # (npw,) 0.5|k+G|^2
    q: np.ndarray  # (npw,3) Cartesian k+G

    @property
    def npw(self) -> int:
        return int(self.miller.shape[0])


def enumerate_sphere(lat: np.ndarray, ecut: float, kred) -> np.ndarray:
    """Brute-force G-sphere: test every Miller triple in a cube that surely holds the sphere,
    keep those with 0.5|k+G|^2 <= Ecut, and sort them into canonical (m3, m2, m1) order."""
    B, _ = reciprocal_lattice(lat)
    gmax = math.sqrt(2.0 * ecut)
    M = [int(math.ceil(gmax * float(np.linalg.norm(lat[i])) / TWO_PI + abs(float(kred[i])))) + 1
         for i in range(3)]
    r = [np.arange(-M[i], M[i] + 1) for i in range(3)]
    m1, m2, m3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    cand = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    qx, qy, qz = q_components(cand, kred, B)
    keep = half_q2(qx, qy, qz) <= ecut
    sel = cand[keep]
    order = np.lexsort((sel[:, 0], sel[:, 1], sel[:, 2]))
    return sel[order].astype(np.int32)


def is_smooth235(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def default_box(spheres: Sequence[np.ndarray]) -> Tuple[int, int, int]:
    """Smallest {2,3,5}-smooth N_i >= 4*max|m_i| + 1 over all spheres of a system (the
    no-aliasing size for products of two sphere functions)."""
    out = []
    for i in range(3):
        mm = max(int(np.abs(s[:, i]).max()) for s in spheres)
        n = 4 * mm + 1
        while not is_smooth235(n):
            n += 1
        out.append(n)
    return tuple(out)


def make_basis(lat: np.ndarray, ecut: float, kred, box: Tuple[int, int, int]) -> Basis:
    miller = enumerate_sphere(lat, ecut, kred)
    N1, N2, N3 = box
    for i, N in enumerate(box):
        if int(np.abs(miller[:, i]).max()) * 2 + 1 > N:
            raise ValueError("FFT box does not hold the sphere")
    m = miller.astype(np.int64)
    offset = (m[:, 0] % N1) + N1 * ((m[:, 1] % N2) + N2 * (m[:, 2] % N3))
    B, _ = reciprocal_lattice(lat)
    qx, qy, qz = q_components(miller, kred, B)
    return Basis(miller=miller, kred=np.asarray(kred, np.float64), box=tuple(box),
                 offset=offset, kinetic=half_q2(qx, qy, qz), q=np.stack([qx, qy, qz], 1))


# ---------------------------------------------------------------------------------------------
# Local potential on the grid
# ---------------------------------------------------------------------------------------------

def grid_points(lat: np.ndarray, box) -> np.ndarray:
    """Cartesian r_j = sum_i (j_i/N_i) a_i, array (N3, N2, N1, 3) indexed [j3, j2, j1]."""
    N1, N2, N3 = box
    j3, j2, j1 = np.meshgrid(np.arange(N3), np.arange(N2), np.arange(N1), indexing="ij")
    f = np.stack([j1 / N1, j2 / N2, j3 / N3], axis=-1)
    return f @ lat


def _image_range(lat: np.ndarray, reach: float):
    B, vol = reciprocal_lattice(lat)
    out = []
    for i in range(3):
        h = TWO_PI / float(np.linalg.norm(B[i]))  # distance between lattice planes
        out.append(int(math.ceil(reach / h)) + 1)
    return out


def vloc_grid(lat: np.ndarray, pos: np.ndarray, amp: float, sigma: float, box) -> np.ndarray:
    """V(r_j) = A sum_a sum_L exp(-|r_j - R_a - L|^2 / (2 sigma^2)) on the grid, (N3,N2,N1).

    Full periodic-image sum over a cube of lattice translations that covers every image
    within GAUSS_CUT_SIGMAS*sigma of any grid point (every omitted term is < 1e-20 |A|)."""
    r = grid_points(lat, box).reshape(-1, 3)
    n = _image_range(lat, GAUSS_CUT_SIGMAS * sigma)
    V = np.zeros(r.shape[0])
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    for R in pos:
        for n1 in range(-n[0], n[0] + 1):
            for n2 in range(-n[1], n[1] + 1):
                for n3 in range(-n[2], n[2] + 1):
                    L = n1 * lat[0] + n2 * lat[1] + n3 * lat[2]
                    d = r - (R + L)
                    V += np.exp(-(d * d).sum(axis=1) * inv2s2)
    N1, N2, N3 = box
    return (amp * V).reshape(N3, N2, N1)


def vloc_grid_orthorhombic(lat: np.ndarray, pos: np.ndarray, amp: float, sigma: float,
                           box) -> np.ndarray:
    """Same sum as ``vloc_grid`` for a diagonal lattice, using the identity
    exp(-|d|^2/2s^2) = prod_i exp(-d_i^2/2s^2) and the fact that, for a diagonal lattice, the
    image sum factorises per Cartesian axis.  Used for the large boxes."""
    if np.count_nonzero(lat - np.diag(np.diag(lat))):
        raise ValueError("lattice is not diagonal")
    N = box
    n = _image_range(lat, GAUSS_CUT_SIGMAS * sigma)
    inv2s2 = 1.0 / (2.0 * sigma * sigma)
    V = np.zeros((N[2], N[1], N[0]))
    for R in pos:
        f = []
        for i in range(3):
            a = float(lat[i, i])
            x = np.arange(N[i]) / N[i] * a
            s = np.zeros(N[i])
            for k in range(-n[i], n[i] + 1):
                d = x - (R[i] + k * a)
                s += np.exp(-d * d * inv2s2)
            f.append(s)
        V += f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    return amp * V


def vloc_for(sys_, box) -> np.ndarray:
    lat = sys_.lattice
    if np.count_nonzero(lat - np.diag(np.diag(lat))) == 0:
        return vloc_grid_orthorhombic(lat, sys_.pos, sys_.vloc_amp, sys_.vloc_sigma, box)
    return vloc_grid(lat, sys_.pos, sys_.vloc_amp, sys_.vloc_sigma, box)


def vloc_fourier_grid(V: np.ndarray) -> np.ndarray:
    """V_N(dm) = N^-3 sum_j V(r_j) e^{-2 pi i dm.j/N}, indexed [dm3 mod N3, dm2, dm1]."""
    return np.fft.fftn(V) / V.size


# ---------------------------------------------------------------------------------------------
# Projectors (Eq. ham-nl, §5.2)
# ---------------------------------------------------------------------------------------------

def projector_constants(alpha: float, vol: float) -> Tuple[float, float]:
    """c_s, c_p such that the continuum norms sum_G |beta|^2 -> 1 for both channels:
    Omega/(2pi)^3 * c_s^2 * int exp(-2 alpha q^2) d^3q = 1 and the q_x^2-weighted analogue."""
    cs = math.sqrt(TWO_PI ** 3 * (2.0 * alpha / math.pi) ** 1.5 / vol)
    cp = cs * math.sqrt(4.0 * alpha)
    return cs, cp


def projectors(lat: np.ndarray, basis: Basis, pos: np.ndarray, nproj_per_atom: int,
               alpha: float) -> np.ndarray:
    """Projector table beta, shape (npw, natom*nproj_per_atom); column 4a+l holds channel
    l in (s, px, py, pz) of atom a (column a when nproj_per_atom == 1: s only)."""
    _, vol = reciprocal_lattice(lat)
    cs, cp = projector_constants(alpha, vol)
    q = basis.q
    q2 = (q * q).sum(axis=1)
    g = np.exp(-alpha * q2)
    cols = []
    for R in pos:
        phase = np.exp(-1j * (q @ R))
        if nproj_per_atom >= 1:
            cols.append(cs * g * phase)
        if nproj_per_atom == 4:
            for ax in range(3):
                cols.append(cp * q[:, ax] * g * phase)
        elif nproj_per_atom not in (0, 1):
            raise ValueError("nproj_per_atom must be 0, 1 or 4")
    if not cols:
        return np.zeros((basis.npw, 0), np.complex128)
    return np.stack(cols, axis=1)


# ---------------------------------------------------------------------------------------------
# Hamiltonian: dense matrix and naive-DFT application
# ---------------------------------------------------------------------------------------------

def dense_hamiltonian(basis: Basis, V: np.ndarray, beta: np.ndarray, D: np.ndarray) -> np.ndarray:
    """H_{GG'} = delta_{GG'} T_G + V_N((m - m') mod N) + sum_i beta_i(G) D_i conj(beta_i(G'))."""
    VN = vloc_fourier_grid(V)
    m = basis.miller.astype(np.int64)
    N1, N2, N3 = basis.box
    d1 = (m[:, None, 0] - m[None, :, 0]) % N1
    d2 = (m[:, None, 1] - m[None, :, 1]) % N2
    d3 = (m[:, None, 2] - m[None, :, 2]) % N3
    H = VN[d3, d2, d1]
    H[np.diag_indices_from(H)] += basis.kinetic
    if beta.shape[1]:
        H += (beta * D[None, :]) @ beta.conj().T
    return H


def dense_hamiltonian_rowwise(basis: Basis, V: np.ndarray, beta: np.ndarray, D: np.ndarray,
                              block: int = 1024, order: str = "C") -> np.ndarray:
    """The same matrix as ``dense_hamiltonian``, filled one block of rows at a time, so that the
    index arrays never exceed block x npw (the config-2 matrix, 34181^2 complex128 = 18.7 GB,
    leaves no room for full-size index arrays).  order="F" allocates the result column-major,
    which LAPACK takes without a copy."""
    VN = vloc_fourier_grid(V)
    m = basis.miller.astype(np.int64)
    N1, N2, N3 = basis.box
    n = basis.npw
    H = np.empty((n, n), np.complex128, order=order)
    bD = beta * D[None, :] if beta.shape[1] else None
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        d1 = (m[r0:r1, None, 0] - m[None, :, 0]) % N1
        d2 = (m[r0:r1, None, 1] - m[None, :, 1]) % N2
        d3 = (m[r0:r1, None, 2] - m[None, :, 2]) % N3
        rows = VN[d3, d2, d1]
        idx = np.arange(r0, r1)
        rows[idx - r0, idx] += basis.kinetic[r0:r1]
        if bD is not None:
            rows += bD[r0:r1] @ beta.conj().T
        H[r0:r1, :] = rows
    return H


def _dft_matrix(N: int, sign: int) -> np.ndarray:
    """F[a, b] = exp(sign * 2 pi i * a*b / N), with the exponent reduced mod N first."""
    a = np.arange(N)
    return np.exp(sign * 2j * math.pi * ((a[:, None] * a[None, :]) % N) / N)


def scatter_to_box(c: np.ndarray, basis: Basis) -> np.ndarray:
    """Band-major (nb, npw) sphere coefficients -> (nb, N3, N2, N1) box, zero elsewhere."""
    N1, N2, N3 = basis.box
    box = np.zeros((c.shape[0], N3 * N2 * N1), np.complex128)
    box[:, basis.offset] = c
    return box.reshape(c.shape[0], N3, N2, N1)


def gather_from_box(box: np.ndarray, basis: Basis) -> np.ndarray:
    return box.reshape(box.shape[0], -1)[:, basis.offset]


def naive_inverse_dft(box: np.ndarray) -> np.ndarray:
    """psi(r_j) = sum_m B(m) e^{+2 pi i sum_i m_i j_i / N_i}: one dense DFT matrix per axis."""
    nb, N3, N2, N1 = box.shape
    x = np.einsum("ja,nzya->nzyj", _dft_matrix(N1, +1), box, optimize=True)
    x = np.einsum("ja,nzay->nzjy", _dft_matrix(N2, +1), x, optimize=True)
    x = np.einsum("ja,nayx->njyx", _dft_matrix(N3, +1), x, optimize=True)
    return x


def naive_forward_dft(f: np.ndarray) -> np.ndarray:
    """F(m) = N^-3 sum_j f(r_j) e^{-2 pi i sum_i m_i j_i / N_i}."""
    nb, N3, N2, N1 = f.shape
    x = np.einsum("ma,nzya->nzym", _dft_matrix(N1, -1), f, optimize=True)
    x = np.einsum("ma,nzay->nzmy", _dft_matrix(N2, -1), x, optimize=True)
    x = np.einsum("ma,nayx->nmyx", _dft_matrix(N3, -1), x, optimize=True)
    return x / (N1 * N2 * N3)


def apply_local_naive(c: np.ndarray, basis: Basis, V: np.ndarray) -> np.ndarray:
    """Local part by scatter -> inverse DFT -> x V(r) -> forward DFT -> gather."""
    box = scatter_to_box(c, basis)
    psi_r = naive_inverse_dft(box)
    psi_r *= V[None]
    return gather_from_box(naive_forward_dft(psi_r), basis)


def apply_nonlocal(c: np.ndarray, beta: np.ndarray, D: np.ndarray) -> np.ndarray:
    """sum_i beta_i D_i <beta_i|psi> for every band (Eq. ham-nl with diagonal h)."""
    if beta.shape[1] == 0:
        return np.zeros_like(c)
    cprj = c @ beta.conj()  # (nb, nproj): <beta_i|psi_n>
    return (cprj * D[None, :]) @ beta.T


def apply_h_naive(c: np.ndarray, basis: Basis, V: np.ndarray, beta: np.ndarray,
                  D: np.ndarray) -> np.ndarray:
    """H psi = T psi + (V psi via naive DFTs) + nonlocal, for a band-major block (nb, npw)."""
    c = np.asarray(c, np.complex128)
    return basis.kinetic[None, :] * c + apply_local_naive(c, basis, V) + apply_nonlocal(c, beta, D)


def dense_overlap(beta: np.ndarray, Q: Optional[np.ndarray]) -> np.ndarray:
    """S_{GG'} = delta_{GG'} + sum_i beta_i(G) q_i conj(beta_i(G'))."""
    S = np.eye(beta.shape[0], dtype=np.complex128)
    if Q is not None and beta.shape[1]:
        S += (beta * np.asarray(Q, np.float64)[None, :]) @ beta.conj().T
    return S


def apply_overlap(c: np.ndarray, beta: np.ndarray, Q: Optional[np.ndarray]) -> np.ndarray:
    """S psi = psi + sum_i beta_i q_i <beta_i|psi> for every band (band-major block)."""
    c = np.asarray(c, np.complex128)
    if Q is None or beta.shape[1] == 0:
        return c.copy()
    return c + apply_nonlocal(c, beta, np.asarray(Q, np.float64))


def density(c: np.ndarray, basis: Basis, occ, vol: float) -> np.ndarray:
    """n(r_j) = sum_n w_n |psi_n(r_j)|^2 on the grid, shape (N3, N2, N1) (Eq. nandtau, §2: w the
    occupancy times the k-point weight), with psi_n(r) = Omega^-1/2 sum_G c_n(G) e^{i(k+G).r}
    (the k phase drops out of the modulus)."""
    c = np.asarray(c, np.complex128)
    occ = np.asarray(occ, np.float64)
    psi_r = naive_inverse_dft(scatter_to_box(c, basis))
    return np.einsum("n,nzyx->zyx", occ, (psi_r * psi_r.conj()).real) / vol


def apply_h_dense(c: np.ndarray, H: np.ndarray) -> np.ndarray:
    return np.asarray(c, np.complex128) @ H.T


# ---------------------------------------------------------------------------------------------
# Eigenpairs and checks
# ---------------------------------------------------------------------------------------------

def lowest_eigenpairs(H: np.ndarray, nband: int):
    """Lowest nband eigenvalues (ascending) and eigenvectors (columns) of Hermitian H (LAPACK)."""
    w, v = scipy.linalg.eigh(H, subset_by_index=[0, nband - 1], driver="evr")
    return w, v


def lowest_generalized_eigenpairs(H: np.ndarray, S: np.ndarray, nband: int):
    """Lowest nband eigenpairs of H x = lambda S x (Hermitian H, Hermitian positive definite S;
    LAPACK): eigenvalues ascending, eigenvectors S-orthonormal columns."""
    w, v = scipy.linalg.eigh(H, S, subset_by_index=[0, nband - 1], driver="gvx")
    return w, v


def all_eigenvalues(H: np.ndarray) -> np.ndarray:
    return scipy.linalg.eigh(H, eigvals_only=True, driver="evd")


def count_below(H: np.ndarray, sigma: float) -> int:
    """Sylvester inertia: number of eigenvalues of H below sigma, from an LDL^H factorisation
    of H - sigma I (the count of negative eigenvalues of the block-diagonal factor)."""
    A = H - sigma * np.eye(H.shape[0])
    A[np.diag_indices_from(A)] = A.diagonal().real  # Hermitian: the diagonal is real
    _, d, _ = scipy.linalg.ldl(A, hermitian=True)
    return int((np.linalg.eigvalsh(d) < 0).sum())


@dataclass
class Problem:
    """Everything the oracle needs for one (system, k-point)."""
    basis: Basis
    V: np.ndarray
    beta: np.ndarray
    D: np.ndarray
    Q: Optional[np.ndarray] = None  # overlap coefficients (None: S = 1)

    def dense(self) -> np.ndarray:
        return dense_hamiltonian(self.basis, self.V, self.beta, self.D)

    def apply(self, c: np.ndarray) -> np.ndarray:
        return apply_h_naive(c, self.basis, self.V, self.beta, self.D)

    def dense_S(self) -> np.ndarray:
        return dense_overlap(self.beta, self.Q)

    def apply_S(self, c: np.ndarray) -> np.ndarray:
        return apply_overlap(c, self.beta, self.Q)

    def apply_filter_operator(self, c: np.ndarray) -> np.ndarray:
        """S^-1 H psi (H psi without an overlap): the operator whose polynomial the generalised
        Chebyshev filter applies; S^-1 through a dense linear solve."""
        h = self.apply(c)
        if self.Q is None:
            return h
        return np.linalg.solve(self.dense_S(), h.T).T

    def lowest(self, nband: int):
        """Lowest nband eigenpairs of H x = lambda S x (standard when Q is None)."""
        if self.Q is None:
            return lowest_eigenpairs(self.dense(), nband)
        return lowest_generalized_eigenpairs(self.dense(), self.dense_S(), nband)


def system_box(sys_) -> Tuple[int, int, int]:
    if sys_.fft_box is not None:
        return tuple(sys_.fft_box)
    spheres = [enumerate_sphere(sys_.lattice, sys_.ecut, k) for k in sys_.kpts]
    return default_box(spheres)


def build_problem(sys_, ik: int = 0, box=None, V: Optional[np.ndarray] = None) -> Problem:
    box = tuple(box) if box is not None else system_box(sys_)
    basis = make_basis(sys_.lattice, sys_.ecut, sys_.kpts[ik], box)
    if V is None:
        V = vloc_for(sys_, box)
    beta = projectors(sys_.lattice, basis, sys_.pos, sys_.nproj_per_atom, sys_.proj_alpha)
    D = np.asarray(sys_.D, np.float64)[: beta.shape[1]]
    Q = getattr(sys_, "Q", None)
    Q = None if Q is None else np.asarray(Q, np.float64)[: beta.shape[1]]
    return Problem(basis=basis, V=V, beta=beta, D=D, Q=Q)


def eigenvalue_error(evals: np.ndarray, ref: np.ndarray) -> float:
    """Max |lambda - lambda_ref| over the wanted bands, both sorted ascending."""
    a = np.sort(np.asarray(evals, np.float64))
    b = np.sort(np.asarray(ref, np.float64))[: a.size]
    return float(np.max(np.abs(a - b)))
