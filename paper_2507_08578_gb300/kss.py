"""ctypes binding of ``libkss.so`` (include/kss.h): argument marshalling only.

Every function keeps the name of its C entry point.  Device buffers are passed as torch CUDA
tensors (their ``data_ptr()``); torch is used for device memory and streams only, all work runs
in the library's kernels.  There is no CPU fallback: if the library or a CUDA device is missing
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_longlong, c_size_t, c_uint64, c_void_p
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkss.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "kss.h")

KSS_OK, KSS_EINVAL, KSS_ENOMEM, KSS_ECUDA, KSS_ENOCONV, KSS_ETIMEOUT, KSS_EBUSY, KSS_ENUMERIC, KSS_ENOTSUP = range(9)
STATUS_NAMES = ["KSS_OK", "KSS_EINVAL", "KSS_ENOMEM", "KSS_ECUDA", "KSS_ENOCONV", "KSS_ETIMEOUT",
                "KSS_EBUSY", "KSS_ENUMERIC", "KSS_ENOTSUP"]
KSS_PREC_FP64, KSS_PREC_MIXED = 0, 1


class KssError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class kss_cell(ctypes.Structure):
    _fields_ = [("lattice", c_double * 9), ("ecut", c_double), ("nk", c_int),
                ("kpts_red", POINTER(c_double)), ("fft_box", c_int * 3)]


class kss_atoms(ctypes.Structure):
    _fields_ = [("natom", c_int), ("pos_cart", POINTER(c_double)), ("vloc_amp", c_double),
                ("vloc_sigma", c_double), ("nproj_per_atom", c_int), ("proj_alpha", c_double),
                ("D", POINTER(c_double)), ("Q", POINTER(c_double))]


class kss_sys_info(ctypes.Structure):
    _fields_ = [("nk", c_int), ("fft_box", c_int * 3), ("nproj", c_int), ("npw_max", c_int),
                ("volume", c_double), ("vloc_max", c_double)]


class kss_solve_opts(ctypes.Structure):
    _fields_ = [("degree", c_int), ("tol", c_double), ("max_iter", c_int), ("nbuffer", c_int),
                ("prec", c_int), ("seed", c_uint64), ("x0", c_void_p), ("x0_nb", c_int),
                ("x0_ld", c_int), ("flags", c_int)]


class kss_server_stats(ctypes.Structure):
    _fields_ = [("completed", c_longlong), ("rejected", c_longlong), ("warm_hits", c_longlong),
                ("p50_ms", c_double), ("p99_ms", c_double), ("mean_ms", c_double),
                ("solves_per_s", c_double), ("peak_bytes", c_size_t), ("in_flight_bytes", c_size_t)]


class kss_solve_stats(ctypes.Structure):
    _fields_ = [("iters", c_int), ("napply", c_longlong), ("max_resid", c_double),
                ("ms_filter", c_double), ("ms_rr", c_double), ("ms_total", c_double),
                ("nb", c_int)]


_lib = None


class kss_tune_entry(ctypes.Structure):
    _fields_ = [("device", c_int), ("precision", c_int), ("N1", c_int), ("N", c_int),
                ("W3", c_int), ("W2", c_int), ("A", c_int), ("B", c_int), ("threads", c_int),
                ("ms", c_double), ("ncand", c_int)]


def lib() -> ctypes.CDLL:
    """Load libkss.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in signatures().items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
        _lib = L
    return _lib


def signatures() -> dict:
    """ctypes prototype (argument types, result type) of every C entry point."""
    P = c_void_p
    return {
        "kss_version": ([], c_int),
        "kss_create": ([POINTER(c_void_p), c_int, c_void_p], c_int),
        "kss_destroy": ([P], c_int),
        "kss_last_error": ([P], c_char_p),
        "kss_setup": ([P, POINTER(kss_cell), POINTER(kss_atoms), POINTER(c_void_p)], c_int),
        "kss_sys_destroy": ([P], c_int),
        "kss_sys_info_get": ([P, POINTER(kss_sys_info)], c_int),
        "kss_sphere": ([P, c_int, POINTER(c_int), POINTER(POINTER(c_int32))], c_int),
        "kss_sphere_host": ([P, c_double, P, c_int, POINTER(c_int), P], c_int),
        "kss_default_box": ([P, c_double, c_int, P, P], c_int),
        "kss_get_maps": ([P, c_int, P, P], c_int),
        "kss_get_tables": ([P, c_int, P, P, P], c_int),
        "kss_upper_bound": ([P, c_int, POINTER(c_double)], c_int),
        "kss_footprint": ([P, c_int, c_int, POINTER(c_size_t)], c_int),
        "kss_apply_H": ([P, c_int, c_int, P, P, c_int, c_int], c_int),
        "kss_cheb_step": ([P, c_int, c_int, P, P, P, c_int, c_double, c_double, c_double, c_int], c_int),
        "kss_apply_H_host": ([P, c_int, c_int, P, P, c_int, c_int], c_int),
        "kss_apply_H_noalloc": ([P, c_int, c_int, P, P, c_int, c_int], c_int),
        "kss_solver_create": ([P, c_int, c_int, POINTER(kss_solve_opts), POINTER(c_void_p)], c_int),
        "kss_solver_destroy": ([P], c_int),
        "kss_solver_step": ([P, POINTER(c_int)], c_int),
        "kss_solver_step_many": ([c_int, POINTER(P), POINTER(c_int)], c_int),
        "kss_solver_results": ([P, P, P, P, c_int, POINTER(kss_solve_stats)], c_int),
        "kss_chebfi_solve": ([P, c_int, c_int, POINTER(kss_solve_opts), P, P, c_int, P,
                              POINTER(kss_solve_stats)], c_int),
        "kss_dense_hegv": ([P, c_int, P, P, P, P, P, P, P, c_int], c_int),
        "kss_dense_hegv_phase_ms": ([P, P], c_int),
        "kss_autotune_gemm_count": ([P], c_int),
        "kss_autotune_gemm_get": ([c_int, P], c_int),
        "kss_autotune_gemm_put": ([P], c_int),
        "kss_gemm": ([P, c_int, c_int, c_int, c_int, P, c_int, P, c_int, P, c_int, c_double,
                      c_double, c_double, c_double, c_int], c_int),
        "kss_selftest_bounded_wait": ([P, c_double], c_int),
        "kss_peak_probe": ([P, c_int, POINTER(c_double)], c_int),
        "kss_solve_batch": ([P, c_int, P, P, P, POINTER(kss_solve_opts), P, P, P], c_int),
        "kss_server_start": ([P, c_size_t, c_int, POINTER(kss_solve_opts)], c_int),
        "kss_server_submit": ([P, POINTER(kss_cell), POINTER(kss_atoms), c_int, POINTER(c_uint64)], c_int),
        "kss_server_pump": ([P, c_double, POINTER(c_int), POINTER(c_int)], c_int),
        "kss_server_poll": ([P, c_uint64, POINTER(c_int), P, P, POINTER(c_double)], c_int),
        "kss_server_get_stats": ([P, POINTER(kss_server_stats)], c_int),
        "kss_server_stop": ([P], c_int),
        "kss_profile_enable": ([P, c_int], c_int),
        "kss_profile_count": ([P, POINTER(c_int), POINTER(c_longlong)], c_int),
        "kss_profile_entry": ([P, c_int, POINTER(c_char_p), POINTER(c_longlong), POINTER(c_double)], c_int),
        "kss_apply_S": ([P, c_int, c_int, P, P, c_int, c_int], c_int),
        "kss_apply_H_gamma": ([P, c_int, c_int, P, P, c_int, c_int], c_int),
        "kss_density_accumulate": ([P, c_int, c_int, P, c_int, P, P, c_int], c_int),
        "kss_lobpcg_solve": ([P, c_int, c_int, POINTER(kss_solve_opts), P, P, c_int, P,
                              POINTER(kss_solve_stats)], c_int),
        "kss_rmmdiis_solve": ([P, c_int, c_int, POINTER(kss_solve_opts), P, P, c_int, P,
                               POINTER(kss_solve_stats)], c_int),
        "kss_autotune_set": ([P, c_int], c_int),
        "kss_autotune_count": ([POINTER(c_int)], c_int),
        "kss_autotune_get": ([c_int, POINTER(kss_tune_entry)], c_int),
        "kss_autotune_put": ([POINTER(kss_tune_entry)], c_int),
        "kss_autotune_clear": ([], c_int),
    }


def header_functions(path: str = HEADER):
    """Names of every function the C header declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kss_[a-zA-Z0-9_]+)\s*\(", txt)) - {"kss_status"})


# --------------------------------------------------------------------------------------------
# marshalling helpers

def _ptr(t) -> int:
    """Device address of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _block_dims(t, prec):
    import torch
    want = torch.complex128 if prec == KSS_PREC_FP64 else torch.complex64
    if t.dtype != want:
        raise ValueError(f"expected {want} for precision {prec}, got {t.dtype}")
    if t.dim() != 2:
        raise ValueError("band blocks are 2-D tensors (nb, ld)")
    return int(t.shape[0]), int(t.shape[1])


def _check(st: int, handle_ctx=None):
    if st != KSS_OK:
        msg = ""
        if handle_ctx is not None:
            m = lib().kss_last_error(handle_ctx)
            msg = m.decode() if m else ""
        raise KssError(st, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


# --------------------------------------------------------------------------------------------
# context and systems

def kss_version() -> int:
    return lib().kss_version()


def kss_create(device: int = 0, stream: Optional[int] = None):
    h = c_void_p()
    st = lib().kss_create(byref(h), int(device), c_void_p(stream) if stream else None)
    if st != KSS_OK:
        raise KssError(st, "kss_create failed (no usable CUDA device?)")
    return h


def kss_destroy(ctx):
    _check(lib().kss_destroy(ctx), ctx)


def kss_last_error(ctx) -> str:
    m = lib().kss_last_error(ctx)
    return m.decode() if m else ""


class System:
    """A kss_sys handle plus the context it belongs to (for error messages)."""

    def __init__(self, ctx, handle, keep):
        self.ctx = ctx
        self.h = handle
        self._keep = keep

    def __int__(self):
        return self.h.value


def kss_setup(ctx, lattice, ecut, kpts, pos, D, fft_box=(0, 0, 0), vloc_amp=-2.0,
              vloc_sigma=1.0, nproj_per_atom=4, proj_alpha=0.25, Q=None) -> System:
    """Q: optional overlap coefficients (one per projector): the generalised problem with
    S = 1 + sum_i |beta_i> q_i <beta_i|."""
    lat = np.ascontiguousarray(np.asarray(lattice, np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(kpts, np.float64).reshape(-1, 3))
    p = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1, 3))
    d = np.ascontiguousarray(np.asarray(D if D is not None else [], np.float64).reshape(-1))
    cell = kss_cell()
    cell.lattice[:] = lat.tolist()
    cell.ecut = float(ecut)
    cell.nk = int(k.shape[0])
    cell.kpts_red = _dptr(k)
    cell.fft_box[:] = [int(v) for v in (fft_box or (0, 0, 0))]
    at = kss_atoms()
    at.natom = int(p.shape[0])
    at.pos_cart = _dptr(p)
    at.vloc_amp = float(vloc_amp)
    at.vloc_sigma = float(vloc_sigma)
    at.nproj_per_atom = int(nproj_per_atom)
    at.proj_alpha = float(proj_alpha)
    at.D = _dptr(d)
    q = None
    if Q is not None:
        q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(-1))
        at.Q = _dptr(q)
    h = c_void_p()
    _check(lib().kss_setup(ctx, byref(cell), byref(at), byref(h)), ctx)
    return System(ctx, h, (k, p, d, q))


def kss_sys_destroy(sys: System):
    _check(lib().kss_sys_destroy(sys.h), sys.ctx)


def kss_sys_info_get(sys: System) -> dict:
    info = kss_sys_info()
    _check(lib().kss_sys_info_get(sys.h, byref(info)), sys.ctx)
    return {"nk": info.nk, "fft_box": tuple(info.fft_box), "nproj": info.nproj,
            "npw_max": info.npw_max, "volume": info.volume, "vloc_max": info.vloc_max}


def kss_sphere(sys: System, ik: int) -> np.ndarray:
    n = c_int()
    mp = POINTER(c_int32)()
    _check(lib().kss_sphere(sys.h, ik, byref(n), byref(mp)), sys.ctx)
    return np.ctypeslib.as_array(mp, shape=(n.value * 3,)).reshape(n.value, 3).copy()


def kss_sphere_host(lattice, ecut: float, kred) -> np.ndarray:
    """G-sphere of one k-point from the library's host code alone (no context, no device):
    Miller triples (npw, 3) in canonical order."""
    lat = np.ascontiguousarray(np.asarray(lattice, np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(kred, np.float64).reshape(3))
    n = c_int()
    _check(lib().kss_sphere_host(lat.ctypes.data, float(ecut), k.ctypes.data, 0, byref(n), None))
    m = np.zeros((n.value, 3), np.int32)
    _check(lib().kss_sphere_host(lat.ctypes.data, float(ecut), k.ctypes.data, n.value, byref(n),
                                 m.ctypes.data))
    return m


def kss_default_box(lattice, ecut: float, kpts) -> tuple:
    """The FFT box kss_setup picks when the cell gives none (host code only)."""
    lat = np.ascontiguousarray(np.asarray(lattice, np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(kpts, np.float64).reshape(-1, 3))
    box = np.zeros(3, np.int32)
    _check(lib().kss_default_box(lat.ctypes.data, float(ecut), int(k.shape[0]), k.ctypes.data,
                                 box.ctypes.data))
    return tuple(int(v) for v in box)


def kss_get_maps(sys: System, ik: int):
    npw = kss_sphere(sys, ik).shape[0]
    miller = np.zeros((npw, 3), np.int32)
    off = np.zeros(npw, np.int32)
    _check(lib().kss_get_maps(sys.h, ik, miller.ctypes.data, off.ctypes.data), sys.ctx)
    return miller, off


def kss_get_tables(sys: System, ik: int):
    info = kss_sys_info_get(sys)
    npw = kss_sphere(sys, ik).shape[0]
    N1, N2, N3 = info["fft_box"]
    V = np.zeros(N1 * N2 * N3)
    kin = np.zeros(npw)
    beta = np.zeros((info["nproj"], npw), np.complex128)
    _check(lib().kss_get_tables(sys.h, ik, V.ctypes.data, kin.ctypes.data,
                                beta.ctypes.data if info["nproj"] else None), sys.ctx)
    return V.reshape(N3, N2, N1), kin, beta


def kss_upper_bound(sys: System, ik: int) -> float:
    b = c_double()
    _check(lib().kss_upper_bound(sys.h, ik, byref(b)), sys.ctx)
    return b.value


def kss_footprint(sys: System, nband: int, prec: int = KSS_PREC_FP64) -> int:
    b = c_size_t()
    _check(lib().kss_footprint(sys.h, nband, prec, byref(b)), sys.ctx)
    return b.value


# --------------------------------------------------------------------------------------------
# H application

def kss_apply_H(sys: System, ik: int, psi, hpsi, prec: int = KSS_PREC_FP64, nb: Optional[int] = None):
    n, ld = _block_dims(psi, prec)
    n2, ld2 = _block_dims(hpsi, prec)
    if (n2, ld2) != (n, ld):
        raise ValueError("psi and hpsi shapes differ")
    _check(lib().kss_apply_H(sys.h, ik, n if nb is None else nb, _ptr(psi), _ptr(hpsi), ld, prec), sys.ctx)


def kss_apply_H_gamma(sys: System, ik: int, psi, hpsi, prec: int = KSS_PREC_FP64):
    """H psi for real-space-real bands at Gamma (two bands per complex FFT)."""
    n, ld = _block_dims(psi, prec)
    n2, ld2 = _block_dims(hpsi, prec)
    if (n2, ld2) != (n, ld):
        raise ValueError("psi and hpsi shapes differ")
    _check(lib().kss_apply_H_gamma(sys.h, ik, n, _ptr(psi), _ptr(hpsi), ld, prec), sys.ctx)


def kss_apply_S(sys: System, ik: int, psi, spsi, prec: int = KSS_PREC_FP64):
    """spsi = S psi (the overlap of a system set up with Q; a copy of psi without one)."""
    n, ld = _block_dims(psi, prec)
    n2, ld2 = _block_dims(spsi, prec)
    if (n2, ld2) != (n, ld):
        raise ValueError("psi and spsi shapes differ")
    _check(lib().kss_apply_S(sys.h, ik, n, _ptr(psi), _ptr(spsi), ld, prec), sys.ctx)


def kss_density_accumulate(sys: System, ik: int, psi, occ, rho, prec: int = KSS_PREC_FP64):
    """rho (device float64 tensor, N3 x N2 x N1) += sum_n occ[n] |psi_n(r)|^2."""
    n, ld = _block_dims(psi, prec)
    o = np.ascontiguousarray(np.asarray(occ, np.float64).reshape(-1))
    if o.size != n:
        raise ValueError("one occupation per band")
    _check(lib().kss_density_accumulate(sys.h, ik, n, _ptr(psi), ld, o.ctypes.data, _ptr(rho), prec), sys.ctx)


def kss_apply_H_noalloc(sys: System, ik: int, psi, hpsi, prec: int = KSS_PREC_FP64):
    """kss_apply_H without any device allocation (static scratch, see include/kss.h)."""
    n, ld = _block_dims(psi, prec)
    n2, ld2 = _block_dims(hpsi, prec)
    if (n2, ld2) != (n, ld):
        raise ValueError("psi and hpsi shapes differ")
    _check(lib().kss_apply_H_noalloc(sys.h, ik, n, _ptr(psi), _ptr(hpsi), ld, prec), sys.ctx)


def kss_cheb_step(sys: System, ik: int, psi, psi_prev, out, alpha, beta, gamma,
                  prec: int = KSS_PREC_FP64):
    n, ld = _block_dims(psi, prec)
    _check(lib().kss_cheb_step(sys.h, ik, n, _ptr(psi), _ptr(psi_prev), _ptr(out), ld,
                               float(alpha), float(beta), float(gamma), prec), sys.ctx)


def kss_apply_H_host(sys: System, ik: int, psi: np.ndarray, hpsi: np.ndarray,
                     prec: int = KSS_PREC_FP64):
    want = np.complex128 if prec == KSS_PREC_FP64 else np.complex64
    if psi.dtype != want or hpsi.dtype != want or psi.shape != hpsi.shape or psi.ndim != 2:
        raise ValueError("psi/hpsi must be 2-D arrays of the precision's complex type")
    if not (psi.flags.c_contiguous and hpsi.flags.c_contiguous):
        raise ValueError("contiguous arrays required")
    nb, ld = psi.shape
    _check(lib().kss_apply_H_host(sys.h, ik, nb, psi.ctypes.data, hpsi.ctypes.data, ld, prec), sys.ctx)


# --------------------------------------------------------------------------------------------
# eigensolver

KSS_SOLVE_NO_GAMMA_REAL = 1
KSS_SOLVE_BATCH_NO_GRAPH = 2
KSS_SOLVE_BATCH_FP32_PROJ = 4


def make_opts(degree=10, tol=0.0, max_iter=0, nbuffer=-1, prec=KSS_PREC_FP64, seed=1234,
              x0=None, x0_nb=0, x0_ld=0, flags=0) -> kss_solve_opts:
    o = kss_solve_opts()
    o.degree = int(degree)
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.nbuffer = int(nbuffer)
    o.prec = int(prec)
    o.seed = int(seed)
    o.x0 = _ptr(x0)
    o.x0_nb = int(x0_nb)
    o.x0_ld = int(x0_ld)
    o.flags = int(flags)
    return o


class Solver:
    def __init__(self, sys, handle, nband, prec):
        self.sys = sys
        self.h = handle
        self.nband = nband
        self.prec = prec


def kss_solver_create(sys: System, ik: int, nband: int, opts: kss_solve_opts) -> Solver:
    h = c_void_p()
    _check(lib().kss_solver_create(sys.h, ik, nband, byref(opts), byref(h)), sys.ctx)
    return Solver(sys, h, nband, opts.prec)


def kss_solver_destroy(s: Solver):
    _check(lib().kss_solver_destroy(s.h), s.sys.ctx)


def kss_solver_step(s: Solver) -> bool:
    c = c_int()
    _check(lib().kss_solver_step(s.h, byref(c)), s.sys.ctx)
    return bool(c.value)


def kss_solver_step_many(solvers) -> list:
    """One iteration of every solver (same context), the Rayleigh-Ritz of one overlapping the
    filter of the next; returns the converged flags."""
    solvers = list(solvers)
    n = len(solvers)
    if n == 0:
        return []
    hs = (c_void_p * n)(*[sv.h.value for sv in solvers])
    flags = (c_int * n)()
    _check(lib().kss_solver_step_many(n, hs, flags), solvers[0].sys.ctx)
    return [bool(f) for f in flags]


def kss_solver_results(s: Solver, evecs=None):
    ev = np.zeros(s.nband)
    rs = np.zeros(s.nband)
    stats = kss_solve_stats()
    ld = 0
    if evecs is not None:
        _, ld = _block_dims(evecs, s.prec)
    _check(lib().kss_solver_results(s.h, ev.ctypes.data, rs.ctypes.data, _ptr(evecs), ld,
                                    byref(stats)), s.sys.ctx)
    return ev, rs, stats_dict(stats)


def stats_dict(st: kss_solve_stats) -> dict:
    return {k: getattr(st, k) for k, _ in kss_solve_stats._fields_}


def kss_chebfi_solve(sys: System, ik: int, nband: int, opts: kss_solve_opts, evecs=None,
                     allow_noconv: bool = False):
    ev = np.zeros(nband)
    rs = np.zeros(nband)
    stats = kss_solve_stats()
    ld = 0
    if evecs is not None:
        _, ld = _block_dims(evecs, opts.prec)
    st = lib().kss_chebfi_solve(sys.h, ik, nband, byref(opts), ev.ctypes.data, _ptr(evecs), ld,
                                rs.ctypes.data, byref(stats))
    if st == KSS_ENOCONV and allow_noconv:
        return ev, rs, stats_dict(stats), st
    _check(st, sys.ctx)
    return ev, rs, stats_dict(stats), st


def kss_lobpcg_solve(sys: System, ik: int, nband: int, opts: kss_solve_opts, evecs=None,
                     allow_noconv: bool = False):
    ev = np.zeros(nband)
    rs = np.zeros(nband)
    stats = kss_solve_stats()
    ld = 0
    if evecs is not None:
        _, ld = _block_dims(evecs, opts.prec)
    st = lib().kss_lobpcg_solve(sys.h, ik, nband, byref(opts), ev.ctypes.data, _ptr(evecs), ld,
                                rs.ctypes.data, byref(stats))
    if st == KSS_ENOCONV and allow_noconv:
        return ev, rs, stats_dict(stats), st
    _check(st, sys.ctx)
    return ev, rs, stats_dict(stats), st


def kss_rmmdiis_solve(sys: System, ik: int, nband: int, opts: kss_solve_opts, evecs=None,
                     allow_noconv: bool = False):
    ev = np.zeros(nband)
    rs = np.zeros(nband)
    stats = kss_solve_stats()
    ld = 0
    if evecs is not None:
        _, ld = _block_dims(evecs, opts.prec)
    st = lib().kss_rmmdiis_solve(sys.h, ik, nband, byref(opts), ev.ctypes.data, _ptr(evecs), ld,
                                rs.ctypes.data, byref(stats))
    if st == KSS_ENOCONV and allow_noconv:
        return ev, rs, stats_dict(stats), st
    _check(st, sys.ctx)
    return ev, rs, stats_dict(stats), st


# --------------------------------------------------------------------------------------------
# launch accounting / per-kernel timing

def kss_profile_enable(ctx, enable: bool = True):
    _check(lib().kss_profile_enable(ctx, 1 if enable else 0), ctx)


def kss_profile_count(ctx):
    n = c_int()
    l = c_longlong()
    _check(lib().kss_profile_count(ctx, byref(n), byref(l)), ctx)
    return n.value, l.value


def kss_profile_entry(ctx, i: int):
    name = c_char_p()
    l = c_longlong()
    ms = c_double()
    _check(lib().kss_profile_entry(ctx, i, byref(name), byref(l), byref(ms)), ctx)
    return name.value.decode(), l.value, ms.value


def profile_table(ctx) -> dict:
    """{kernel name: (launches, total_ms)} since the last kss_profile_enable."""
    n, _ = kss_profile_count(ctx)
    out = {}
    for i in range(n):
        name, l, ms = kss_profile_entry(ctx, i)
        if l:
            out[name] = (l, ms)
    return out


# --------------------------------------------------------------------------------------------
# autotuner of the FFT pass-B schedule

def kss_autotune_set(ctx, mode: int):
    _check(lib().kss_autotune_set(ctx, int(mode)), ctx)


def kss_autotune_put(device: int, precision: int, N1: int, N: int, W3: int, A: int, B: int,
                     threads: int):
    e = kss_tune_entry(device=device, precision=precision, N1=N1, N=N, W3=W3, W2=0, A=A, B=B,
                       threads=threads, ms=0.0, ncand=0)
    _check(lib().kss_autotune_put(byref(e)))


def kss_autotune_clear():
    _check(lib().kss_autotune_clear())


def kss_autotune_table() -> list:
    """Every table entry as a dict (kss_autotune_count / kss_autotune_get)."""
    n = c_int()
    _check(lib().kss_autotune_count(byref(n)))
    out = []
    for i in range(n.value):
        e = kss_tune_entry()
        _check(lib().kss_autotune_get(i, byref(e)))
        out.append({k: getattr(e, k) for k, _ in kss_tune_entry._fields_})
    return out


def kss_gemm(ctx, op: int, A, B, C, alpha=1.0, beta=0.0, prec: int = KSS_PREC_FP64):
    """op 0: C = alpha A^H B + beta C; op 1: C = alpha A B + beta C.  Matrices are torch tensors
    holding column-major matrices as (ncols, ld) row-major arrays (one column per row)."""
    ka, lda = int(A.shape[0]), int(A.shape[1])
    kb, ldb = int(B.shape[0]), int(B.shape[1])
    n, ldc = int(C.shape[0]), int(C.shape[1])
    if op == 0:
        M, K = ka, lda
    else:
        K, M = ka, lda
    _check(lib().kss_gemm(ctx, op, M, n, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc,
                          complex(alpha).real, complex(alpha).imag, complex(beta).real,
                          complex(beta).imag, prec), ctx)


def kss_dense_hegv(ctx, As, Bs, ws, real: bool = False):
    """FP64 generalised Hermitian eigensolves A x = lambda B x of several pencils (torch complex128
    device tensors holding column-major matrices as (n, ld) arrays, one column per row; ws: float64
    device tensors of n entries).  Returns the host info array."""
    count = len(As)
    n = (c_int * count)(*[int(a.shape[0]) for a in As])
    lda = (c_int * count)(*[int(a.shape[1]) for a in As])
    ldb = (c_int * count)(*[int(b.shape[1]) for b in Bs])
    pa = (c_void_p * count)(*[a.data_ptr() for a in As])
    pb = (c_void_p * count)(*[b.data_ptr() for b in Bs])
    pw = (c_void_p * count)(*[w.data_ptr() for w in ws])
    info = (c_int * count)()
    _check(lib().kss_dense_hegv(ctx, count, n, pa, lda, pb, ldb, pw, info, 1 if real else 0), ctx)
    return np.array(list(info), dtype=np.int32)


DENSE_PHASES = ("cholesky", "reduce", "tridiagonalise", "bisection", "inverse_iteration", "back_transform")


def kss_dense_hegv_phase_ms(ctx) -> dict:
    """{phase: ms} of the last grid-team (order >= 160) dense eigensolve of the context."""
    ms = (c_double * 6)()
    _check(lib().kss_dense_hegv_phase_ms(ctx, ms), ctx)
    return dict(zip(DENSE_PHASES, list(ms)))


class kss_gemm_tune_entry(ctypes.Structure):
    _fields_ = [("device", c_int), ("kind", c_int), ("Mr", c_int), ("Nr", c_int), ("kblocks", c_int),
                ("splits", c_int), ("ms", c_double), ("ncand", c_int), ("form", c_int)]


def kss_autotune_gemm_table():
    """The GEMM K-split table (process-wide) as a list of dicts."""
    n = c_int()
    _check(lib().kss_autotune_gemm_count(byref(n)))
    out = []
    for i in range(n.value):
        e = kss_gemm_tune_entry()
        _check(lib().kss_autotune_gemm_get(i, byref(e)))
        out.append({f: getattr(e, f) for f, _ in e._fields_})
    return out


def kss_autotune_gemm_put(device: int, kind: int, Mr: int, Nr: int, kblocks: int, splits: int, form: int = 0):
    """Pin the schedule (kernel form and K-split) of a (kind, shape) GEMM configuration."""
    e = kss_gemm_tune_entry(device, kind, Mr, Nr, kblocks, splits, 0.0, 0, form)
    _check(lib().kss_autotune_gemm_put(byref(e)))


def kss_peak_probe(ctx, pipe: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the CUDA cores: pipe 0 FP64, 1 FP32."""
    v = c_double()
    _check(lib().kss_peak_probe(ctx, int(pipe), byref(v)), ctx)
    return v.value


def kss_selftest_bounded_wait(ctx, limit_ms: float = 50.0) -> int:
    """Run the bounded-wait failure path once (a wait on a word nothing writes); returns the
    status, KSS_ETIMEOUT when the path works."""
    return lib().kss_selftest_bounded_wait(ctx, float(limit_ms))


def kss_solve_batch(ctx, systems, iks, nbands, opts: kss_solve_opts, allow_noconv: bool = False):
    """Solve many (system, k-point) units together; returns (evals list, resid list, stats list, status)."""
    n = len(systems)
    hs = (c_void_p * n)(*[s.h.value for s in systems])
    ik = (c_int * n)(*[int(k) for k in iks])
    nbd = (c_int * n)(*[int(b) for b in nbands])
    ev = [np.zeros(int(b)) for b in nbands]
    rs = [np.zeros(int(b)) for b in nbands]
    evp = (c_void_p * n)(*[a.ctypes.data for a in ev])
    rsp = (c_void_p * n)(*[a.ctypes.data for a in rs])
    st = (kss_solve_stats * n)()
    status = lib().kss_solve_batch(ctx, n, hs, ik, nbd, byref(opts), evp, rsp, st)
    if not (status == KSS_ENOCONV and allow_noconv):
        _check(status, ctx)
    return ev, rs, [stats_dict(x) for x in st], status


# --------------------------------------------------------------------------------------------
# request server

def _cell_atoms(lattice, ecut, kpts, pos, D, fft_box, vloc_amp, vloc_sigma, nproj_per_atom, proj_alpha):
    lat = np.ascontiguousarray(np.asarray(lattice, np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(kpts, np.float64).reshape(-1, 3))
    p = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1, 3))
    d = np.ascontiguousarray(np.asarray(D if D is not None else [], np.float64).reshape(-1))
    cell = kss_cell()
    cell.lattice[:] = lat.tolist()
    cell.ecut = float(ecut)
    cell.nk = int(k.shape[0])
    cell.kpts_red = _dptr(k)
    cell.fft_box[:] = [int(v) for v in (fft_box or (0, 0, 0))]
    at = kss_atoms()
    at.natom = int(p.shape[0])
    at.pos_cart = _dptr(p)
    at.vloc_amp = float(vloc_amp)
    at.vloc_sigma = float(vloc_sigma)
    at.nproj_per_atom = int(nproj_per_atom)
    at.proj_alpha = float(proj_alpha)
    at.D = _dptr(d)
    return cell, at, (k, p, d)


def kss_server_start(ctx, hbm_budget_bytes: int, max_slots: int, opts: kss_solve_opts):
    _check(lib().kss_server_start(ctx, int(hbm_budget_bytes), int(max_slots), byref(opts)), ctx)


def kss_server_submit(ctx, lattice, ecut, kpts, pos, D, nband, fft_box=(0, 0, 0), vloc_amp=-2.0,
                      vloc_sigma=1.0, nproj_per_atom=4, proj_alpha=0.25) -> int:
    cell, at, keep = _cell_atoms(lattice, ecut, kpts, pos, D, fft_box, vloc_amp, vloc_sigma,
                                 nproj_per_atom, proj_alpha)
    t = c_uint64()
    _check(lib().kss_server_submit(ctx, byref(cell), byref(at), int(nband), byref(t)), ctx)
    return t.value


def kss_server_pump(ctx, max_ms: float = 0.0):
    a = c_int()
    q = c_int()
    _check(lib().kss_server_pump(ctx, float(max_ms), byref(a), byref(q)), ctx)
    return a.value, q.value


def kss_server_poll(ctx, ticket: int, nk: int, nband: int):
    """Returns None while running, else (status, evals (nk, nband), resid, latency_ms)."""
    d = c_int()
    ev = np.zeros((nk, nband))
    rs = np.zeros((nk, nband))
    lat = c_double()
    st = lib().kss_server_poll(ctx, c_uint64(ticket), byref(d), ev.ctypes.data, rs.ctypes.data, byref(lat))
    if st not in (KSS_OK, KSS_ENOCONV):
        _check(st, ctx)
    if not d.value:
        return None
    return st, ev, rs, lat.value


def kss_server_get_stats(ctx) -> dict:
    s = kss_server_stats()
    _check(lib().kss_server_get_stats(ctx, byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in kss_server_stats._fields_}


def kss_server_stop(ctx):
    _check(lib().kss_server_stop(ctx), ctx)
