"""Shared helpers for the tests: build/load the library, create a context on torch's stream,
and set up a workloads.System through the C ABI."""
import numpy as np

import paper_2507_08578_gb300.kss as K
from paper_2507_08578_gb300 import build as B


def ensure_built():
    B.build()
    return K.lib()


def make_ctx():
    import torch
    return K.kss_create(0, torch.cuda.current_stream().cuda_stream)


def setup(ctx, s):
    """kss_setup for a workloads.System."""
    return K.kss_setup(ctx, s.lattice, s.ecut, s.kpts, s.pos, s.D,
                       fft_box=s.fft_box or (0, 0, 0), vloc_amp=s.vloc_amp,
                       vloc_sigma=s.vloc_sigma, nproj_per_atom=s.nproj_per_atom,
                       proj_alpha=s.proj_alpha, Q=getattr(s, "Q", None))


def rel_err_rows(a, b):
    """max over rows of |a_n - b_n| / |b_n|."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.linalg.norm(a - b, axis=-1)
    den = np.maximum(np.linalg.norm(b, axis=-1), 1e-300)
    return float(np.max(num / den))


def rel_err_elem(a, b):
    """max over rows of max_g |a_ng - b_ng| / max_g |b_ng|: the element-wise form of the parity
    bar (a row norm can hide large relative errors in the small coefficients of a row)."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.max(np.abs(a - b), axis=-1)
    den = np.maximum(np.max(np.abs(b), axis=-1), 1e-300)
    return float(np.max(num / den))
