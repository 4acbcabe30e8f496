"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every function
the header declares, and refuses to run without a GPU (no CPU fallback)."""
import pytest

import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def test_exports_every_header_symbol(lib):
    names = K.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_every_header_function_has_a_ctypes_prototype():
    """A function without a prototype would pass 64-bit pointers as C ints."""
    missing = set(K.header_functions()) - set(K.signatures())
    assert not missing, sorted(missing)


def test_version(lib):
    assert K.kss_version() == 1


def test_no_cpu_fallback_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(K.KssError) as e:
        K.kss_create(0)
    assert e.value.status == K.KSS_ECUDA


def test_null_arguments_rejected(lib):
    assert lib.kss_destroy(None) == K.KSS_EINVAL
    assert lib.kss_sys_destroy(None) == K.KSS_EINVAL
    assert lib.kss_apply_H(None, 0, 1, None, None, 1, 0) == K.KSS_EINVAL
    assert lib.kss_solver_step(None, None) == K.KSS_EINVAL
    assert lib.kss_last_error(None) == b"null context"
