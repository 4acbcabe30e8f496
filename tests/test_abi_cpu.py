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


def _declarations():
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kss.h")
    src = open(path).read()
    decl = re.compile(r"^(?:kss_status|const char\*|int|void)\s+(kss_\w+)\s*\(", re.M)
    sec = re.compile(r"/\* -{20,}\n((?: \*.*\n)+?) \* -{20,}")
    out = []
    for m in decl.finditer(src):
        pre = src[:m.start()]
        comment = pre[pre.rfind("/*"):pre.rfind("*/")]
        secs = list(sec.finditer(pre))
        out.append((m.group(1), comment, secs[-1].group(1) if secs else ""))
    return out


def test_header_documents_every_entry_point():
    """Every declaration in kss.h carries, in its comment or its section header, the passage of
    the paper it follows (or says it has none), and its error behaviour."""
    import re
    decls = _declarations()
    assert len(decls) == len(K.header_functions())
    no_cite = [n for n, c, s in decls if not re.search(r"§|Eq\.|counterpart", c + s)]
    no_err = [n for n, c, s in decls if not re.search(r"Error|error|Cannot fail|Returns|KSS_E", c)]
    assert not no_cite, no_cite
    assert not no_err, no_err
