"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/tnmc.h declares (no compute calls: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tnmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnmc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_06538_gb300 import _capi, build
    build()
    return _capi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tnmc_create", "tnmc_build_env", "tnmc_propose", "tnmc_accept", "tnmc_observables",
                 "tnmc_destroy", "tnmc_couplings_pmj", "tnmc_eval_conditionals"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2409_06538_gb300 import _capi
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _capi.SIGNATURES, f"binding lacks {name}"


def test_version_and_null_handling(lib):
    assert lib.tnmc_version() >= 100
    assert lib.tnmc_destroy(None) == 0
    # NULL context is rejected with TNMC_ERR_ARG without touching a device
    assert lib.tnmc_build_env(None, None) == 1
    assert lib.tnmc_propose(None, 1, 0, None, None, None) == 1
    assert lib.tnmc_accept(None, None, None) == 1


def test_product_path_has_no_fallback():
    """The binding refuses to run without the compiled library (no CPU fallback)."""
    from paper_2409_06538_gb300 import _capi
    with pytest.raises(ImportError):
        _capi.load(path=os.path.join(ROOT, "does_not_exist", "libtnmc.so"))
    import paper_2409_06538_gb300.tnmc as t
    src = open(t.__file__).read()
    assert "oracle" not in src
