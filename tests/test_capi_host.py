"""Host-side checks of the C ABI library (no GPU): it builds for sm_103a, loads, exports
every entry point the header declares, and its host-only functions agree with the oracle."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1901_09745_gb300 import build
    build.build()
    import paper_1901_09745_gb300 as P
    P.lib()
    return P


def test_library_exports_every_declared_symbol(P):
    names = P.exported_symbols()
    assert "lbm_create" in names and "lbm_step" in names
    L = C.CDLL(P.library_path())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_header_cites_the_paper_for_each_hot_path_entry_point():
    """Each hot-path prototype sits under a comment that cites the passage defining it."""
    text = open(os.path.join(ROOT, "include", "psc_lbm.h")).read()
    assert "arXiv 1901.09745" in text
    for name in ("lbm_create", "lbm_set_particles", "lbm_step", "lbm_get_forces"):
        pos = text.index(name + "(")
        block = text[:pos]
        comment = block[block.rfind("/*"):]
        assert re.search(r"(Eq\.|Sec\.|Table)", comment), name


@pytest.mark.parametrize("lattice", [9, 19])
def test_lattice_tables_match_oracle(P, lattice):
    e, w, o = P.lbm_lattice_tables(lattice)
    eo, wo, oo = O.lattice_tables(lattice)
    assert np.array_equal(e, eo)
    assert np.array_equal(o, oo)
    assert np.allclose(w, wo, rtol=0, atol=1e-17)


def test_create_without_gpu_fails_cleanly_or_validates(P):
    """Invalid parameters are rejected before any device work (works without a GPU)."""
    with pytest.raises(P.LbmError) as ei:
        P.lbm_create(9, 16, 16, 2, tau=0.8)   # D2Q9 with nz = 2
    assert ei.value.status == P.LBM_ERR_ARG
    with pytest.raises(P.LbmError) as ei:
        P.lbm_create(19, 8, 8, 8, tau=0.5)    # tau must exceed 1/2
    assert ei.value.status == P.LBM_ERR_ARG
    with pytest.raises(P.LbmError) as ei:
        P.lbm_create(7, 8, 8, 8)
    assert ei.value.status == P.LBM_ERR_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1901_09745_gb300 as P
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(ImportError):
        P.lib()


def test_unchecked_build_reports_no_checks(P):
    """The default library is the unchecked build: it says so, and the check word call
    answers LBM_ERR_UNSUPPORTED rather than a misleading zero."""
    assert not P.lbm_checked_build()
    with pytest.raises(P.LbmError) as ei:
        P.lbm_check_violations()
    assert ei.value.status == P.LBM_ERR_UNSUPPORTED
