"""The C-ABI library builds, loads and exports every function declared in
include/fkfast.h; host-side argument checking works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1910_06451_gb300 import build, fkfast

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fkfast.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fkfast.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fkfast.EXPORTS)


def test_chain_argument_errors(lib):
    dh = np.array([[0.3, 1.5707963, 0.0, 0.0, 0.0]] * 3)
    with pytest.raises(fkfast.FkError) as e:
        fkfast.fk_chain_create(dh, None, [0, 1, 5], np.zeros((3, 3)))
    assert e.value.code == fkfast.FK_ERR_ARG and "outside" in str(e.value)
    bad = dh.copy()
    bad[1, 4] = 7
    with pytest.raises(fkfast.FkError):
        fkfast.fk_chain_create(bad, None, [0, 1], np.zeros((2, 3)))
    base = np.eye(4)
    base[3, 0] = 1.0
    with pytest.raises(fkfast.FkError):
        fkfast.fk_chain_create(dh, base, [0, 1], np.zeros((2, 3)))
    with pytest.raises(fkfast.FkError):
        fkfast.fk_chain_create(np.zeros((17, 5)), None, [0], np.zeros((1, 3)))
    h = fkfast.fk_chain_create(dh, None, [0, 1, 2, 3], np.zeros((4, 3)))
    assert h.value
    out = ctypes.c_void_p()
    assert lib.fastron_model_create(None, ctypes.byref(out)) == fkfast.FK_ERR_ARG
    assert b"chain is NULL" in lib.fk_last_error()
    fkfast.fk_chain_destroy(h)


def test_library_fails_loudly_when_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(fkfast, "_lib", None)
    monkeypatch.setattr(fkfast, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(fkfast.FkError):
        fkfast.load()
