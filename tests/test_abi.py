"""The C ABI library loads without a GPU and exports every declared entry point."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nif.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nif_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2604_24666_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_resolves_all_entry_points():
    from paper_2604_24666_gb300 import nif
    got = set(nif.exported_symbols())
    assert set(_declared()) <= got | {"nif_last_error"}


def test_create_without_device_fails_cleanly():
    """Argument validation runs before any device call."""
    from paper_2604_24666_gb300 import nif, synth as S
    bad = S.NetConfig(voxel_res=12)     # not a power of two
    with pytest.raises(nif.NifError) as e:
        nif.nif_create(bad, S.torus_mesh())
    assert e.value.status == nif.NIF_ERR_ARG
