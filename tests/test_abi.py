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


def test_binding_constants_match_the_header():
    """Every NIF_* integer constant the binding defines has the header's value."""
    from paper_2604_24666_gb300 import nif
    src = open(os.path.join(ROOT, "include", "nif.h")).read()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(NIF_[A-Z0-9_]+)\s+(\d+)u?\b", src)}
    for m in re.finditer(r"\b(NIF_[A-Z0-9_]+)\s*=\s*(-?\d+)", src):
        vals.setdefault(m.group(1), int(m.group(2)))
    checked = 0
    for name, v in vals.items():
        if hasattr(nif, name) and isinstance(getattr(nif, name), int):
            assert getattr(nif, name) == v, name
            checked += 1
    assert checked >= 10
    assert nif.NIF_FLAG_BILINEAR_FACES == 16 and nif.NIF_FLAG_CONCAT_ENCODING == 8


def test_unknown_flag_fails_validation_without_device():
    """A config with a flag bit the library does not define fails in argument
    validation, before any device call."""
    from paper_2604_24666_gb300 import nif, synth as S
    with pytest.raises(nif.NifError) as e:
        nif.nif_create(S.NetConfig(), S.torus_mesh(), flags=1 << 20)
    assert e.value.status == nif.NIF_ERR_ARG and "flag" in str(e.value)


def test_product_code_never_touches_the_oracle():
    """The library and its binding neither import, load nor name a path of
    the oracle package: it is test infrastructure only."""
    pkg = os.path.join(ROOT, "paper_2604_24666_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(os.path.join(dirpath, f), encoding="utf-8").read()
                if re.search(r"^\s*(import|from)\s+oracle\b|nif_oracle|oracle/", src, flags=re.M):
                    offenders.append(f)
    assert not offenders, offenders


def test_bounds_check_reports_the_normal_build_without_device():
    """The normal build's index checks compile away: nif_bounds_check says so
    without touching the device; null arguments fail validation."""
    from paper_2604_24666_gb300 import nif
    assert nif.nif_bounds_check() == (False, 0)
    assert nif.lib().nif_bounds_check(None, None) == nif.NIF_ERR_ARG
