"""The C-ABI library builds, loads and exports every function include/genesis.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "genesis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declarations_found():
    names = _declared()
    for must in ["me_synth", "ga_invert_batch", "lm_polish", "me_synth_vjp", "me_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1208_0302_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1208_0302_gb300 import _lib
    assert set(_declared()) <= set(_lib._SIGNATURES), set(_declared()) - set(_lib._SIGNATURES)
