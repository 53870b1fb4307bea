"""The C ABI library loads without a GPU and exports every function include/stmg.h declares."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:stmg_status|const char\*)\s+(stmg_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2408_04372_gb300 as stmg
    if not os.path.exists(stmg.LIB_PATH):
        from paper_2408_04372_gb300 import build
        build.build()
    lib = ctypes.CDLL(stmg.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert set(stmg.EXPORTS) <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", stmg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (stmg_\w+)", out))
    assert declared <= exported


def test_binding_loads_and_reports_missing_gpu_loudly():
    import paper_2408_04372_gb300 as stmg
    lib = stmg.load()
    assert lib.stmg_last_error(None) == b"null context"
