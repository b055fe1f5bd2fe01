"""The C ABI library loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

from paper_2606_31548_b300 import hcao

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hcao_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = hcao.lib()
    decl = _declared()
    assert len(decl) >= 20
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(hcao.EXPORTS) <= decl


def test_default_config_without_gpu():
    cfg = hcao.Config()
    hcao.lib().hcao_default_config(ctypes.byref(cfg))
    assert cfg.precision == hcao.FP64 and cfg.table_points == 2048 and cfg.max_rounds == 2
