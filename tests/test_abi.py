"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(open_cf_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2508_07605_b300 as ocf
    path = ocf.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding marshals every declared call
    assert declared <= set(ocf.exported_symbols()) | {"open_cf_create", "open_cf_destroy"}


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    import paper_2508_07605_b300 as ocf
    try:
        ocf.OpenCF(k=8, lam=0.1)
    except ocf.OpenCFError as e:
        assert e.code == ocf.UNSUPPORTED
    else:
        raise AssertionError("create succeeded without a GPU")
