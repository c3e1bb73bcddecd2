"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares (no compute calls)."""
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
        names |= set(re.findall(r"\b(susp_[a-z_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("susp_create", "susp_build_neighbors", "susp_step", "susp_stress",
              "susp_create_batch", "susp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._load_builder().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2307_13802_gb300 as s
    assert set(s._SIGNATURES) == _declared()


def test_create_without_gpu_fails_cleanly():
    import paper_2307_13802_gb300 as s
    try:
        import torch
        if torch.cuda.is_available():
            return
    except Exception:
        pass
    try:
        s.System([1.0] * 10, [30.0, 30.0, 30.0])
    except s.SuspError as e:
        assert e.code == s.SUSP_ENODEV
    else:
        raise AssertionError("expected SUSP_ENODEV without a GPU")



def test_green_kubo_argument_errors_need_no_device():
    import numpy as np

    import paper_2307_13802_gb300 as s

    x = np.zeros(10)
    for args in ((x, 1, 0.1, 1.0, 1.0), (x, 11, 0.1, 1.0, 1.0), (x, 5, 0.0, 1.0, 1.0),
                 (x, 5, 0.1, -1.0, 1.0), (x, 5, 0.1, 1.0, 0.0)):
        try:
            s.green_kubo(*args)
        except s.SuspError as e:
            assert e.code == s.SUSP_EINVAL
        else:
            raise AssertionError(f"accepted {args[1:]}")
