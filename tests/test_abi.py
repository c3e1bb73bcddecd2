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


def test_params_struct_layout_matches_the_header(tmp_path):
    # the binding's ctypes mirror of susp_params has the C layout: compile a
    # probe against include/susp.h that prints sizeof and every offsetof
    import subprocess

    import paper_2307_13802_gb300 as s

    fields = [f for f, _ in s.susp_params._fields_]
    src = tmp_path / "probe.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "susp.h"\nint main(void){\n'
        '  printf("%zu\\n", sizeof(susp_params));\n'
        + "".join(f'  printf("%zu\\n", offsetof(susp_params, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(s.susp_params)
    for f, off in zip(fields, out[1:]):
        assert getattr(s.susp_params, f).offset == off, f


def test_parameters_are_checked_before_any_device_work():
    # invalid parameters are reported as SUSP_EINVAL with or without a GPU
    import paper_2307_13802_gb300 as s

    for bad in (dict(deterministic=1, precision="mixed"), dict(deterministic=2),
                dict(rebuild_every=-1), dict(autotune=2),
                dict(sample_every=0), dict(xi_min=0.1, xi_max=0.05)):
        try:
            s.System([1.0] * 10, [30.0, 30.0, 30.0], **bad)
        except s.SuspError as e:
            assert e.code == s.SUSP_EINVAL, bad
        else:
            raise AssertionError(f"accepted {bad}")
