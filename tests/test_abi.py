"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function include/adscl.h declares, the Python binding names match, and invalid configurations
are rejected before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adscl.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adscl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("adscl_create", "adscl_set_initial", "adscl_evolve", "adscl_spectrum",
                     "adscl_grad", "adscl_get_state", "adscl_set_state", "adscl_last_error",
                     "adscl_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1706_07413_b300 import adscl, build
    lib = adscl.load()
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(adscl_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in adscl.SIGNATURES, f"binding lacks {n}"


def test_build_targets_sm_103a_only():
    from paper_1706_07413_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_invalid_configs_rejected_before_device_work():
    from paper_1706_07413_b300 import adscl
    lib = adscl.load()
    for Ns in ([15], [18], [100], [adscl.load().adscl_max_points() + 8]):
        arr = (ctypes.c_int32 * len(Ns))(*Ns)
        cfg = adscl.adscl_config()
        cfg.num_instances = len(Ns)
        cfg.N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
        h = ctypes.c_void_p()
        assert lib.adscl_create(ctypes.byref(cfg), ctypes.byref(h)) == adscl.ADSCL_EINVAL
        assert not h.value
    cfg = adscl.adscl_config()
    cfg.num_instances = 0
    h = ctypes.c_void_p()
    assert lib.adscl_create(ctypes.byref(cfg), ctypes.byref(h)) == adscl.ADSCL_EINVAL
    assert lib.adscl_create(None, ctypes.byref(h)) == adscl.ADSCL_EINVAL
    # null context handling of the query functions
    assert lib.adscl_launch_count(None) == 0
    assert lib.adscl_last_error(None) == b"null context"
    assert lib.adscl_adjoint_storage(None, None, None, None, None) == adscl.ADSCL_EINVAL
    assert lib.adscl_get_clock(None, None, None) == adscl.ADSCL_EINVAL
    lib.adscl_destroy(None)


def test_config_struct_layout_matches_header(tmp_path):
    """The binding's adscl_config has the C compiler's size and field offsets."""
    from paper_1706_07413_b300 import adscl
    fields = [f[0] for f in adscl.adscl_config._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("{f} %zu\\n", offsetof(adscl_config, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "adscl.h"\nint main(void) {\n'
                   f'{body}    printf("sizeof %zu\\n", sizeof(adscl_config));\n    return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for f in fields:
        assert int(got[f]) == getattr(adscl.adscl_config, f).offset, f
    assert int(got["sizeof"]) == ctypes.sizeof(adscl.adscl_config)
