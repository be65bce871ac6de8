"""The C library builds for sm_103a, loads, and exports every function the
header declares; host-side argument checks need no GPU."""
import ctypes
import subprocess

import pytest


def test_library_exports_header_functions():
    torch = pytest.importorskip("torch")  # noqa: F841 (loads the CUDA runtime the library links)
    from paper_1705_02876_gb300 import build, kf
    build.build()
    kf.load()
    syms = subprocess.run(["nm", "-D", "--defined-only", kf.library_path()], capture_output=True,
                          text=True, check=True).stdout
    exported = {line.split()[-1] for line in syms.splitlines() if " T " in line}
    declared = kf.header_functions()
    assert declared, "no functions parsed from kf.h"
    missing = [f for f in declared if f not in exported]
    assert not missing, missing


def test_options_defaults_and_struct_size():
    pytest.importorskip("torch")
    from paper_1705_02876_gb300 import kf
    o = kf.options()
    assert o.precision_mode == kf.PRECISION_ROUTED
    assert o.max_cands == 6 and abs(o.chi2_cut - 30.0) < 1e-6 and o.topk == 4
    # the ctypes mirror has the C struct's size: 17 four-byte fields
    assert ctypes.sizeof(kf.Options) == 17 * 4


def test_context_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1705_02876_gb300 import kf
    with pytest.raises(kf.KFError):
        kf.Context(0)
