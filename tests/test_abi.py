"""The C library builds for sm_103a, loads, and exports every function the
header declares; host-side argument checks need no GPU."""
import ctypes
import os
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
    assert abs(o.window_max_dphi - 0.05) < 1e-7 and abs(o.window_max_dz - 5.0) < 1e-6


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of kf_options, kf_seeding and kf_geometry have the C
    structs' sizes and field offsets, as gcc lays them out from kf.h."""
    pytest.importorskip("torch")
    import shutil
    from paper_1705_02876_gb300 import kf
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    mirrors = {"kf_options": kf.Options, "kf_seeding": kf.Seeding, "kf_geometry": kf.Geometry}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kf.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(kf.HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_context_create_fails_cleanly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1705_02876_gb300 import kf
    with pytest.raises(kf.KFError):
        kf.Context(0)


def _header_params():
    """Parameter declarations of every function declared in kf.h, from the
    header text."""
    import re
    from paper_1705_02876_gb300 import kf
    text = re.sub(r"/\*.*?\*/", "", open(kf.HEADER).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"\b(kf_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        args = " ".join(m.group(2).split())
        out[m.group(1)] = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
    return out


def _header_arity():
    return {k: len(v) for k, v in _header_params().items()}


# C parameter type (without its name) -> (kind, size in bytes) as the calling
# convention sees it; every pointer, kf_stream included, is one kind
_SCALARS = {"int": ("int", 4), "int32_t": ("int", 4), "unsigned": ("int", 4), "uint32_t": ("int", 4),
            "int64_t": ("int", 8), "size_t": ("int", 8), "float": ("float", 4), "double": ("float", 8)}


def _c_kind(decl):
    if "*" in decl or decl.split()[0] == "kf_stream":
        return ("ptr", 8)
    t = " ".join(w for w in decl.split()[:-1] if w != "const")
    return _SCALARS[t]


def _ctypes_kind(t):
    if t in (ctypes.c_float, ctypes.c_double):
        return ("float", ctypes.sizeof(t))
    if t is ctypes.c_void_p or t is ctypes.c_char_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return ("ptr", 8)
    return ("int", ctypes.sizeof(t))


def test_binding_declares_every_header_function_with_its_arity():
    """The ctypes binding gives every function of kf.h argument types, as many
    as the header's declaration has parameters (a missing or extra argument
    would be passed silently otherwise)."""
    pytest.importorskip("torch")
    from paper_1705_02876_gb300 import build, kf
    build.build()
    L = kf.load()
    arity = _header_arity()
    assert set(arity) == set(kf.header_functions())
    wrong = {}
    for name, n in arity.items():
        f = getattr(L, name)
        if f.argtypes is None or len(f.argtypes) != n:
            wrong[name] = (n, None if f.argtypes is None else len(f.argtypes))
    assert not wrong, wrong


def test_binding_argument_types_match_the_header():
    """Each argument's ctypes type has the kind (pointer, integer, floating)
    and width of the header's parameter: an int passed where the header takes
    an int64_t, or a float for a double, would be read wrongly by the callee."""
    pytest.importorskip("torch")
    from paper_1705_02876_gb300 import build, kf
    build.build()
    L = kf.load()
    wrong = []
    for name, params in _header_params().items():
        for i, (decl, t) in enumerate(zip(params, getattr(L, name).argtypes)):
            if _c_kind(decl) != _ctypes_kind(t):
                wrong.append((name, i, decl, t.__name__))
    assert not wrong, wrong


def test_library_defaults_equal_the_oracle_defaults():
    """kf_options_default and kf_seeding_default give the settings the
    oracle's build and seeding functions default to, so that a test calling
    both sides with defaults compares like with like (float32 on the library
    side)."""
    import inspect

    import numpy as np
    pytest.importorskip("torch")
    from oracle import kf_oracle as orc
    from paper_1705_02876_gb300 import kf
    o, s = kf.options(), kf.seeding()
    b = {k: v.default for k, v in inspect.signature(orc.build_arrays).parameters.items()}
    pairs = [(o.max_cands, b["max_cands"]), (o.chi2_cut, b["chi2_cut"]), (o.window_nsigma, b["nsigma"]),
             (o.hit_sigma_rphi, b["sigma_rphi"]), (o.hit_sigma_z, b["sigma_z"]), (o.topk, b["topk"]),
             (o.window_max_dphi, b["dphi_max"]), (o.window_max_dz, b["dz_max"])]
    f = {k: v.default for k, v in inspect.signature(orc.seed_fit_inputs).parameters.items()}
    pairs += [(getattr(s, k), v) for k, v in orc.SEED_DEFAULTS.items()]
    pairs += [(getattr(s, k), f[k]) for k in ("pt_min", "pt_both_charges", "pt_unresolved", "p_sigma_resolved",
                                              "p_sigma_unresolved")]
    for lib_value, oracle_value in pairs:
        assert lib_value == np.float32(oracle_value), (lib_value, oracle_value)


C_CLIENT = r"""
#include <stdio.h>
#include "kf.h"

#define EXPECT(cond, code) do { if (!(cond)) { printf("failed %d\n", code); return code; } } while (0)

int main(void)
{
    kf_options o;
    kf_seeding s;
    kf_context *ctx = (kf_context *)&o;
    float r[3] = {4.0f, 8.0f, 12.0f}, xx0[3] = {0.01f, 0.01f, 0.01f};
    kf_geometry g;
    float f[8];
    kf_options_default(&o);
    kf_seeding_default(&s);
    EXPECT(o.max_cands == 6 && o.topk == 4 && o.precision_mode == 1, 1);
    EXPECT(s.n_phi_bins == 256 && s.n_z_bins == 64, 2);
    /* no sm_103a device here: a clean error, no context */
    EXPECT(kf_context_create(&ctx, 0) == KF_ERR_UNSUPPORTED && ctx == NULL, 3);
    EXPECT(kf_context_create(NULL, 0) == KF_ERR_ARG, 4);
    EXPECT(kf_last_error(NULL) != NULL && kf_last_error(NULL)[0] != 0, 5);
    kf_context_destroy(NULL);
    EXPECT(kf_fit_tracks(NULL, NULL, 0, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                         &o, NULL) == KF_ERR_ARG, 6);
    EXPECT(kf_transport_batch(NULL, 0, NULL, NULL, NULL) == KF_ERR_ARG, 7);
    /* the context-free fit checks its arguments on the host first */
    g.n_layers = 3;
    g.r = r;
    g.x_over_x0 = xx0;
    g.z_half = 100.0f;
    g.bz_tesla = 3.8f;
    EXPECT(kf_fit_tracks_noalloc(NULL, 1, f, f, NULL, f, f, NULL, f, f, f, NULL, NULL, &o, NULL) == KF_ERR_ARG, 8);
    EXPECT(kf_fit_tracks_noalloc(&g, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, &o, NULL)
           == KF_OK, 9);
    EXPECT(kf_fit_tracks_noalloc(&g, -1, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, &o, NULL)
           == KF_ERR_ARG, 10);
    EXPECT(kf_fit_tracks_noalloc(&g, KF_NOALLOC_MAX_TRACKS + 1, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                                 NULL, NULL, &o, NULL) == KF_ERR_TOO_LARGE, 11);
    EXPECT(kf_fit_tracks_noalloc(&g, 1, NULL, f, NULL, f, f, NULL, f, f, f, NULL, NULL, &o, NULL) == KF_ERR_ARG, 12);
    EXPECT(kf_fit_tracks_noalloc(&g, 1, (const float *)((const char *)f + 2), f, (const int8_t *)f, f, f,
                                 (const uint32_t *)f, f, f, f, (int16_t *)f, (uint32_t *)f, &o, NULL) == KF_ERR_ARG, 13);
    g.n_layers = 0;
    EXPECT(kf_fit_tracks_noalloc(&g, 1, f, f, (const int8_t *)f, f, f, (const uint32_t *)f, f, f, f, (int16_t *)f,
                                 (uint32_t *)f, &o, NULL) == KF_ERR_ARG, 14);
    printf("ok\n");
    return 0;
}
"""


def test_c_client_without_a_gpu(tmp_path):
    """kf.h compiles as strict C99 and a C program linked against the library
    gets the documented error codes, without a GPU and without a crash: no
    context on a machine without an sm_103a device, KF_ERR_ARG for null
    arguments, and the context-free fit's host-side checks (empty batch,
    negative or too large sizes, null and misaligned pointers, bad geometry)."""
    torch = pytest.importorskip("torch")
    import shutil
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_1705_02876_gb300 import build, kf
    build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    lib = kf.library_path()
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.dirname(kf.HEADER),
                    str(src), "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
