"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/ccdyk.h declares, and argument checks
that run before any device call reject bad options."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ccdyk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src)) - {"cc_alloc_fn", "cc_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1901_10084_gb300 import build, _native
    build()
    return _native.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_1901_10084_gb300 import _native
    assert set(_native.EXPORTS) <= set(names)


def test_opts_defaults(lib):
    from paper_1901_10084_gb300 import _native as N
    o = N.cc_opts_default()
    assert o.eps == 0.2 and o.schedule == N.CC_SCHED_TILED and o.tile == 16
    assert o.precision == N.CC_PREC_FP64 and o.check_every == 10 and o.debug_skip_cta == -1
    assert o.refine_sweeps == 5 and o.refine_at == 1e-5 and o.variant == -1


@pytest.mark.parametrize("field,value", [("eps", 0.0), ("eps", -1.0), ("eps", float("inf")),
                                         ("tile", 12), ("check_every", 0),
                                         ("barrier_timeout_s", 0.0), ("precision", 7), ("variant", 5),
                                         ("variant", -2), ("refine_sweeps", 0), ("refine_sweeps", -3)])
def test_bad_options_rejected_before_device_work(lib, field, value):
    import numpy as np
    from paper_1901_10084_gb300 import _native as N
    o = N.cc_opts_default()
    setattr(o, field, value)
    with pytest.raises(N.CCError) as e:
        N.cc_create(10, np.zeros(45), np.ones(45), o)
    assert e.value.code == N.CC_ERR_ARG
    assert N.cc_last_error(None)


def test_small_n_rejected(lib):
    import numpy as np
    from paper_1901_10084_gb300 import _native as N
    with pytest.raises(N.CCError) as e:
        N.cc_create(2, np.zeros(1), np.ones(1), None)
    assert e.value.code == N.CC_ERR_ARG


def test_null_handle_calls_fail_cleanly(lib):
    from paper_1901_10084_gb300 import _native as N
    assert lib.cc_sweep(None, 1) == N.CC_ERR_ARG
    assert lib.cc_check(None, None) == N.CC_ERR_ARG
    lib.cc_destroy(None)


def test_warm_start_calls_reject_null_arguments(lib):
    """Argument checks of the warm-start entry points run before any device call."""
    from paper_1901_10084_gb300 import _native as N
    fp = ctypes.POINTER(ctypes.c_float)
    p = (ctypes.c_float * N.CC_WS_NPARAM)()
    pp = ctypes.cast(p, fp)
    assert lib.cc_warm_start_mlp(None, pp, 0.0, None) == N.CC_ERR_ARG
    assert lib.cc_ws_samples(None, None, None, 0, None) == N.CC_ERR_ARG
    assert lib.cc_mlp_forward(None, None, None, 4, None) == N.CC_ERR_ARG
    assert lib.cc_pair_passes(None, 1) == N.CC_ERR_ARG
    assert lib.cc_mlp_forward(pp, None, None, -1, None) == N.CC_ERR_ARG
    assert lib.cc_mlp_grad(pp, None, None, 16, 1.0, pp, None, None) == N.CC_ERR_ARG
    assert lib.cc_mlp_train(pp, None, None, 16, 16, 1, 1e-3, 0, 1.0, None, None) == N.CC_ERR_ARG
    assert lib.cc_mlp_train(pp, ctypes.c_void_p(16), ctypes.c_void_p(16), 16, 0, 1, 1e-3, 0, 1.0, None, None) \
        == N.CC_ERR_ARG
    dev = ctypes.c_void_p(16)    # never dereferenced: the weight check fails first
    for wt in (0.0, -1.0, float("inf"), float("nan")):
        assert lib.cc_mlp_grad(pp, dev, dev, 16, wt, pp, None, None) == N.CC_ERR_ARG
        assert lib.cc_mlp_train(pp, dev, dev, 16, 16, 1, 1e-3, 0, wt, None, None) == N.CC_ERR_ARG


def test_warm_start_parameter_count_matches_the_network():
    from paper_1901_10084_gb300 import _native as N
    from paper_1901_10084_gb300 import warmstart
    assert N.CC_WS_NPARAM == 10 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3
    src = open(os.path.join(ROOT, "include", "ccdyk.h")).read()
    assert re.search(r"#define CC_WS_NPARAM %d\b" % N.CC_WS_NPARAM, src)
    assert re.search(r"#define CC_WS_FEAT %d\b" % N.CC_WS_FEAT, src)
    assert re.search(r"#define CC_WS_PAIR_PASSES %d\b" % N.CC_WS_PAIR_PASSES, src)
    assert re.search(r"#define CC_NOALLOC_MAX_N %d\b" % N.CC_NOALLOC_MAX_N, src)
    p = warmstart.init_params(0)
    assert p.shape == (N.CC_WS_NPARAM,) and p.dtype.name == "float32"
    W1, b1, W2, b2, W3, b3 = warmstart.unpack(p)
    assert W1.shape == (10, 64) and W2.shape == (64, 64) and W3.shape == (64, 3) and b3.shape == (3,)


def test_checked_library_exports_the_same_symbols(lib):
    """libccdyk_checked.so (CCD_CHECKED) is built beside the normal library."""
    from paper_1901_10084_gb300 import buildlib
    chk = ctypes.CDLL(buildlib.LIB_CHECKED)
    for name in _declared():
        assert hasattr(chk, name), name
    src = open(os.path.join(ROOT, "include", "ccdyk.h")).read()
    assert re.search(r"#define CC_ERR_BOUNDS 7\b", src)


def _declarations():
    """name -> number of parameters, for every function include/ccdyk.h declares."""
    src = open(os.path.join(ROOT, "include", "ccdyk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(?:int|int32_t|int64_t|void|const char|cc_opts|cc_handle)\s*\**\s*(cc_[a-z0-9_]+)\s*"
                         r"\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_bindings_pass_as_many_arguments_as_the_header_declares(lib):
    decl = _declarations()
    assert set(decl) == set(_declared())
    checked = 0
    for name, count in decl.items():
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue
        assert len(fn.argtypes) == count, (name, len(fn.argtypes), count)
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("struct", ["cc_opts", "cc_stats"])
def test_struct_layout_matches_the_header(struct):
    """The ctypes mirrors of the option and statistics structs against the C
    compiler's layout of include/ccdyk.h: size and every field's offset."""
    import shutil
    import subprocess
    from paper_1901_10084_gb300 import _native as N
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    cls = getattr(N, struct)
    names = [f for f, _ in cls._fields_]
    work = os.path.join(ROOT, "tests", "_build")
    os.makedirs(work, exist_ok=True)
    prog = __import__("pathlib").Path(work) / f"layout_{struct}_{os.getpid()}.c"
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"ccdyk.h\"\nint main(void) {\n"
                    f"  printf(\"%zu\\n\", sizeof({struct}));\n"
                    + "".join(f"  printf(\"%zu\\n\", offsetof({struct}, {f}));\n" for f in names)
                    + "  return 0;\n}\n")
    exe = prog.with_suffix("")
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    prog.unlink()
    exe.unlink()
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in names]
