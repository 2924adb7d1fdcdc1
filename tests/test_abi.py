"""The C ABI library loads and exports what include/nimbus.h declares; the ctypes
binding's structs match the header's layouts.  CPU only (no compute calls)."""
import ctypes as C
import os
import re
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nimbus.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2402_13747_b300 import build, _abi
    build.build()
    return _abi.load()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"NIMBUS_API\s+[\w\s\*]*?\b(nimbus_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("nimbus_voxelize", "nimbus_trace_coarse", "nimbus_refine", "nimbus_query"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2402_13747_b300 import _abi
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(nimbus_\w+)", out))
    assert set(declared()) <= exported
    assert set(_abi.EXPORTS) == set(declared())


def test_struct_layouts_match_header(tmp_path):
    from paper_2402_13747_b300 import _abi
    structs = {"nimbus_cloud": _abi.Cloud, "nimbus_edges": _abi.Edges, "nimbus_vox_params": _abi.VoxParams,
               "nimbus_trace_params": _abi.TraceParams, "nimbus_refine_params": _abi.RefineParams,
               "nimbus_path_counts": _abi.Counts, "nimbus_path_view": _abi.PathView,
               "nimbus_coarse_view": _abi.CoarseView, "nimbus_scene_view": _abi.SceneView,
               "nimbus_static_tables": _abi.StaticTables, "nimbus_static_info": _abi.StaticInfo,
               "nimbus_tuning": _abi.Tuning, "nimbus_segment_params": _abi.SegmentParamsC,
               "nimbus_segment_counts": _abi.SegmentCounts}
    lines = []
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname}.{f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    src = tmp_path / "lay.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"nimbus.h\"\nint main(){\n" +
                   "\n".join(lines) + "\nreturn 0;}\n")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f in py._fields_:
            assert int(got[f"{cname}.{f[0]}"]) == getattr(py, f[0]).offset, (cname, f[0])


def test_product_path_does_not_load_the_oracle(lib):
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import importlib, os
        import paper_2402_13747_b300, paper_2402_13747_b300._abi
        for m in ('serve', 'scenes', 'config'):
            if os.path.exists(os.path.join(%r, 'paper_2402_13747_b300', m + '.py')):
                importlib.import_module('paper_2402_13747_b300.' + m)
        paper_2402_13747_b300._abi.load()
        assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), sorted(sys.modules)
        print('ok')
    """ % (ROOT, ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr
    pkg = os.path.join(ROOT, "paper_2402_13747_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".hpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), fn
                assert "nimbus_oracle" not in txt, fn


def test_missing_library_fails_loudly(tmp_path):
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        from paper_2402_13747_b300 import _abi
        _abi.LIB_PATH = %r
        try:
            _abi.load()
        except ImportError as e:
            print('raised', e)
    """ % (ROOT, str(tmp_path / "missing.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "raised" in r.stdout


def test_param_blocks():
    from paper_2402_13747_b300 import _abi, config
    p = config.Params(max_refl=3, max_diff=1)
    t = _abi.trace_params(p)
    assert t.max_int == 4 and t.kappa == 100 and t.n_launch == 165012
    v = _abi.vox_params(p, region=[[0, 0, 0], [1, 2, 3]])
    assert v.has_region == 1 and list(v.region_max) == [1, 2, 3]
    r = _abi.refine_params(p)
    assert r.rho == 2000 and r.delta == 1e-4


def test_error_codes_without_a_context(lib):
    """The boundary's error behaviour, with no device work: a device index no machine
    has is an argument error that leaves no context; every entry point refuses a null
    context with NIMBUS_ERR_ARG (no crash, no exception); the null context has an error
    text; the launch counter reads without a context."""
    from paper_2402_13747_b300 import _abi
    ctx = C.c_void_p(12345)
    assert lib.nimbus_create(C.byref(ctx), 1 << 20, 0) == _abi.ERR_ARG
    assert ctx.value is None
    assert lib.nimbus_last_error(None) == b"null context"
    pointer_types = (C.c_void_p, C.c_char_p)
    for name in _abi.EXPORTS:
        if name in ("nimbus_create", "nimbus_last_error", "nimbus_kernel_launches", "nimbus_device_allocations"):
            continue
        f = getattr(lib, name)
        args = [None if (t in pointer_types or hasattr(t, "contents") or t.__name__.startswith("LP_")) else t(0)
                for t in f.argtypes]
        assert f(*args) == _abi.ERR_ARG, name
    n = C.c_int64(-1)
    assert lib.nimbus_kernel_launches(None) == _abi.ERR_ARG
    assert lib.nimbus_kernel_launches(C.byref(n)) == _abi.OK and n.value >= 0
    assert lib.nimbus_device_allocations(None) == _abi.ERR_ARG
    assert lib.nimbus_device_allocations(C.byref(n)) == _abi.OK and n.value >= 0


def test_a_c_program_links_and_calls_the_library(lib, tmp_path):
    """A plain C caller: the header compiles as C, the program links against
    libnimbus.so, and the calls that need no device answer as declared (an absent
    device is NIMBUS_ERR_ARG and leaves no context; the launch counter reads)."""
    from paper_2402_13747_b300 import _abi
    src = tmp_path / "caller.c"
    src.write_text(textwrap.dedent("""\
        #include <stdio.h>
        #include "nimbus.h"
        int main(void) {
          nimbus_ctx* ctx = (nimbus_ctx*)1;
          int rc = nimbus_create(&ctx, 1 << 20, 0);
          int64_t n = -1;
          int rl = nimbus_kernel_launches(&n);
          printf("%d %d %d %lld %s\\n", rc, ctx == NULL, rl, (long long)n, nimbus_last_error(NULL));
          return 0;
        }
        """))
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_abi.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    os.path.join(libdir, "libnimbus.so"), "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split(maxsplit=4)
    assert out[:4] == [str(_abi.ERR_ARG), "1", str(_abi.OK), "0"]
    assert out[4].strip() == "null context"
