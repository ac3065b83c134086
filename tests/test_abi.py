"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/flints.h declares (no compute calls here)."""
import ctypes
import subprocess

import pytest

from paper_1003_4984_gb300 import api
from paper_1003_4984_gb300.build import build


@pytest.fixture(scope="module")
def lib_path():
    return build()


def test_header_declares_the_boundary():
    names = api.header_functions()
    for required in ("flints_plan", "flints_lens_spin0", "flints_lens_spin2", "flints_free", "flints_lens_range",
                     "flints_stencil", "flints_lens_batch", "flints_get_stats", "flints_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in api.header_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(api.header_functions()) <= exported


def test_binding_loads_and_reports_errors_without_gpu(lib_path):
    lib = api.load_library()
    assert lib.flints_last_error() is not None
    # argument validation happens on the host before any device call
    h = ctypes.c_void_p()
    rc = lib.flints_plan(ctypes.byref(h), 0, 10, None, None, 0, 32, 0, 0, None)
    assert rc == 1 and not h.value
    assert b"nside" in lib.flints_last_error() or b"cl" in lib.flints_last_error()
    cl = (ctypes.c_double * 33)(*([0.0, 0.0] + [1.0] * 31))
    rc = lib.flints_plan(ctypes.byref(h), 16, 32, cl, None, 0, 16, 0, 1 << 12, None)
    assert rc == 1 and not h.value and b"flag" in lib.flints_last_error()
    rc = lib.flints_plan(ctypes.byref(h), 16, 32, cl, None, 0, 20, 0, 0, None)
    assert rc == 1 and b"K must be" in lib.flints_last_error()


def test_paper_plan_validates_arguments_without_gpu(lib_path):
    lib = api.load_library()
    h = ctypes.c_void_p()
    cl = (ctypes.c_double * 33)(*([0.0, 0.0] + [1.0] * 31))
    for args, msg in [((16, 32, cl, None, 3, 0, 0, 0), b"level y"), ((15, 32, cl, None, 2, 0, 0, 0), b"divisible"),
                      ((16, 32, cl, None, 1, 0, 5, 0), b"precision"), ((16, 32, None, None, 1, 0, 0, 0), b"cl is NULL"),
                      ((16384, 32, cl, None, 1, 0, 0, 0), b"nside"), ((16, 32, cl, None, 1, 3, 0, 0), b"spin"),
                      ((16, 32, cl, None, 1, 2, 0, 8), b"flag"), ((16, 32, cl, None, 1, 0, 0, 1), b"AUGMENTED"),
                      ((16, 32, cl, None, 1, 2, 1, 1), b"AUGMENTED")]:
        rc = lib.flints_paper_plan(ctypes.byref(h), *args, None)
        assert rc == 1 and not h.value and msg in lib.flints_paper_last_error(), (args, lib.flints_paper_last_error())
    assert lib.flints_paper_lens(None, 0, 1, None, None, None, None, None, None) == 1


def test_product_path_refuses_without_library(tmp_path):
    with pytest.raises(api.FlintsError):
        api.load_library.__wrapped__(str(tmp_path / "missing.so")) if hasattr(api.load_library, "__wrapped__") else \
            _load_missing(tmp_path)


def _load_missing(tmp_path):
    saved = api._lib
    api._lib = None
    try:
        api.load_library(str(tmp_path / "missing.so"))
    finally:
        api._lib = saved


def test_noalloc_rejects_misaligned_buffers_without_gpu(lib_path):
    """flints_lens_noalloc checks the alignment rules of the plan-based entry points on
    the host, before any device call (the addresses below are never dereferenced)."""
    lib = api.load_library()
    cl = (ctypes.c_double * 33)(*([0.0, 0.0] + [1.0] * 31))
    a16, a8 = 0x10000, 0x10008
    cases = [(0, a16, a16, a16, 0x10004, b"var 8 bytes"),   # var misaligned
             (2, a8, a16, a16, a16, b"map, out 16 bytes"),   # spin-2 map on 8 bytes
             (0, a16, a8, a16, a16, b"defl 16 bytes"),       # deflections on 8 bytes
             (2, a16, a16, a8, a16, b"map, out 16 bytes")]   # spin-2 output on 8 bytes
    for spin, m, d, o, v, msg in cases:
        rc = lib.flints_lens_noalloc(16, 32, cl, None, spin, 16, 0, 0, 12, m, d, o, v, None, None)
        assert rc == 1 and msg in lib.flints_noalloc_last_error(), (spin, lib.flints_noalloc_last_error())
    # spin 0 maps and outputs need 8 bytes only: this call passes the checks up to the
    # device address lookup, so it is not made here
    rc = lib.flints_measure_fma_peak(0, 0, None, None)
    assert rc == 1 and b"tflops is NULL" in lib.flints_measure_last_error()


def test_binding_refuses_host_or_mistyped_buffers_on_the_host(lib_path):
    """The binding hands raw pointers to kernels, so a host tensor, a wrong dtype or a
    strided view is refused before the library is called (a host address given to a
    kernel would be an invalid device access)."""
    import numpy as np
    import torch

    api.load_library()
    m = torch.zeros(12, dtype=torch.float64)
    d = torch.zeros((12, 2), dtype=torch.float64)
    with pytest.raises(api.FlintsError, match="map must be a contiguous float64 CUDA tensor"):
        api.lens_noalloc(1, np.ones(33), m, d, m.clone(), K=16)

    class _Plan:  # stand-in: only the fields the job table reads
        spin, npix, handle = 2, 12, 0

    for job, msg in [((_Plan(), 0, 12, m, d, d, None, None), "job 0: map must be"),
                     ((_Plan(), 0, 0, None, None, None, None, None), None)]:
        if msg is None:  # an empty job carries no buffers
            api._job_array([job])
        else:
            with pytest.raises(api.FlintsError, match=msg):
                api._job_array([job])
    with pytest.raises(api.FlintsError, match="status must be a contiguous uint8 CUDA tensor"):
        api._dev_buf(torch.zeros(24, dtype=torch.uint8)[::2], 12, "status", "uint8")


C_LAYOUT = r"""
#include <stddef.h>
#include <stdio.h>
#include "flints.h"
#define F(T, f) printf(#T " " #f " %zu %zu\n", offsetof(T, f), sizeof(((T *)0)->f))
#define S(T) printf(#T " sizeof %zu 0\n", sizeof(T))
int main(void) {
    flints_plan_t h = 0;
    S(flints_stats); F(flints_stats, points); F(flints_stats, nugget); F(flints_stats, fallback);
    F(flints_stats, window); F(flints_stats, failed);
    S(flints_plan_info); F(flints_plan_info, nside); F(flints_plan_info, lmax); F(flints_plan_info, spin);
    F(flints_plan_info, K); F(flints_plan_info, precision); F(flints_plan_info, t_max);
    F(flints_plan_info, n_intervals); F(flints_plan_info, xi0); F(flints_plan_info, search_radius);
    F(flints_plan_info, device_bytes);
    S(flints_launch_cfg); F(flints_launch_cfg, warps_per_block); F(flints_launch_cfg, blocks_per_sm);
    F(flints_launch_cfg, tile_points);
    S(flints_job); F(flints_job, plan); F(flints_job, first); F(flints_job, count); F(flints_job, map);
    F(flints_job, defl); F(flints_job, out); F(flints_job, var); F(flints_job, status);
    S(flints_paper_info); F(flints_paper_info, nside); F(flints_paper_info, nside_coarse); F(flints_paper_info, y);
    F(flints_paper_info, K); F(flints_paper_info, slots); F(flints_paper_info, t_max);
    F(flints_paper_info, n_intervals); F(flints_paper_info, xi0); F(flints_paper_info, table_bytes);
    F(flints_paper_info, max_pair_t); F(flints_paper_info, nugget_slots); F(flints_paper_info, failed_slots);
    F(flints_paper_info, points); F(flints_paper_info, window); F(flints_paper_info, precision);
    F(flints_paper_info, spin); F(flints_paper_info, flags); F(flints_paper_info, device_bytes);
    printf("const FLINTS_FP64 %d\nconst FLINTS_MIXED %d\n", FLINTS_FP64, FLINTS_MIXED);
    printf("const FLINTS_SPIN2_AUGMENTED %u\nconst FLINTS_ROTATE_TO_TARGET %u\n", FLINTS_SPIN2_AUGMENTED,
           FLINTS_ROTATE_TO_TARGET);
    printf("const FLINTS_NO_VARIANCE %u\nconst FLINTS_FORCE_FALLBACK %u\n", FLINTS_NO_VARIANCE, FLINTS_FORCE_FALLBACK);
    printf("const ST_NUGGET %u\nconst ST_FALLBACK %u\nconst ST_WINDOW %u\n", FLINTS_ST_NUGGET, FLINTS_ST_FALLBACK,
           FLINTS_ST_WINDOW);
    printf("const ST_FAILED %u\nconst ST_POLE %u\nconst ST_INPUT %u\n", FLINTS_ST_FAILED, FLINTS_ST_POLE,
           FLINTS_ST_INPUT);
    /* argument checks run on the host: no device is touched */
    printf("call %d %s\n", flints_plan(&h, 0, 16, 0, 0, 0, 16, FLINTS_FP64, 0u, 0), flints_last_error());
    return h != 0;
}
"""


def test_header_is_c_and_its_layouts_match_the_binding(lib_path, tmp_path):
    """include/flints.h compiles as strict C99; a C program linked against the
    library sees the struct layouts and constants the ctypes binding uses (a field
    offset the binding got wrong would hand the library a garbled job or plan info),
    and gets FLINTS_EINVAL from a plan with Nside 0 without touching a device."""
    import os
    import shutil

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(C_LAYOUT)
    exe = tmp_path / "layout"
    libdir = os.path.dirname(lib_path)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(api.HEADER),
                        str(src), "-o", str(exe), "-L", libdir, "-lflints", f"-Wl,-rpath,{libdir}",
                        "-Wl,--allow-shlib-undefined"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    structs = {"flints_stats": api._Stats, "flints_plan_info": api._Info, "flints_launch_cfg": api.LaunchCfg,
               "flints_job": api._Job, "flints_paper_info": api._PaperInfo}
    seen = set()
    for line in out:
        kind, *rest = line.split()
        if kind in structs:
            field, off, size = rest[0], int(rest[1]), int(rest[2])
            cls = structs[kind]
            if field == "sizeof":
                assert ctypes.sizeof(cls) == off, kind
            else:
                desc = getattr(cls, field)
                assert (desc.offset, desc.size) == (off, size), (kind, field)
                seen.add((kind, field))
        elif kind == "const":
            name, value = rest
            assert getattr(api, name) == int(value), name
        else:
            assert kind == "call" and rest[0] == "1" and "nside" in " ".join(rest[1:]), line
    # every field the binding declares was checked against the header
    assert seen == {(k, f) for k, c in structs.items() for f, _ in c._fields_}


def _prototypes():
    """{name: (return type, [parameter types])} of the functions in include/flints.h,
    types as written with the parameter names removed."""
    import re

    txt = re.sub(r"/\*.*?\*/", "", open(api.HEADER).read(), flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"\b((?:const\s+)?[a-z_0-9]+\s*\*?)\s*(flints_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;",
                                        txt):
        types = []
        for p in params.split(","):
            p = " ".join(p.split())
            if p in ("", "void"):
                continue
            types.append(re.sub(r"\s*\b[A-Za-z_0-9]+$", "", p).replace(" *", "*"))
        protos[name] = (" ".join(ret.split()).replace(" *", "*"), types)
    return protos


def _ctype_of(c: str):
    """The ctypes class that passes a C type with the same calling convention."""
    if c.endswith("*") or c.endswith("_t") and c.startswith("flints_") or c == "void*":
        return "ptr"
    return {"int64_t": ctypes.c_int64, "int": ctypes.c_int, "unsigned": ctypes.c_uint, "double": ctypes.c_double,
            "void": None}[c]


def test_binding_signatures_match_the_header(lib_path):
    """The argtypes and restype the binding sets for every function of the header
    match its prototype: same parameter count, integers of the same width and
    signedness, pointers for pointers (a wrong width would pass garbage in a
    register)."""
    lib = api.load_library()
    protos = _prototypes()
    assert set(protos) == set(api.header_functions())
    checked = 0
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        checked += 1
        argtypes = fn.argtypes if fn.argtypes is not None else []  # none set: a (void) function
        assert len(argtypes) == len(params), (name, fn.argtypes, params)
        for a, c in zip(argtypes, params):
            want = _ctype_of(c)
            if want == "ptr":
                assert a is ctypes.c_void_p or a is ctypes.c_char_p or hasattr(a, "_type_") and issubclass(
                    a, ctypes._Pointer), (name, a, c)
            else:
                assert a is want, (name, a, c)
        r = _ctype_of(ret)
        if r == "ptr":
            assert fn.restype in (ctypes.c_char_p, ctypes.c_void_p), (name, fn.restype)
        else:
            assert fn.restype is (r if r is not None else None) or (r is ctypes.c_int and fn.restype is ctypes.c_int), \
                (name, fn.restype, ret)
    assert checked == len(protos)
