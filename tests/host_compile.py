"""Compile sections of the library's device code for the host (test helper).

Device functions that only do arithmetic are cut out of the CUDA sources by
their banners or first lines, their ``__device__ __forceinline__`` qualifiers
replaced by ``inline``, and compiled with g++ next to correctly rounded host
stand-ins for the CUDA intrinsics they call: __fadd_rn is a + b in float,
__fmaf_rn is fmaf, and so on.  Three stand-ins are approximate on the device:
rsqrtf (2 ulp) is the correctly rounded value moved by 2 ulp so that the code
that refines it is tested at that bound, rsqrt (1 ulp) and __fdividef (2 ulp)
are the correctly rounded operations.  Warp shuffles return the calling
thread's own value: the sections compiled here do not use them."""
from __future__ import annotations

import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1003_4984_gb300", "csrc")

SHIM = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fdiv_rn(float a, float b) { volatile float r = a / b; return r; }
static inline float __fdividef(float a, float b) { volatile float r = a / b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline float __fsqrt_rn(float a) { return std::sqrt(a); }
static inline float __frcp_rn(float a) { volatile float r = 1.0f / a; return r; }
// rsqrtf: 1/sqrt(a) moved by 2 ulp (down or up with the input's last bit)
static inline float rsqrtf(float a) {
    float f = (float)(1.0 / std::sqrt((double)a));
    unsigned u, ua;
    std::memcpy(&u, &f, 4);
    std::memcpy(&ua, &a, 4);
    u = (ua & 1u) ? u + 2u : u - 2u;
    std::memcpy(&f, &u, 4);
    return f;
}
static inline double rsqrt(double a) { volatile double r = 1.0 / std::sqrt(a); return r; }
static inline float __double2float_rn(double x) { volatile float r = (float)x; return r; }
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
template <class T> static inline T __shfl_sync(unsigned, T v, int) { return v; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
using std::fma;
using std::sqrt;
"""


def cut(path: str, start: str, stop: str, drop_banner: bool = True) -> str:
    """The text of ``path`` from ``start`` up to ``stop`` (the comment banner of the
    next section dropped), with device qualifiers removed."""
    src = open(os.path.join(CSRC, path)).read()
    a = src.index(start)
    b = src.index(stop, a)
    body = src[a:b]
    if drop_banner and "// ----" in body:
        body = body[:body.rindex("// ----")]
    return body.replace("__device__ __forceinline__", "inline")


def compiler() -> str | None:
    return shutil.which("g++") or shutil.which("c++")


def build(tmpdir, name: str, text: str) -> str:
    """Compile ``SHIM + text`` into an executable (strict IEEE: no contraction)."""
    src = os.path.join(str(tmpdir), name + ".cpp")
    with open(src, "w") as f:
        f.write(SHIM + text)
    exe = os.path.join(str(tmpdir), name)
    r = subprocess.run([compiler(), "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run(exe: str, text: str) -> str:
    p = subprocess.run([exe], input=text, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return p.stdout
