"""Compile sections of the library's device code for the host (test helper).

Device functions that only do arithmetic are cut out of the CUDA sources by
their banners or first lines, their ``__device__ __forceinline__`` qualifiers
replaced by ``inline``, and compiled with g++ next to correctly rounded host
stand-ins for the CUDA intrinsics they call: __fadd_rn is a + b in float,
__fmaf_rn is fmaf, and so on.  Three stand-ins are approximate on the device:
rsqrtf (2 ulp) is the correctly rounded value moved by 2 ulp so that the code
that refines it is tested at that bound, rsqrt (1 ulp) and __fdividef (2 ulp)
are the correctly rounded operations.  Warp shuffles either return the
calling thread's own value (sections that only declare them) or run on a
warp of 32 host threads that meet at every shuffle (warp-synchronous code)."""
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
using std::fma;
using std::sqrt;
"""

# Warp shuffles that return the calling thread's own value, for sections that
# only declare shuffles (in a struct they share with arithmetic under test).
WARP_IDENTITY = r"""
template <class T> static inline T __shfl_sync(unsigned, T v, int) { return v; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
"""

# A warp of 32 host threads that meet at every shuffle and __syncwarp (warp-
# synchronous code calls them convergently, in the same order in every lane):
# run_warp(f) calls f(lane) on 32 threads.  A shuffle publishes each lane's
# value, waits, reads the source lane's value and waits again before the slot
# is reused.
WARP_THREADS = r"""
#include <atomic>
#include <thread>
// the lanes' barrier: a generation count; waiting lanes yield their core
struct WarpBarrier {
    std::atomic<int> count{0};
    std::atomic<unsigned> gen{0};
    void arrive_and_wait() {
        const unsigned g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == 31) {
            count.store(0, std::memory_order_relaxed);
            gen.store(g + 1, std::memory_order_release);
        } else {
            while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }
};
static WarpBarrier *g_warp_bar = nullptr;
static thread_local int t_lane = 0;
static uint64_t g_warp_slot[32];
template <class T> static inline T __shfl_sync(unsigned, T v, int src) {
    static_assert(sizeof(T) <= 8, "one word per lane");
    uint64_t b = 0;
    std::memcpy(&b, &v, sizeof(T));
    g_warp_slot[t_lane] = b;
    g_warp_bar->arrive_and_wait();
    const uint64_t r = g_warp_slot[src & 31];
    g_warp_bar->arrive_and_wait();
    T out;
    std::memcpy(&out, &r, sizeof(T));
    return out;
}
template <class T> static inline T __shfl_xor_sync(unsigned m, T v, int x) { return __shfl_sync(m, v, t_lane ^ x); }
template <class T> static inline T __shfl_up_sync(unsigned m, T v, int d) {
    return __shfl_sync(m, v, t_lane >= d ? t_lane - d : t_lane);
}
static inline void __syncwarp(unsigned = 0xffffffffu) { g_warp_bar->arrive_and_wait(); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
template <class F> static void run_warp(F f) {
    WarpBarrier bar;
    g_warp_bar = &bar;
    std::vector<std::thread> th;
    for (int l = 0; l < 32; ++l) th.emplace_back([&f, l] { t_lane = l; f(l); });
    for (auto &t : th) t.join();
}
"""

# Further stand-ins for compiling a whole kernel header (csrc/lens.cuh) on the host
# warp: vector types, read-only loads, sincospi and sinpif as sin/cos of pi x (the
# device functions are within an ulp or two), bit casts, a warp ballot.
LENS_SHIM = r"""
#include <cstddef>
#include <type_traits>
#include <math.h>
#define __align__(x) alignas(x)
#define __device__
struct double2 { double x, y; };
static inline double2 make_double2(double x, double y) { return {x, y}; }
struct float4 { float x, y, z, w; };
template <class T> static inline T __ldg(const T *p) { return *p; }
static inline void sincospi(double x, double *s, double *c) { *s = std::sin(M_PI * x); *c = std::cos(M_PI * x); }
static inline float sinpif(float x) { return (float)std::sin(M_PI * (double)x); }
static inline double __longlong_as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
static inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static bool g_ballot_slot[32];
static inline unsigned __ballot_sync(unsigned, int pred) {
    g_ballot_slot[t_lane] = pred != 0;
    g_warp_bar->arrive_and_wait();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (unsigned)g_ballot_slot[l] << l;
    g_warp_bar->arrive_and_wait();
    return m;
}
template <class T> static inline T atomicAdd(T *p, T v) { T o = *p; *p += v; return o; }
using std::floor; using std::fabs; using std::fmax; using std::isfinite; using std::atan2;
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


# address sanitizer and the undefined-behaviour checks that matter for kernel code
# (array bounds, shifts, signed overflow); -O0 keeps the build short (the emulated
# barriers, not the arithmetic, set the run time) and, without contraction or
# fast-math, rounds exactly as the plain -O1 build does
SANITIZE = {
    "address": ["-fsanitize=address,bounds,shift,signed-integer-overflow", "-fno-sanitize-recover=all",
                "-fno-omit-frame-pointer", "-O0"],
    # data races between the emulated threads: two threads of a block touching the same
    # word, one of them writing, with no barrier between them
    "thread": ["-fsanitize=thread", "-O1"],
}


def build(tmpdir, name: str, text: str, warp: str = "identity", sanitize: str | None = None) -> str:
    """Compile ``SHIM`` + the warp stand-ins (``"identity"``, ``"threads"`` or none) +
    ``text`` into an executable (strict IEEE: no contraction or fast-math, so the
    optimisation level does not change a result; -O1 compiles the large sources
    quickly and runs as fast as -O2 here, where the emulated barriers set the pace;
    ``sanitize``: "address" or "thread", the run then fails on any finding)."""
    src = os.path.join(str(tmpdir), name + ".cpp")
    with open(src, "w") as f:
        f.write(SHIM + {"threads": WARP_THREADS, "identity": WARP_IDENTITY}.get(warp, "") + text)
    exe = os.path.join(str(tmpdir), name)
    r = subprocess.run([compiler(), "-std=c++20", "-O1", "-pthread", "-ffp-contract=off", "-fno-fast-math"]
                       + (SANITIZE[sanitize] if sanitize else []) + [src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run(exe: str, text: str) -> str:
    p = subprocess.run([exe], input=text, capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return p.stdout
