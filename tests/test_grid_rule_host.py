"""The library's correlation-table grid (table_grid in csrc/api.cu, the host
function that flints_plan and flints_lens_noalloc share) compiled for the
host and compared with the oracle's independent statement of the same rule
(oracle.xi.grid_rule): the same domain t_max and the same interval count on
the workloads' spectra and on edge cases (the 64-interval floor, the 65536
cap, negative and zero spectra, B-mode terms).  FP64 parity at 1e-9 rests on
both sides tabulating xi on the same grid."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as wl
from oracle import xi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1003_4984_gb300", "csrc")

DRIVER = r"""
int main() {
    long long nside;
    int K, lmax, has_bb;
    char b[64];
    while (scanf("%lld %d %d %d", &nside, &K, &lmax, &has_bb) == 4) {
        std::vector<double> cl(lmax + 1), bb(lmax + 1);
        for (int l = 0; l <= lmax; ++l) { if (scanf("%63s", b) != 1) return 2; cl[l] = strtod(b, nullptr); }
        if (has_bb)
            for (int l = 0; l <= lmax; ++l) { if (scanf("%63s", b) != 1) return 2; bb[l] = strtod(b, nullptr); }
        const flints::TableGrid g = flints::table_grid(nside, K, lmax, cl.data(), has_bb ? bb.data() : nullptr);
        printf("%d %a %a %d\n", g.n, g.t_max, g.r, g.R_rings);
    }
    return 0;
}
"""


def _block(src: str, start: str) -> str:
    """Text of the declaration or definition that begins with ``start``, up to its
    matching closing brace (and the semicolon of a struct)."""
    a = src.index(start)
    depth, k = 0, src.index("{", a)
    while True:
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                break
        k += 1
    end = k + 1
    if src[end:end + 1] == ";":
        end += 1
    return src[a:end]


@pytest.fixture(scope="module")
def grid(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    common = open(os.path.join(CSRC, "common.cuh")).read()
    api = open(os.path.join(CSRC, "api.cu")).read()
    pi_line = next(ln for ln in common.splitlines() if ln.startswith("constexpr double PI"))
    text = ("#include <cmath>\n#include <cstdint>\n#include <cstdio>\n#include <cstdlib>\n#include <vector>\n"
            "namespace flints {\n" + pi_line + "\n" + _block(common, "struct TableGrid {") + "\n"
            + _block(api, "TableGrid table_grid(") + "\n}\n" + DRIVER)
    d = tmp_path_factory.mktemp("grid")
    (d / "grid_host.cpp").write_text(text)
    exe = d / "grid_host"
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", str(d / "grid_host.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    def call(cases):
        lines = []
        for nside, K, cl, bb in cases:
            lines.append(f"{nside} {K} {cl.size - 1} {0 if bb is None else 1} " + " ".join(x.hex() for x in cl)
                         + ("" if bb is None else " " + " ".join(x.hex() for x in bb)))
        p = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
        return [(int(t[0]), float.fromhex(t[1]), float.fromhex(t[2]), int(t[3]))
                for t in (ln.split() for ln in p.stdout.splitlines())]

    return call


def _cases():
    out = []
    for W in (wl.C1, wl.C2, wl.C3):
        cl, bb = W.cl()
        out.append((W.nside, W.K, cl, bb))
    for m in wl.batched_maps(64):
        cl = wl.cl_tt(m.lmax, m.l_damp) if m.spin == 0 else wl.cl_ee(m.lmax, m.l_damp)
        out.append((m.nside, m.K, cl, np.zeros_like(cl) if m.spin == 2 else None))
    cl = wl.cl_ee(64, 20.0)
    out.append((32, 24, cl, 0.3 * cl))                       # a B-mode term adds |C^BB|
    out.append((32, 24, cl, wl.cl_ee(64, 1e4)))               # ... and one of another shape moves the grid
    out.append((16, 16, wl.cl_tt(8, 5.0), None))              # band limit far below the grid: the floor
    out.append((4, 48, wl.cl_tt(16384, 1e5), None))           # coarse grid, huge lmax: the cap
    out.append((64, 32, -wl.cl_tt(128, 100.0), None))         # magnitudes count
    out.append((64, 32, np.zeros(129), None))                 # no power at all
    out.append((8192, 32, wl.cl_tt(8192, 5000.0), None))
    for K in (16, 24, 32, 48):
        for nside in (1, 2, 256, 16384):
            out.append((nside, K, wl.cl_tt(min(2 * nside, 4096), 0.61 * min(2 * nside, 4096)), None))
    return out


def test_library_grid_equals_the_oracle_grid(grid):
    cases = _cases()
    got = grid(cases)
    ns = set()
    for (nside, K, cl, bb), (n, t_max, r, R_rings) in zip(cases, got):
        weight = np.abs(cl) + (np.abs(bb) if bb is not None else 0.0)
        t_ref, n_ref = xi.grid_rule(weight, K, nside)
        assert n == n_ref, (nside, K, cl.size - 1, n, n_ref)
        assert t_max == t_ref and t_max == 4 * r * r
        ns.add(n)
    assert 64 in ns and 65536 in ns and len(ns) >= 5  # floor, cap and several sizes between
