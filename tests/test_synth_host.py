"""The harmonic synthesis (csrc/synth.cu: flints_synth_plan, flints_synthesize;
the Wigner-d l-recurrence kernels in FP64 and double-float, the ring folding,
the Bluestein polar rings) run on the host through tests/cuda_host.py (its
cuFFT stand-in sums the ring transforms directly), with the kernels' threads
running freely between barriers, against the oracle's synthesis on whole
small skies: spin 0, the spin-1 gradient of a potential and spin-2 Q/U, with
band limits above 2 Nside so that the folding modulo the ring length runs,
and one above the kernels' 256-multipole staging chunk.
Tolerances as on the GPU: 1e-10 (FP64) and 1e-9 (double-float) of the map's
rms."""
import numpy as np
import pytest

import workloads as wl
from oracle import sht
from tests import cuda_host as ch
from tests import host_compile as hc

DRIVER = r"""
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
// Every argument check of the synthesis API; prints "rc|message" per refused call, then
// whether the output map is untouched.
static void reject() {
    auto rep = [](int rc) { printf("%d|%s\n", rc, flints_synth_last_error()); };
    flints_synth_t h = nullptr;
    rep(flints_synth_plan(nullptr, 8, 16, 0, 0, nullptr));
    rep(flints_synth_plan(&h, 0, 16, 0, 0, nullptr));
    rep(flints_synth_plan(&h, 8193, 16, 0, 0, nullptr));
    rep(flints_synth_plan(&h, 8, 16, 3, 0, nullptr));
    rep(flints_synth_plan(&h, 8, 1, 2, 0, nullptr));
    rep(flints_synth_plan(&h, 8, 16, 0, 2, nullptr));
    if (flints_synth_plan(&h, 8, 16, 2, 0, nullptr)) { printf("plan failed\n"); return; }
    static double buf[4096] __attribute__((aligned(64)));
    for (double &v : buf) v = std::nan("");
    static double map[2 * 768] __attribute__((aligned(64)));
    for (double &v : map) v = std::nan("");
    rep(flints_synthesize(nullptr, buf, nullptr, map, nullptr));
    rep(flints_synthesize(h, nullptr, nullptr, map, nullptr));
    rep(flints_synthesize(h, buf, nullptr, nullptr, nullptr));
    rep(flints_synthesize(h, buf + 1, nullptr, map, nullptr));
    rep(flints_synthesize(h, buf, buf + 1, map, nullptr));
    rep(flints_synthesize(h, buf, nullptr, map + 1, nullptr));
    printf("untouched %d\n", std::all_of(map, map + 2 * 768, [](double v) { return std::isnan(v); }) ? 1 : 0);
    flints_synth_free(h);
}

int main() {
    long long nside;
    int lmax, spin, prec, has_b;
    char op[16];
    while (scanf("%15s", op) == 1) {
        if (std::string(op) == "reject") {
            reject();
            continue;
        }
        if (scanf("%lld %d %d %d %d", &nside, &lmax, &spin, &prec, &has_b) != 5) return 2;
        const size_t na = (size_t)(lmax + 1) * (lmax + 1);
        std::vector<double> alm(2 * na), blm(2 * na, 0.0);
        for (double &v : alm) v = rd();
        if (has_b) for (double &v : blm) v = rd();
        const long long npix = 12 * nside * nside;
        std::vector<double> map(spin == 0 ? npix : 2 * npix, std::nan(""));
        flints_synth_t h = nullptr;
        int rc = flints_synth_plan(&h, nside, lmax, spin, prec, nullptr);
        if (rc == 0) rc = flints_synthesize(h, alm.data(), has_b ? blm.data() : nullptr, map.data(), nullptr);
        printf("%d\n", rc);
        if (rc != 0) { printf("%s\n", flints_synth_last_error()); continue; }
        for (double v : map) printf("%a\n", v);
        flints_synth_free(h);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    exe = ch.build(tmp_path_factory.mktemp("synth"), "synth_host", ["common.cuh", "synth.cu"], DRIVER)

    def call(nside, lmax, spin, prec, alm, blm=None):
        def flat(a):
            return " ".join(float(x).hex() for x in np.stack([a.real, a.imag], -1).ravel())

        line = f"synth {nside} {lmax} {spin} {prec} {0 if blm is None else 1} " + flat(alm) + (
            "" if blm is None else " " + flat(blm))
        lines = hc.run(exe, line + "\n").splitlines()
        assert lines[0] == "0", lines[:2]
        v = np.array([float.fromhex(t) for t in lines[1:]])
        return v if spin == 0 else v[0::2] + 1j * v[1::2]

    call.exe = exe
    return call


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


TOL = {0: 1e-10, 1: 1e-9}


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("nside,lmax", [(8, 16), (4, 20), (16, 24), (4, 300)])
def test_synthesis_matches_the_oracle(nside, lmax, prec, run):
    alm = wl.draw_alm(wl.cl_tt(lmax, 0.7 * lmax), 11 + nside)
    assert _rel(run(nside, lmax, 0, prec, alm), sht.synth_map(nside, lmax, alm)) <= TOL[prec]
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    e, b = wl.draw_alm(cl, 12 + nside), wl.draw_alm(0.4 * cl, 13 + nside)
    assert _rel(run(nside, lmax, 2, prec, e, b), sht.synth_map(nside, lmax, e, spin=2, blm=b)) <= TOL[prec]
    # spin 1: the gradient of a potential, E_lm = sqrt(l(l+1)) phi_lm
    phi = wl.draw_alm(wl.cl_phiphi(lmax), 14 + nside)
    ell = np.arange(lmax + 1)
    g = sht.synth_map(nside, lmax, phi, gradient=True)
    got = run(nside, lmax, 1, prec, phi * np.sqrt(ell * (ell + 1.0))[:, None])
    assert _rel(got, g[:, 0] + 1j * g[:, 1]) <= TOL[prec]


def test_invalid_calls_are_refused(run):
    """Every argument check of the synthesis API (plan sizes, spin, precision, null
    and misaligned buffers) returns FLINTS_EINVAL with a message naming the fault,
    and a refused synthesis leaves the output map untouched."""
    lines = hc.run(run.exe, "reject\n").splitlines()
    expect = ["out is NULL", "nside outside", "nside outside", "spin must be", "lmax outside", "precision must be",
              "plan is NULL", "alm and map must not be NULL", "alm and map must not be NULL", "16-byte aligned",
              "16-byte aligned", "16-byte aligned"]
    assert len(lines) == len(expect) + 1, lines
    for line, msg in zip(lines, expect):
        rc, text = line.split("|", 1)
        assert rc == "1" and msg in text, (line, msg)
    assert lines[-1] == "untouched 1"
