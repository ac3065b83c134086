"""The paper's stencil with tabulated inverses, run through its own C API
(flints_paper_plan, flints_paper_lens in csrc/paper.cu) on the host: the
plan's kernels (pixel tables, stencils and classes, the per-class L^-1 in a
64-thread block with __syncthreads) and the apply kernels (128-thread blocks
of warp-synchronous code) execute on host threads that run freely between
barriers (tests/cuda_host.py), so a missing __syncthreads or __syncwarp shows
as a wrong result.  Results are compared with the oracle's class route (Secs.
2.3-2.5) on whole skies at Nside 8 and 16, spin 0 and 2, levels y = 1 (9
pixels) and 2 (36 pixels), FP64 and mixed, and the augmented spin-2
estimator; tolerances as on the GPU (1e-9 FP64, 1e-6 mixed, of sigma_map and
xi(0))."""

import numpy as np
import pytest

import workloads as wl
from oracle import faces as fc
from oracle import healpix as hp
from oracle import sht
from oracle import xi
from tests import cuda_host as ch
from tests import host_compile as hc

DRIVER = r"""
namespace flints {
int device_sm_count() { return 152; }
size_t device_smem_optin() { return 232448; }
}
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
// Every argument check of the paper API on plans of spin 0 (FP64) and spin 2 (mixed): each
// call is refused before any launch or copy; prints "rc|message" per call, then whether the
// output buffers are untouched.
static void reject(long long nside, int lmax) {
    std::vector<double> cl(lmax + 1);
    for (double &v : cl) v = rd();
    flints_paper_t p0 = nullptr, p2 = nullptr;
    if (flints_paper_plan(&p0, nside, lmax, cl.data(), nullptr, 1, 0, 0, 0, nullptr) ||
        flints_paper_plan(&p2, nside, lmax, cl.data(), nullptr, 1, 2, 1, 0, nullptr)) {
        printf("plan failed: %s\n", flints_paper_last_error());
        return;
    }
    const long long npix = 12 * nside * nside;
    static double buf[4096] __attribute__((aligned(64)));
    for (double &v : buf) v = std::nan("");
    static uint8_t st[256];
    std::memset(st, 255, sizeof st);
    static int32_t mem[1 << 16];
    std::fill(mem, mem + (1 << 16), -7);
    double *m = buf, *d = buf + 2048, *out = buf + 3072, *var = buf + 3584;
    auto shift = [](const void *q, int by) { return (double *)((const char *)q + by); };
    auto rep = [](int rc) { printf("%d|%s\n", rc, flints_paper_last_error()); };
    flints_paper_info info{};
    rep(flints_paper_lens(nullptr, 0, 4, m, d, out, var, st, nullptr));
    rep(flints_paper_lens(p0, -1, 4, m, d, out, var, st, nullptr));
    rep(flints_paper_lens(p0, npix - 2, 4, m, d, out, var, st, nullptr));
    rep(flints_paper_lens(p0, 0, 4, nullptr, d, out, var, st, nullptr));
    rep(flints_paper_lens(p0, 0, 4, m, nullptr, out, var, st, nullptr));
    rep(flints_paper_lens(p0, 0, 4, m, shift(d, 8), out, var, st, nullptr));
    rep(flints_paper_lens(p2, 0, 4, shift(m, 8), d, out, var, st, nullptr));
    rep(flints_paper_lens(p2, 0, 4, m, d, shift(out, 8), var, st, nullptr));
    rep(flints_paper_lens(p0, 0, 4, m, d, out, shift(var, 4), st, nullptr));
    rep(flints_paper_supersample(p0, 0, 0, 4, m, out, var, st, nullptr));
    rep(flints_paper_supersample(p0, 16385, 0, 4, m, out, var, st, nullptr));
    rep(flints_paper_supersample(p0, 2 * nside, 4 * npix - 1, 2, m, out, var, st, nullptr));
    rep(flints_paper_get_info(p0, nullptr, nullptr));
    rep(flints_paper_tables(nullptr, mem, nullptr, nullptr, nullptr));
    rep(flints_paper_tables(p2, mem, mem + (1 << 15), buf + 3072, nullptr));
    // empty ranges are accepted with any buffers and launch nothing
    rep(flints_paper_lens(p0, npix, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
    rep(flints_paper_supersample(p2, 2 * nside, 5, 0, nullptr, nullptr, nullptr, nullptr, nullptr));
    const bool untouched = std::all_of(buf + 3072, buf + 4096, [](double v) { return std::isnan(v); }) &&
                           std::all_of(st, st + 256, [](uint8_t v) { return v == 255; }) &&
                           std::all_of(mem, mem + (1 << 16), [](int32_t v) { return v == -7; });
    flints_paper_get_info(p0, &info, nullptr);
    printf("untouched %d points %lld\n", untouched ? 1 : 0, (long long)info.points);
    flints_paper_free(p0);
    flints_paper_free(p2);
}

// Device memory of plans of every kind: what the plan reports (table_bytes and
// device_bytes), what it allocated (the runtime stand-in's ledger) and what
// flints_paper_free returns.
static void bytes(long long nside, int lmax) {
    std::vector<double> cl(lmax + 1);
    for (double &v : cl) v = rd();
    const int kinds[6][4] = {{1, 0, 0, 0}, {2, 0, 1, 0}, {1, 1, 1, 0}, {2, 2, 0, 0}, {1, 2, 1, 0}, {2, 2, 0, 1}};
    for (const auto &k : kinds) {  // y, spin, precision, flags
        flints_paper_t p = nullptr;
        const size_t live = g_dev_live;
        const int rc = flints_paper_plan(&p, nside, lmax, cl.data(), nullptr, k[0], k[1], k[2], (unsigned)k[3],
                                         nullptr);
        flints_paper_info i{};
        if (rc == 0) flints_paper_get_info(p, &i, nullptr);
        const size_t held = g_dev_live;
        flints_paper_free(p);
        printf("%d %lld %lld %lld %lld\n", rc, (long long)i.table_bytes, (long long)i.device_bytes,
               (long long)(held - live), (long long)(held - g_dev_live));
    }
}

int main() {
    long long nside;
    int lmax, y, spin, prec, flags, has_bb;
    char op[16];
    while (scanf("%15s", op) == 1) {
        if (std::string(op) == "bytes") {
            if (scanf("%lld %d", &nside, &lmax) != 2) return 2;
            bytes(nside, lmax);
            continue;
        }
        if (std::string(op) == "reject") {
            if (scanf("%lld %d", &nside, &lmax) != 2) return 2;
            reject(nside, lmax);
            continue;
        }
        if (scanf("%lld %d %d %d %d %d %d", &nside, &lmax, &y, &spin, &prec, &flags, &has_bb) != 7) return 2;
        std::vector<double> cl(lmax + 1), bb(lmax + 1);
        for (double &v : cl) v = rd();
        if (has_bb) for (double &v : bb) v = rd();
        const long long npix = 12 * nside * nside;
        const int comp = spin == 0 ? 1 : 2;
        std::vector<double> map(npix * comp), defl(2 * npix), out(npix * comp), var(npix);
        std::vector<uint8_t> status(npix);
        for (double &v : map) v = rd();
        for (double &v : defl) v = rd();
        flints_paper_t h = nullptr;
        int rc = flints_paper_plan(&h, nside, lmax, cl.data(), has_bb ? bb.data() : nullptr, y, spin, prec, flags,
                                   nullptr);
        if (rc == 0) {
            const size_t a0 = g_dev_alloc_calls;
            rc = flints_paper_lens(h, 0, npix, map.data(), defl.data(), out.data(), var.data(), status.data(), nullptr);
            if (g_dev_alloc_calls != a0) return 5;  // the per-call path allocates nothing
        }
        printf("%d\n", rc);
        if (rc != 0) { printf("%s\n", flints_paper_last_error()); continue; }
        for (long long p = 0; p < npix; ++p) {
            printf("%d %a %a", (int)status[p], out[p * comp], var[p]);
            if (comp == 2) printf(" %a", out[p * comp + 1]);
            printf("\n");
        }
        flints_paper_free(h);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    exe = ch.build(tmp_path_factory.mktemp("paper"), "paper_host",
                   ["common.cuh", "lens.cuh", "paper_geom.cuh", "xi_table.cu", "paper.cu"], DRIVER)

    def call(nside, lmax, y, spin, prec, flags, cl, bb, m, defl):
        head = f"lens {nside} {lmax} {y} {spin} {prec} {flags} {0 if bb is None else 1} "
        body = " ".join(x.hex() for x in cl) + ("" if bb is None else " " + " ".join(x.hex() for x in bb))
        body += " " + " ".join(float(x).hex() for x in np.ravel(m)) + " " + " ".join(float(x).hex() for x in np.ravel(defl))
        lines = hc.run(exe, head + body + "\n").splitlines()
        assert lines[0] == "0", lines[:2]
        rows = [ln.split() for ln in lines[1:]]
        status = np.array([int(r[0]) for r in rows])
        out = np.array([float.fromhex(r[1]) for r in rows])
        if spin:
            out = out + 1j * np.array([float.fromhex(r[3]) for r in rows])
        return status, out, np.array([float.fromhex(r[2]) for r in rows])

    call.exe = exe
    return call


CASES = [(0, 8, 16, 1), (0, 16, 32, 1), (0, 16, 32, 2), (2, 16, 32, 1), (2, 16, 32, 2)]


@pytest.mark.parametrize("spin,nside,lmax,y", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_paper_route_matches_the_oracle(spin, nside, lmax, y, prec, run):
    npix = hp.npix(nside)
    seed = 100 * nside + 10 * y + spin
    if spin == 0:
        cl, bb = wl.cl_tt(lmax, 0.7 * lmax), None
        m = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed))
        sigma = float(np.std(m))
    else:
        cl = wl.cl_ee(lmax, 0.7 * lmax)
        bb = 0.3 * cl
        P = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed), spin=2, blm=wl.draw_alm(bb, seed + 1))
        m = np.stack([P.real, P.imag], axis=1)
        sigma = float(np.sqrt(np.mean(np.abs(P) ** 2)))
    defl = wl.random_deflection(npix, seed + 2, rms=0.5 * np.sqrt(4 * np.pi / npix))
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tab, x0 = xi.spin0_table(cl, t_max, n) if spin == 0 else xi.spin2_tables(cl, bb, t_max, n)[::2]
    rv, rs2, _, _ = fc.paper_lens(nside, y, m, defl, np.arange(npix), tab, x0, classes=True, spin=spin)
    status, v, s2 = run(nside, lmax, y, spin, prec, 0, cl, bb, m, defl)
    tol = 1e-9 if prec == 0 else 1e-6
    assert np.all(status & (4 | 8) == 0)  # no window or failed points
    assert np.max(np.abs(v - rv)) <= tol * sigma, np.max(np.abs(v - rv)) / sigma
    assert np.max(np.abs(s2 - rs2)) <= tol * x0, np.max(np.abs(s2 - rs2)) / x0


@pytest.mark.parametrize("nside,lmax,y", [(8, 16, 1), (16, 32, 2)])
def test_augmented_paper_route_matches_the_oracle(nside, lmax, y, run):
    npix = hp.npix(nside)
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    bb = 0.3 * cl
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, 7 + nside), spin=2, blm=wl.draw_alm(bb, 8 + nside))
    m = np.stack([P.real, P.imag], axis=1)
    sigma = float(np.sqrt(np.mean(np.abs(P) ** 2)))
    defl = wl.random_deflection(npix, 9 + nside, rms=0.5 * np.sqrt(4 * np.pi / npix))
    t_max, n = fc.paper_grid_rule(cl, nside, y, bb)
    tp, tm, x0 = xi.spin2_tables(cl, bb, t_max, n)
    rv, rs2, _, _ = fc.paper_lens(nside, y, m, defl, np.arange(npix), tp, x0, classes=True, spin=2, f_minus=tm)
    status, v, s2 = run(nside, lmax, y, 2, 0, 1, cl, bb, m, defl)  # flags: FLINTS_SPIN2_AUGMENTED
    assert np.all(status & (4 | 8) == 0)
    assert np.max(np.abs(v - rv)) <= 1e-9 * sigma and np.max(np.abs(s2 - rs2)) <= 1e-9 * x0


def test_invalid_calls_are_refused_before_any_launch(run):
    """Every argument check of the paper API (null and out-of-range arguments,
    misaligned buffers, supersampling grids, the L^-1 copy a mixed plan cannot
    give) returns FLINTS_EINVAL with a message naming the fault, before any
    launch or copy: the output buffers stay untouched and no point is counted.
    Empty ranges succeed with any buffers."""
    cl = wl.cl_tt(16, 12.0)
    lines = hc.run(run.exe, "reject 8 16 " + " ".join(x.hex() for x in cl) + "\n").splitlines()
    expect = ["plan is NULL", "target range", "target range", "map and out must not be NULL", "defl is NULL",
              "16-byte aligned", "16-byte aligned", "16-byte aligned", "8-byte", "nside_out must be positive",
              "nside_out 16385 outside", "target range", "must not be NULL", "plan is NULL",
              "mixed plans keep only double-float", None, None]
    assert len(lines) == len(expect) + 1, lines
    for line, msg in zip(lines, expect):
        rc, text = line.split("|", 1)
        assert (rc == "0") if msg is None else (rc == "1" and msg in text), (line, msg)
    assert lines[-1] == "untouched 1 points 0", lines[-1]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_nonfinite_deflections_on_the_tabulated_route(prec, run):
    """NaN and infinite deflections on the tabulated route: FLINTS_ST_INPUT |
    FLINTS_ST_FAILED and NaN outputs there, every other target bit-identical to the
    run with the finite deflections (the 128-thread apply blocks keep their barriers
    with bad lanes among them)."""
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 0.7 * lmax)
    m = sht.synth_map(nside, lmax, wl.draw_alm(cl, 71))
    defl = wl.random_deflection(npix, 72, rms=0.5 * np.sqrt(4 * np.pi / npix))
    bad = np.array([0, 1, 33, 130, 131, npix - 1])
    d_bad = defl.copy()
    d_bad[bad[0], 0] = np.nan
    d_bad[bad[1], 1] = np.inf
    d_bad[bad[2]] = [-np.inf, 0.0]
    d_bad[bad[3]] = [np.nan, np.nan]
    d_bad[bad[4], 1] = -np.inf
    d_bad[bad[5], 0] = np.inf
    st0, v0, s0 = run(nside, lmax, 1, 0, prec, 0, cl, None, m, defl)
    st, v, s2 = run(nside, lmax, 1, 0, prec, 0, cl, None, m, d_bad)
    good = np.setdiff1d(np.arange(npix), bad)
    assert np.all(st[bad] & (32 | 8) == 32 | 8) and np.all(st[good] == st0[good])
    assert np.all(np.isnan(v[bad])) and np.all(np.isnan(s2[bad]))
    np.testing.assert_array_equal(v[good], v0[good])
    np.testing.assert_array_equal(s2[good], s0[good])


def test_plans_report_the_device_memory_they_hold(run):
    """flints_paper_get_info's device_bytes equals what flints_paper_plan allocated
    (counted by the runtime stand-in) and what flints_paper_free returns, for spin 0,
    1 and 2, y = 1 and 2, FP64, mixed and augmented plans; table_bytes (pixel,
    stencil and class tables, L^-1 blocks) is part of it."""
    for nside in (8, 16):
        cl = wl.cl_tt(32, 22.0)
        lines = hc.run(run.exe, f"bytes {nside} 32 " + " ".join(x.hex() for x in cl) + "\n").splitlines()
        assert len(lines) == 6
        for line in lines:
            rc, table, dev, alloc, freed = map(int, line.split())
            assert rc == 0 and 0 < table < dev == alloc == freed, (nside, line)
