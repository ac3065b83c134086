"""Full-size parity and accuracy: Nside 2048 (spin 0) and Nside 4096 (spin 2),
lmax 4096, K = 32, in the launch configuration the benchmark times (batches of
2^24 consecutive targets of a resident whole-sky map).

The source map is a band-limited realisation synthesised exactly on bands of
rings around sampled target stretches (north cap, cap/belt transition,
equator, south cap), or around 10^4 seeded random pixels on rings drawn over
the whole sky; the GPU lenses the whole 2^24-target batches containing them,
and the sampled outputs are compared with
  * the FP64 oracle (same tabulated correlation function): parity metric
    max|gpu - oracle| / sigma_map <= 1e-9 (FP64 path), 1e-6 (mixed path);
  * the exact benchmark of Sec. 3.2, the spherical-harmonic sum at the
    displaced directions: relative L2 error (Sec. 3.2 / Table 2 definition),
    and measured error / predicted sigma ~ 1 (Fig. cmb_exp_error).
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests.gpu_common import oracle_table, parity_metric, require_gpu, to_host, unexplained_mismatches
from tests.paper_values import LENSED_L2_NSIDE4096, SUPERSAMPLE_2048_4096_9NGB

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
BATCH = 1 << 24


class BandMap:
    """Map values known on a sorted set of pixels, indexable like a RING array."""

    def __init__(self, pix, vals):
        o = np.argsort(pix)
        self.pix, self.vals = pix[o], vals[o]

    def __getitem__(self, key):
        idx, comp = key if isinstance(key, tuple) else (key, None)
        pos = np.searchsorted(self.pix, idx)
        assert np.all(self.pix[np.minimum(pos, self.pix.size - 1)] == idx), "stencil outside the synthesised band"
        v = self.vals[pos]
        return v if comp is None else v[..., comp]


def _bands(W, n_targets):
    """Four target stretches (north cap, cap/belt transition, equator, south cap): for each the
    first pixel, the count, the deflections of its whole 2^24-target batch and the
    rings its stencils reach (from the oracle's own search), plus one ring of margin."""
    out = []
    for ring in (W.nside // 2, W.nside + 3, 2 * W.nside, 4 * W.nside - W.nside // 3):
        first, n_in = [int(x[0]) for x in hp.ring_info(W.nside, np.array([ring]))[:2]]
        start = first + n_in // 3
        b0 = (start // BATCH) * BATCH
        bn = min(BATCH, W.npix - b0)
        defl = wl.random_deflection(bn, 1000 + b0 // BATCH)
        pix = np.arange(start, start + n_targets)
        tv = kr.displace(W.nside, pix, defl[start - b0:start - b0 + n_targets])
        idx, _ = kr.knn(W.nside, tv, W.K)
        r = hp.pix2ring(W.nside, idx.ravel())[0]
        out.append((start, n_targets, b0, bn, defl, np.arange(r.min() - 1, r.max() + 2)))
    return out


def _setup(W, n_targets):
    cl, bb = W.cl()
    alm = wl.draw_alm(cl, W.seed_map)
    bands = _bands(W, n_targets)
    pix_all, val_all = [], []
    for *_, rings in bands:
        p, v = sht.synth_rings(W.nside, rings, W.lmax, alm, spin=W.spin)
        pix_all.append(p)
        val_all.append(v if W.spin == 0 else np.stack([v.real, v.imag], axis=1))
    pix = np.concatenate(pix_all)
    vals = np.concatenate(val_all)
    return cl, bb, alm, bands, pix, vals


@pytest.fixture(scope="module")
def fl():
    return require_gpu()


@pytest.mark.parametrize("W", [wl.C2, wl.C3], ids=["c2", "c3"])
def test_fullsize_parity_and_exact_benchmark(fl, W):
    import torch

    n_targets = 1024
    cl, bb, alm, bands, pix, vals = _setup(W, n_targets)
    dev = torch.device("cuda")
    shape = (W.npix,) if W.spin == 0 else (W.npix, 2)
    m = torch.zeros(shape, dtype=torch.float64, device=dev)
    m[torch.from_numpy(pix).to(dev)] = torch.from_numpy(vals).to(dev)
    sigma = float(np.sqrt(np.mean(vals ** 2) * (1 if W.spin == 0 else 2)))
    tab, x0, _, _ = oracle_table(cl, bb, W.spin, W.K, W.nside)
    band_map = BandMap(pix, vals)
    results = {}
    variants = [("fp64", 0), ("mixed", 0)]
    if W.spin == 2:  # the augmented (xi+, xi-) estimator on the same bands
        variants += [("fp64-aug", fl.FLINTS_SPIN2_AUGMENTED), ("mixed-aug", fl.FLINTS_SPIN2_AUGMENTED)]
    for precision, flags in variants:
        plan = fl.Plan(W.nside, cl, bb, spin=W.spin, K=W.K, precision=precision.split("-")[0], flags=flags)
        got_v, got_s2 = [], []
        for first, count, b0, bn, defl_np, _ in bands:
            defl = torch.from_numpy(defl_np).to(dev)
            var = torch.empty(bn, dtype=torch.float64, device=dev)
            st = torch.empty(bn, dtype=torch.uint8, device=dev)
            out, var, st = plan.lens(m, defl, var=var, status=st, first=b0, count=bn)
            torch.cuda.synchronize()
            sl = slice(first - b0, first - b0 + count)
            o = to_host(out[sl])
            got_v.append(o if W.spin == 0 else o[:, 0] + 1j * o[:, 1])
            got_s2.append(to_host(var[sl]))
            assert int((st & fl.ST_FAILED).sum()) == 0
            if precision == "fp64":
                results.setdefault("defl", []).append(defl_np[sl])
        results[precision] = (np.concatenate(got_v), np.concatenate(got_s2))
        s = plan.stats()
        assert s["failed"] == 0 and s["window"] == 0, s
        plan.close()
    targets = np.concatenate([np.arange(b[0], b[0] + b[1]) for b in bands])
    defl = np.concatenate(results["defl"])
    ref = kr.lens(W.nside, W.K, W.spin, band_map, defl, targets, tab, x0)
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-6)):
        v, s2 = results[precision]
        assert parity_metric(v, ref.value, sigma) <= tol, precision
        assert parity_metric(s2, ref.variance, x0) <= tol, precision
    if W.spin == 2:
        _, t_max, n = oracle_table(cl, bb, W.spin, W.K, W.nside)[1:]
        tp, tm, _ = xi.spin2_tables(cl, bb, t_max, n)
        ref_aug = kr.lens(W.nside, W.K, 2, band_map, defl, targets, tp, x0, f_minus=tm)
        for precision, tol in (("fp64-aug", 1e-9), ("mixed-aug", 1e-6)):
            v, s2 = results[precision]
            assert parity_metric(v, ref_aug.value, sigma) <= tol, precision
            assert parity_metric(s2, ref_aug.variance, x0) <= tol, precision
    # exact benchmark on a subsample of the targets
    sub = np.arange(0, targets.size, 6)
    truth = sht.synth_points(W.lmax, alm, ref.target[sub], spin=W.spin)
    v = results["mixed"][0][sub]
    err = v - truth
    rel_l2 = math.sqrt(np.mean(np.abs(err) ** 2) / np.mean(np.abs(truth) ** 2))
    ratio = np.mean(np.abs(err) ** 2 / results["mixed"][1][sub])
    pred = math.sqrt(np.mean(results["mixed"][1][sub]) / np.mean(np.abs(truth) ** 2))
    print(f"{W.name}: rel L2 {rel_l2:.3e}, predicted {pred:.3e}, <|err|^2/sigma^2> {ratio:.3f}")
    if W.spin == 2:
        v_aug = results["mixed-aug"][0][sub]
        rel_aug = math.sqrt(np.mean(np.abs(v_aug - truth) ** 2) / np.mean(np.abs(truth) ** 2))
        print(f"{W.name}: augmented (xi+, xi-) rel L2 {rel_aug:.3e}")
        assert rel_aug <= LENSED_L2_NSIDE4096 and rel_aug <= 1.02 * rel_l2
    if W.name == "c3":
        # Nside 4096, lmax 4096: the paper's precision (Table 2, abstract).  Here the
        # 1.49e-8 nugget dominates the predicted variance (it models noisy data), so
        # the prediction is an upper bound rather than a match.
        assert rel_l2 <= LENSED_L2_NSIDE4096
        assert ratio < 1.5
    else:
        # Nside 2048: measured error / predicted sigma ~ 1 (Fig. cmb_exp_error)
        assert 0.6 < ratio < 1.5
        assert rel_l2 <= 3.0 * pred


def test_supersampling_2048_to_4096(fl):
    """Sec. 2.6 / Table 1 at full size: an Nside 2048 map (lmax 4096) predicted at
    the pixel centres of the Nside 4096 grid, K = 32, launched over whole 2^24-target
    batches; sampled outputs against the oracle and against the harmonic sum."""
    import torch

    W = wl.C2
    nout, n_targets = 2 * W.nside, 1024
    cl, bb = W.cl()
    alm = wl.draw_alm(cl, 91)
    stretches, rings = [], []
    for ring in (nout // 2, nout + 3, 2 * nout):
        first, n_in = [int(x[0]) for x in hp.ring_info(nout, np.array([ring]))[:2]]
        start = first + n_in // 3
        tv = hp.pix2vec(nout, np.arange(start, start + n_targets))
        idx, _ = kr.knn(W.nside, tv, W.K)
        r = hp.pix2ring(W.nside, idx.ravel())[0]
        rings.append(np.arange(r.min() - 1, r.max() + 2))
        stretches.append(start)
    pix_l, val_l = zip(*[sht.synth_rings(W.nside, rr, W.lmax, alm) for rr in rings])
    pix, vals = np.concatenate(pix_l), np.concatenate(val_l)
    dev = torch.device("cuda")
    m = torch.zeros(W.npix, dtype=torch.float64, device=dev)
    m[torch.from_numpy(pix).to(dev)] = torch.from_numpy(vals).to(dev)
    sigma = float(np.std(vals))
    tab, x0, _, _ = oracle_table(cl, bb, 0, W.K, W.nside)
    targets = np.concatenate([np.arange(s, s + n_targets) for s in stretches])
    ref = kr.supersample(W.nside, nout, W.K, 0, BandMap(pix, vals), targets, tab, x0)
    npix_out = 12 * nout * nout
    got = {}
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-6)):
        plan = fl.Plan(W.nside, cl, spin=0, K=W.K, precision=precision)
        v_l, s_l = [], []
        for s in stretches:
            b0 = (s // BATCH) * BATCH
            bn = min(BATCH, npix_out - b0)
            var = torch.empty(bn, dtype=torch.float64, device=dev)
            st = torch.empty(bn, dtype=torch.uint8, device=dev)
            out, var, st = plan.supersample(m, nout, var=var, status=st, first=b0, count=bn)
            torch.cuda.synchronize()
            sl = slice(s - b0, s - b0 + n_targets)
            v_l.append(to_host(out[sl]))
            s_l.append(to_host(var[sl]))
            assert int((st & fl.ST_FAILED).sum()) == 0
        v, s2 = np.concatenate(v_l), np.concatenate(s_l)
        # exact ties for the K-th place (symmetric centres): checked on every valid stencil
        bad = unexplained_mismatches(W.nside, W.K, 0, BandMap(pix, vals), ref.target, v, s2, ref, tab, x0, sigma,
                                     tol)
        assert bad == [], (precision, len(bad))
        got[precision] = (v, s2)
        plan.close()
    truth = sht.synth_points(W.lmax, alm, ref.target)
    v, s2 = got["mixed"]
    ratio = np.mean((v - truth) ** 2 / s2)
    pred = math.sqrt(np.mean(s2)) / sigma
    meas = math.sqrt(np.mean((v - truth) ** 2)) / sigma
    print(f"supersampling 2048 -> 4096: measured {meas:.3e}, predicted {pred:.3e} (Table 1 precision column)")
    assert 0.6 < ratio < 1.5
    assert meas < SUPERSAMPLE_2048_4096_9NGB  # K = 32 against the paper's 9-neighbour figure


def _whole_sky_sample(W, n_targets, seed):
    """n_targets seeded random pixels over the whole sky: 64 rings drawn uniformly in z
    (so that caps and belt are sampled by area) plus both poles' first rings, both
    cap/belt transitions and the equator, with random pixels on each ring; the source
    map is then synthesised exactly on the rings the stencils reach."""
    rng = np.random.default_rng(seed)
    N = W.nside
    z = rng.uniform(-1.0, 1.0, 64)
    rings = {int(r) for r in np.clip(hp.ring_above(N, z), 1, 4 * N - 1)}
    rings |= {1, 2, 4 * N - 2, 4 * N - 1, N - 1, N, N + 1, 3 * N - 1, 3 * N, 3 * N + 1, 2 * N}
    rings = np.array(sorted(rings))
    first, n_in = hp.ring_info(N, rings)[:2]
    per = n_targets // rings.size
    pix = []
    for f, n in zip(first, n_in):
        k = min(int(n), per)
        pix.append(int(f) + rng.choice(int(n), size=k, replace=False))
    pix = np.unique(np.concatenate(pix))
    while pix.size < n_targets:  # fill up with random pixels of the sampled rings (the pole rings are short)
        extra = n_targets - pix.size
        rr = rng.choice(rings.size, size=extra)
        cand = first[rr] + (rng.random(extra) * n_in[rr]).astype(np.int64)
        pix = np.unique(np.concatenate([pix, cand]))
    return pix[:n_targets]


@pytest.mark.parametrize("W", [wl.C2, wl.C3], ids=["c2", "c3"])
def test_exact_benchmark_on_random_pixels_over_the_whole_sky(fl, W):
    """Sec. 3.2 / Table 2 / abstract: the lensed map against the harmonic sum at the
    displaced directions, on 10^4 seeded random pixels over the whole sky (both caps,
    both cap/belt transitions, the equator): relative L2 <= 2e-4 at Nside 4096 (c3);
    at Nside 2048 (c2) the error matches the predicted variance (<|err|^2 / sigma^2>
    ~ 1, Fig. cmb_exp_error); the same pixels also give the parity of both GPU paths
    against the oracle."""
    import torch

    n_targets = 10_000
    cl, bb = W.cl()
    alm = wl.draw_alm(cl, W.seed_map)
    targets = _whole_sky_sample(W, n_targets, W.seed_sample)
    batches = np.unique(targets // BATCH)
    defl_b = {int(b): wl.random_deflection(min(BATCH, W.npix - int(b) * BATCH), 2000 + int(b)) for b in batches}
    defl = np.concatenate([defl_b[int(t // BATCH)][t - (t // BATCH) * BATCH][None, :] for t in targets])
    tv = kr.displace(W.nside, targets, defl)
    idx, _ = kr.knn(W.nside, tv, W.K)
    stencil_rings = np.unique(hp.pix2ring(W.nside, idx.ravel())[0])
    rings = np.unique(np.clip(np.concatenate([stencil_rings - 1, stencil_rings, stencil_rings + 1]), 1,
                              4 * W.nside - 1))
    p, v = sht.synth_rings(W.nside, rings, W.lmax, alm, spin=W.spin)
    vals = v if W.spin == 0 else np.stack([v.real, v.imag], axis=1)
    dev = torch.device("cuda")
    shape = (W.npix,) if W.spin == 0 else (W.npix, 2)
    m = torch.zeros(shape, dtype=torch.float64, device=dev)
    m[torch.from_numpy(p).to(dev)] = torch.from_numpy(vals).to(dev)
    sigma = float(np.sqrt(np.mean(vals ** 2) * (1 if W.spin == 0 else 2)))
    tab, x0, _, _ = oracle_table(cl, bb, W.spin, W.K, W.nside)
    got = {}
    for precision in ("fp64", "mixed"):
        plan = fl.Plan(W.nside, cl, bb, spin=W.spin, K=W.K, precision=precision)
        v_all = np.empty(n_targets, dtype=np.float64 if W.spin == 0 else np.complex128)
        s_all = np.empty(n_targets)
        for b in batches:
            b0 = int(b) * BATCH
            bn = min(BATCH, W.npix - b0)
            out, var, st = plan.lens(m, torch.from_numpy(defl_b[int(b)]).to(dev),
                                     var=torch.empty(bn, dtype=torch.float64, device=dev),
                                     status=torch.empty(bn, dtype=torch.uint8, device=dev), first=b0, count=bn)
            torch.cuda.synchronize()
            sel = np.nonzero(targets // BATCH == b)[0]
            loc = torch.from_numpy(targets[sel] - b0).to(dev)
            o = to_host(out[loc])
            v_all[sel] = o if W.spin == 0 else o[:, 0] + 1j * o[:, 1]
            s_all[sel] = to_host(var[loc])
            assert int((st[loc] & fl.ST_FAILED).sum()) == 0
        s = plan.stats()
        assert s["failed"] == 0 and s["window"] == 0, s
        got[precision] = (v_all, s_all)
        plan.close()
    ref = kr.lens(W.nside, W.K, W.spin, BandMap(p, vals), defl, targets, tab, x0)
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-6)):
        v, s2 = got[precision]
        assert parity_metric(v, ref.value, sigma) <= tol, precision
        assert parity_metric(s2, ref.variance, x0) <= tol, precision
    truth = sht.synth_points(W.lmax, alm, ref.target, spin=W.spin)
    south = ref.target[:, 2] < 0
    for precision in ("fp64", "mixed"):
        v, s2 = got[precision]
        err = v - truth
        rel_l2 = math.sqrt(np.mean(np.abs(err) ** 2) / np.mean(np.abs(truth) ** 2))
        rel_s = math.sqrt(np.mean(np.abs(err[south]) ** 2) / np.mean(np.abs(truth[south]) ** 2))
        ratio = float(np.mean(np.abs(err) ** 2 / s2))
        print(f"{W.name} whole sky, {n_targets} random pixels ({south.sum()} south), {precision}: "
              f"rel L2 {rel_l2:.3e} (south {rel_s:.3e}), <|err|^2/sigma^2> {ratio:.3f}")
        if W.name == "c3":
            assert rel_l2 <= LENSED_L2_NSIDE4096 and rel_s <= LENSED_L2_NSIDE4096, precision
            # the nugget dominates the predicted variance at Nside 4096 and bounds the error
            # from above; the oracle on this sample gives <|err|^2/sigma^2> = 0.158
            assert 0.1 < ratio < 0.25, precision
        else:
            # the standardised error (v - truth) / sigma ~ N(0, 1) (Sec. 3.2, Fig. cmb_exp_error);
            # the oracle on this sample gives mean -0.007, std 0.972
            r = err / np.sqrt(s2)
            assert abs(np.mean(r)) < 0.05 and 0.9 < np.std(r) < 1.1, (precision, np.mean(r), np.std(r))
            assert 0.8 < ratio < 1.25, precision
