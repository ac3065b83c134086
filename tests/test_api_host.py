"""The K-nearest path's C API (csrc/api.cu, noalloc.cu and the kernels they
launch) run on the host through tests/cuda_host.py: plans, range and whole-map
lensing (spin 0 and 2 go through the persistent class kernel with a one-job
table, as on the GPU), the stencil entry point, supersampling, batches (the
convenience call and the batch objects), statistics and the no-allocation
entry point, with the kernels' threads running freely between barriers.
Results are compared with the FP64 oracle (whole skies at Nside 8 and 16,
and a band of the Nside 4096 spin-2 workload) within the GPU tolerances, and
the alternative entry points with each other (identical, as they run the
same per-tile code).  Every run also checks, at exit, that the per-call entry
points (lensing, supersampling, stencils, staging and launching a batch, the
no-allocation call) made no device allocation and that flints_free returned
what the plans reported holding."""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import sht
from oracle import xi
from tests import cuda_host as ch
from tests import host_compile as hc

DRIVER = r"""
#include <map>
#include <sys/mman.h>
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
static long long rl() { long long v; if (scanf("%lld", &v) != 1) exit(2); return v; }
static std::map<long long, flints_plan_t> g_plans;
static int g_hot_allocs = 0;  // per-call entry points that allocated device memory (none may)
static std::map<long long, double *> g_maps;
struct Buffers {
    std::vector<double> defl, out, var;
    std::vector<uint8_t> status;
};
static Buffers read_job(long long count, int comp) {
    Buffers b;
    b.defl.resize(2 * count);
    for (double &v : b.defl) v = rd();
    b.out.assign(comp * count, std::nan(""));
    b.var.assign(count, std::nan(""));
    b.status.assign(count, 255);
    return b;
}
static void print_rows(const Buffers &b, long long count, int comp) {
    for (long long p = 0; p < count; ++p)
        printf("%d %a %a %a\n", (int)b.status[p], b.out[comp * p], comp == 2 ? b.out[2 * p + 1] : 0.0, b.var[p]);
}
static int spin_of(flints_plan_t p) {
    flints_plan_info i;
    flints_get_info(p, &i);
    return i.spin;
}
int main() {
    char op[16];
    while (scanf("%15s", op) == 1) {
        const std::string o(op);
        if (o == "plan") {
            const long long id = rl(), nside = rl();
            const int lmax = (int)rl(), spin = (int)rl(), K = (int)rl(), prec = (int)rl(), flags = (int)rl(),
                      has_bb = (int)rl();
            std::vector<double> cl(lmax + 1), bb(lmax + 1);
            for (double &v : cl) v = rd();
            if (has_bb) for (double &v : bb) v = rd();
            flints_plan_t p = nullptr;
            const size_t live = g_dev_live;
            const int rc = flints_plan(&p, nside, lmax, cl.data(), has_bb ? bb.data() : nullptr, spin, K, prec,
                                       (unsigned)flags, nullptr);
            g_plans[id] = p;
            flints_plan_info i{};
            if (rc == 0) flints_get_info(p, &i);
            // the plan's reported device bytes, and what it allocated
            printf("%d %a %d %a %lld %lld\n", rc, i.t_max, i.n_intervals, i.xi0, (long long)i.device_bytes,
                   (long long)(g_dev_live - live));
        } else if (o == "launch") {  // plan warps_per_block blocks_per_sm tile_points
            flints_plan_t p = g_plans[rl()];
            flints_launch_cfg cfg{(int)rl(), (int)rl(), (int)rl()};
            printf("%d\n", flints_plan_set_launch(p, &cfg));
        } else if (o == "map") {  // id nside comp n, then n pixel indices and n * comp values
            const long long id = rl(), nside = rl(), comp = rl(), n = rl();
            const size_t bytes = (size_t)12 * nside * nside * comp * sizeof(double);
            double *m = static_cast<double *>(
                mmap(nullptr, bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS | MAP_NORESERVE, -1, 0));
            std::vector<long long> pix(n);
            for (long long &v : pix) v = rl();
            const long long lo = *std::min_element(pix.begin(), pix.end()), hi = *std::max_element(pix.begin(), pix.end());
            for (long long q = lo * comp; q < (hi + 1) * comp; ++q) m[q] = std::nan("");
            for (long long k = 0; k < n; ++k)
                for (int c = 0; c < comp; ++c) m[pix[k] * comp + c] = rd();
            g_maps[id] = m;
            printf("0\n");
        } else if (o == "lens" || o == "full") {
            flints_plan_t p = g_plans[rl()];
            const int comp = spin_of(p) == 0 ? 1 : 2;
            flints_plan_info i;
            flints_get_info(p, &i);
            long long first = 0, count = 12 * i.nside * i.nside;
            if (o == "lens") { first = rl(); count = rl(); }
            double *m = g_maps[rl()];
            Buffers b = read_job(count, comp);
            int rc;
            const size_t a0 = g_dev_alloc_calls;
            if (o == "lens")
                rc = flints_lens_range(p, first, count, m, b.defl.data(), b.out.data(), b.var.data(), b.status.data(),
                                       nullptr);
            else {
                rc = comp == 1 ? flints_lens_spin0(p, m, b.defl.data(), b.out.data(), b.var.data(), nullptr)
                               : flints_lens_spin2(p, m, b.defl.data(), b.out.data(), b.var.data(), nullptr);
                std::fill(b.status.begin(), b.status.end(), 0);
            }
            g_hot_allocs += g_dev_alloc_calls != a0;
            printf("%d\n", rc);
            print_rows(b, count, comp);
        } else if (o == "super") {
            flints_plan_t p = g_plans[rl()];
            const int comp = spin_of(p) == 0 ? 1 : 2;
            const long long nout = rl(), first = rl(), count = rl();
            double *m = g_maps[rl()];
            Buffers b = read_job(0, comp);
            b.out.assign(comp * count, 0.0);
            b.var.assign(count, 0.0);
            b.status.assign(count, 255);
            const size_t a0 = g_dev_alloc_calls;
            const int rc = flints_supersample(p, nout, first, count, m, b.out.data(), b.var.data(), b.status.data(),
                                              nullptr);
            g_hot_allocs += g_dev_alloc_calls != a0;
            printf("%d\n", rc);
            print_rows(b, count, comp);
        } else if (o == "stencil") {
            flints_plan_t p = g_plans[rl()];
            flints_plan_info i;
            flints_get_info(p, &i);
            const long long first = rl(), count = rl();
            Buffers b = read_job(count, 1);
            std::vector<int64_t> idx((size_t)count * i.K, -9);
            const size_t a0 = g_dev_alloc_calls;
            const int rc = flints_stencil(p, first, count, b.defl.data(), idx.data(), b.status.data(), nullptr);
            g_hot_allocs += g_dev_alloc_calls != a0;
            printf("%d\n", rc);
            for (long long q = 0; q < count; ++q) {
                printf("%d", (int)b.status[q]);
                for (int k = 0; k < i.K; ++k) printf(" %lld", (long long)idx[(size_t)q * i.K + k]);
                printf("\n");
            }
        } else if (o == "stats") {
            flints_stats s{};
            const int rc = flints_get_stats(g_plans[rl()], &s, nullptr);
            printf("%d %lld %lld %lld %lld %lld\n", rc, (long long)s.points, (long long)s.nugget,
                   (long long)s.fallback, (long long)s.window, (long long)s.failed);
        } else if (o == "batch" || o == "bobj") {  // n jobs [wpb tile], then per job: plan first count map defl
            const int n = (int)rl();
            flints_launch_cfg cfg{0, 0, 0};
            if (o == "bobj") { cfg.warps_per_block = (int)rl(); cfg.tile_points = (int)rl(); }
            std::vector<Buffers> bufs(n);
            std::vector<flints_job> jobs(n);
            std::vector<int> comps(n);
            for (int j = 0; j < n; ++j) {
                flints_plan_t p = g_plans[rl()];
                const long long first = rl(), count = rl();
                double *m = g_maps[rl()];
                comps[j] = spin_of(p) == 0 ? 1 : 2;
                bufs[j] = read_job(count, comps[j]);
                jobs[j] = flints_job{p, first, count, m, bufs[j].defl.data(), bufs[j].out.data(), bufs[j].var.data(),
                                     bufs[j].status.data()};
            }
            int rc;
            if (o == "batch") rc = flints_lens_batch(jobs.data(), n, nullptr);
            else {
                flints_batch_t bt = nullptr;
                rc = flints_batch_create(&bt, n);  // allocates; staging and launching must not
                const size_t a0 = g_dev_alloc_calls;
                if (rc == 0) rc = flints_batch_stage(bt, jobs.data(), n, cfg.tile_points);
                if (rc == 0) rc = flints_batch_launch(bt, &cfg, nullptr);
                g_hot_allocs += g_dev_alloc_calls != a0;
                flints_batch_free(bt);
            }
            printf("%d\n", rc);
            for (int j = 0; j < n; ++j) print_rows(bufs[j], jobs[j].count, comps[j]);
        } else if (o == "noalloc") {
            const long long nside = rl();
            const int lmax = (int)rl(), spin = (int)rl(), K = (int)rl(), prec = (int)rl(), has_bb = (int)rl();
            std::vector<double> cl(lmax + 1), bb(lmax + 1);
            for (double &v : cl) v = rd();
            if (has_bb) for (double &v : bb) v = rd();
            const long long first = rl(), count = rl();
            double *m = g_maps[rl()];
            const int comp = spin == 0 ? 1 : 2;
            Buffers b = read_job(count, comp);
            const size_t a0 = g_dev_alloc_calls;
            const int rc = flints_lens_noalloc(nside, lmax, cl.data(), has_bb ? bb.data() : nullptr, spin, K, prec,
                                               first, count, m, b.defl.data(), b.out.data(), b.var.data(),
                                               b.status.data(), nullptr);
            g_hot_allocs += g_dev_alloc_calls != a0;
            printf("%d\n", rc);
            print_rows(b, count, comp);
        } else if (o == "table") {  // plan which: the plan's xi table copied to the host
            flints_plan_t p = g_plans[rl()];
            const int which = (int)rl();
            flints_plan_info i;
            flints_get_info(p, &i);
            std::vector<double> f(i.n_intervals + 1), g(i.n_intervals + 1);
            printf("%d\n", flints_get_table(p, which, f.data(), g.data(), nullptr));
            for (int k = 0; k <= i.n_intervals; ++k) printf("%a %a\n", f[k], g[k]);
        } else if (o == "reset") {
            printf("%d\n", flints_reset_stats(g_plans[rl()], nullptr));
        } else if (o == "reject") {  // plans of spin 0 and 2 (FP64, K = 16) and spin 1: calls refused before any launch
            flints_plan_t p0 = g_plans[rl()], p2 = g_plans[rl()], p1 = g_plans[rl()];
            flints_plan_info i;
            flints_get_info(p0, &i);
            const long long npix = 12 * i.nside * i.nside;
            static double buf[4096] __attribute__((aligned(64)));
            for (double &v : buf) v = std::nan("");
            static uint8_t st[256];
            std::memset(st, 255, sizeof st);
            static int64_t idx[64 * 16];
            std::fill(idx, idx + 64 * 16, -9);
            double *m = buf, *d = buf + 2048, *out = buf + 3072, *var = buf + 3584;
            auto shift = [](const void *q, int by) { return (void *)((const char *)q + by); };
            auto rep = [](int rc, const char *msg) { printf("%d|%s\n", rc, msg); };
            const char *(*le)() = flints_last_error;
            rep(flints_lens_range(nullptr, 0, 4, m, d, out, var, st, nullptr), le());
            rep(flints_lens_range(p0, -1, 4, m, d, out, var, st, nullptr), le());
            rep(flints_lens_range(p0, npix - 2, 4, m, d, out, var, st, nullptr), le());
            rep(flints_lens_range(p0, 0, 4, m, nullptr, out, var, st, nullptr), le());
            rep(flints_lens_range(p0, 0, 4, nullptr, d, out, var, st, nullptr), le());
            rep(flints_lens_range(p0, 0, 4, m, (double *)shift(d, 8), out, var, st, nullptr), le());
            rep(flints_lens_range(p2, 0, 4, (double *)shift(m, 8), d, out, var, st, nullptr), le());
            rep(flints_lens_range(p2, 0, 4, m, d, (double *)shift(out, 8), var, st, nullptr), le());
            rep(flints_lens_range(p0, 0, 4, m, d, out, (double *)shift(var, 4), st, nullptr), le());
            rep(flints_stencil(p0, 0, 4, d, nullptr, st, nullptr), le());
            rep(flints_stencil(p0, 0, 4, d, (int64_t *)shift(idx, 4), st, nullptr), le());
            rep(flints_lens_spin0(p2, m, d, out, var, nullptr), le());
            rep(flints_lens_spin2(p0, m, d, out, var, nullptr), le());
            rep(flints_supersample(p0, 0, 0, 4, m, out, var, st, nullptr), le());
            rep(flints_supersample(p0, 2 * i.nside, 48 * i.nside * i.nside - 1, 2, m, out, var, st, nullptr), le());
            flints_launch_cfg bad[3] = {{9, 0, 0}, {0, 33, 0}, {0, 0, 17}};
            for (const auto &c : bad) rep(flints_plan_set_launch(p0, &c), le());
            double f[4], g[4];
            rep(flints_get_table(p0, 1, f, g, nullptr), le());
            rep(flints_get_stats(p0, nullptr, nullptr), le());
            flints_batch_t b = nullptr;
            rep(flints_batch_create(&b, 0), le());
            rep(flints_batch_create(&b, 2), le());
            flints_job ok{p0, 0, 4, m, d, out, var, st};
            flints_job two[2] = {ok, ok};
            rep(flints_batch_stage(b, two, 3, 0), le());
            rep(flints_batch_stage(b, two, 2, 17), le());
            flints_stats s0{}, s1{};
            flints_get_stats(p0, &s0, nullptr);
            two[1].plan = nullptr;
            rep(flints_batch_stage(b, two, 2, 0), le());
            two[1] = ok;
            two[1].plan = p1;
            rep(flints_batch_stage(b, two, 2, 0), le());
            two[1] = ok;
            two[1].first = npix - 1;
            rep(flints_batch_stage(b, two, 2, 0), le());
            two[1] = ok;
            two[1].map = nullptr;
            rep(flints_batch_stage(b, two, 2, 0), le());
            two[1] = ok;
            two[1].var = (double *)shift(var, 4);
            rep(flints_batch_stage(b, two, 2, 0), le());
            flints_get_stats(p0, &s1, nullptr);
            printf("points %lld\n", (long long)(s1.points - s0.points));  // refused stages count no points
            flints_launch_cfg wide{9, 0, 0};
            rep(flints_batch_launch(b, &wide, nullptr), le());
            rep(flints_lens_batch(two, -1, nullptr), le());
            // empty ranges are accepted with any buffers, and launch nothing
            rep(flints_lens_range(p0, npix, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr), le());
            rep(flints_lens_range(p2, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr), le());
            rep(flints_stencil(p0, 5, 0, nullptr, idx, nullptr, nullptr), le());
            rep(flints_supersample(p0, 16, 3, 0, nullptr, nullptr, nullptr, nullptr, nullptr), le());
            rep(flints_lens_batch(nullptr, 0, nullptr), le());
            flints_job empty{p2, 7, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
            rep(flints_lens_batch(&empty, 1, nullptr), le());
            flints_batch_free(b);
            bool untouched = std::all_of(buf + 3072, buf + 4096, [](double v) { return std::isnan(v); }) &&
                             std::all_of(st, st + 256, [](uint8_t v) { return v == 255; }) &&
                             std::all_of(idx, idx + 64 * 16, [](int64_t v) { return v == -9; });
            printf("untouched %d\n", untouched ? 1 : 0);
        } else if (o == "nreject") {  // the no-allocation entry point's checks, each refused before any launch
            static double buf[4096] __attribute__((aligned(64)));
            for (double &v : buf) v = std::nan("");
            static uint8_t st[256];
            std::memset(st, 255, sizeof st);
            double *m = buf, *d = buf + 2048, *out = buf + 3072, *var = buf + 3584;
            std::vector<double> cl(4001, 1.0), zero(17, 0.0), bad(17, 1.0);
            bad[5] = std::nan("");
            auto rep = [](int rc) { printf("%d|%s\n", rc, flints_noalloc_last_error()); };
            auto call = [&](long long nside, int lmax, const double *c, int spin, int K, int prec, long long first,
                            long long count, const double *mm, const double *dd, double *oo, double *vv) {
                rep(flints_lens_noalloc(nside, lmax, c, nullptr, spin, K, prec, first, count, mm, dd, oo, vv, st,
                                        nullptr));
            };
            call(0, 16, cl.data(), 0, 16, 0, 0, 4, m, d, out, var);
            call(8, 9000, cl.data(), 0, 16, 0, 0, 4, m, d, out, var);
            call(8, 16, nullptr, 0, 16, 0, 0, 4, m, d, out, var);
            call(8, 16, cl.data(), 1, 16, 0, 0, 4, m, d, out, var);
            call(8, 16, cl.data(), 0, 20, 0, 0, 4, m, d, out, var);
            call(8, 16, cl.data(), 0, 16, 2, 0, 4, m, d, out, var);
            call(8, 16, cl.data(), 0, 16, 0, 766, 4, m, d, out, var);
            call(8, 16, cl.data(), 0, 16, 0, 0, 4, nullptr, d, out, var);
            call(8, 16, cl.data(), 0, 16, 0, 0, 4, m, d, out, (double *)((char *)var + 4));
            call(8, 16, cl.data(), 2, 16, 0, 0, 4, m + 1, d, out, var);
            call(8, 16, bad.data(), 0, 16, 0, 0, 4, m, d, out, var);
            call(16, 4000, cl.data(), 0, 16, 0, 0, 4, m, d, out, var);
            call(8, 16, zero.data(), 0, 16, 0, 0, 4, m, d, out, var);
            call(8, 16, cl.data(), 2, 16, 1, 768, 0, nullptr, nullptr, nullptr, nullptr);  // empty: accepted
            printf("untouched %d\n", std::all_of(buf + 3072, buf + 4096, [](double v) { return std::isnan(v); }) &&
                                             std::all_of(st, st + 256, [](uint8_t v) { return v == 255; }) ? 1 : 0);
        } else return 3;
        printf("end\n");
        fflush(stdout);
    }
    const size_t live = g_dev_live;
    long long held = 0;
    for (auto &kv : g_plans) {
        flints_plan_info i{};
        if (kv.second && flints_get_info(kv.second, &i) == 0) held += i.device_bytes;
        flints_free(kv.second);  // every plan's allocations come back (leak check)
    }
    if ((long long)(live - g_dev_live) != held) return 4;  // flints_free returned what the plans reported
    if (g_hot_allocs) return 5;  // a lens, supersampling, stencil, batch-launch or no-allocation call allocated
    return 0;
}
"""

FILES = ["common.cuh", "lens.cuh", "batch_types.cuh", "batch.cuh", "xi_table.cu", "lens_spin0.cu", "lens_spin1.cu",
         "lens_spin2.cu", "lens_spin2a.cu", "batch_p0.cu", "batch_p1.cu", "api.cu", "noalloc.cu"]


class Session:
    """A script of API calls for the host build, run at once; results in call order."""

    def __init__(self, exe):
        self.exe, self.lines, self.kinds = exe, [], []

    @staticmethod
    def _h(a):
        return " ".join(float(x).hex() for x in np.ravel(a))

    def plan(self, pid, nside, cl, bb=None, spin=0, K=32, prec=0, flags=0):
        self.lines.append(f"plan {pid} {nside} {cl.size - 1} {spin} {K} {prec} {flags} {0 if bb is None else 1} "
                          + self._h(cl) + ("" if bb is None else " " + self._h(bb)))
        self.kinds.append("plan")

    def launch(self, pid, wpb, bps=0, tile=0):
        self.lines.append(f"launch {pid} {wpb} {bps} {tile}")
        self.kinds.append("map")

    def map(self, mid, nside, pix, vals):
        comp = 1 if vals.ndim == 1 else 2
        self.lines.append(f"map {mid} {nside} {comp} {len(pix)} " + " ".join(str(int(p)) for p in pix) + " "
                          + self._h(vals))
        self.kinds.append("map")

    def lens(self, pid, first, count, mid, defl):
        self.lines.append(f"lens {pid} {first} {count} {mid} " + self._h(defl))
        self.kinds.append("rows")

    def full(self, pid, mid, defl):
        self.lines.append(f"full {pid} {mid} " + self._h(defl))
        self.kinds.append("rows")

    def super(self, pid, nout, first, count, mid):
        self.lines.append(f"super {pid} {nout} {first} {count} {mid}")
        self.kinds.append("rows")

    def stencil(self, pid, first, count, defl):
        self.lines.append(f"stencil {pid} {first} {count} " + self._h(defl))
        self.kinds.append("stencil")

    def table(self, pid, which=0):
        self.lines.append(f"table {pid} {which}")
        self.kinds.append("table")

    def reset(self, pid):
        self.lines.append(f"reset {pid}")
        self.kinds.append("map")

    def stats(self, pid):
        self.lines.append(f"stats {pid}")
        self.kinds.append("stats")

    def batch(self, jobs, obj=None):
        head = f"batch {len(jobs)}" if obj is None else f"bobj {len(jobs)} {obj[0]} {obj[1]}"
        self.lines.append(head + " " + " ".join(f"{p} {f} {c} {m} " + self._h(d) for p, f, c, m, d in jobs))
        self.kinds.append(("batch", [c for _, _, c, _, _ in jobs]))

    def noalloc(self, nside, cl, bb, spin, K, prec, first, count, mid, defl):
        self.lines.append(f"noalloc {nside} {cl.size - 1} {spin} {K} {prec} {0 if bb is None else 1} " + self._h(cl)
                          + ("" if bb is None else " " + self._h(bb)) + f" {first} {count} {mid} " + self._h(defl))
        self.kinds.append("rows")

    def reject(self, p0, p2, p1):
        self.lines.append(f"reject {p0} {p2} {p1}")
        self.kinds.append("reject")

    def nreject(self):
        self.lines.append("nreject")
        self.kinds.append("reject")

    def run(self):
        out = hc.run(self.exe, "\n".join(self.lines) + "\n").split("end\n")
        res = []
        for kind, block in zip(self.kinds, out):
            rows = [ln.split() for ln in block.strip().splitlines()]
            if kind in ("plan", "map"):
                res.append([float.fromhex(t) if "x" in t else int(t) for t in rows[0]])
            elif kind == "table":
                assert rows[0] == ["0"], rows[:2]
                fg = np.array([[float.fromhex(a) for a in r] for r in rows[1:]])
                res.append((fg[:, 0], fg[:, 1]))
            elif kind == "reject":
                res.append(block.strip().splitlines())
            elif kind == "stats":
                res.append([int(t) for t in rows[0]])
            elif kind == "stencil":
                assert rows[0] == ["0"], rows[:2]
                res.append((np.array([int(r[0]) for r in rows[1:]]), np.array([[int(t) for t in r[1:]] for r in rows[1:]])))
            else:
                assert rows[0] == ["0"], rows[:2]
                data = [(int(r[0]), float.fromhex(r[1]) + 1j * float.fromhex(r[2]), float.fromhex(r[3]))
                        for r in rows[1:]]
                st = np.array([d[0] for d in data])
                val = np.array([d[1] for d in data])
                var = np.array([d[2] for d in data])
                if isinstance(kind, tuple):  # split the batch's rows per job
                    out_j, k = [], 0
                    for c in kind[1]:
                        out_j.append((st[k:k + c], val[k:k + c], var[k:k + c]))
                        k += c
                    res.append(out_j)
                else:
                    res.append((st, val, var))
        return res


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    return ch.build(tmp_path_factory.mktemp("api"), "api_host", FILES, DRIVER)


def _sky(spin, nside, lmax, seed):
    if spin == 0:
        cl, bb = wl.cl_tt(lmax, 0.7 * lmax), None
        m = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed))
        return cl, bb, m, float(np.std(m))
    cl = wl.cl_ee(lmax, 0.7 * lmax)
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl, seed), spin=2)
    return cl, None, np.stack([P.real, P.imag], 1), float(np.sqrt(np.mean(np.abs(P) ** 2)))


def _oracle(spin, nside, K, cl, bb, m, defl, pix):
    weight = np.abs(cl) + (np.abs(bb) if bb is not None else 0.0)
    t_max, n = xi.grid_rule(weight, K, nside)
    tab, x0 = xi.spin0_table(cl, t_max, n) if spin == 0 else xi.spin2_tables(cl, bb, t_max, n)[::2]
    return kr.lens(nside, K, spin, m, defl, pix, tab, x0), x0, t_max, n


# (spin, K, precision, warps per block of the plan's launches: 0 = the default, 8)
@pytest.mark.parametrize("spin,K,prec,wpb", [(0, 16, 0, 0), (2, 32, 1, 0), (2, 24, 0, 2)])
def test_whole_sky_entry_points_match_the_oracle_and_each_other(spin, K, prec, wpb, exe):
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    cl, bb, m, sigma = _sky(spin, nside, lmax, 10 * K + spin)
    defl = wl.random_deflection(npix, 3 + K) * 8
    ref, x0, t_max, n = _oracle(spin, nside, K, cl, bb, m, defl, np.arange(npix))
    a, b, c, d = 100, 100 + 333, 500, 500 + 150
    s = Session(exe)
    s.plan(1, nside, cl, bb, spin, K, prec)
    if wpb:
        s.launch(1, wpb, 0, 0)
    s.map(1, nside, np.arange(npix), m)
    s.full(1, 1, defl)                                   # flints_lens_spin0 / spin2, whole sky
    s.lens(1, a, b - a, 1, defl[a:b])                    # flints_lens_range, a ragged range
    s.stats(1)
    s.noalloc(nside, cl, bb, spin, K, prec, a, b - a, 1, defl[a:b])
    s.noalloc(nside, cl, bb, spin, K, prec, c, d - c, 1, defl[c:d])  # the shared array keeps the last call's contents
    s.stencil(1, c, d - c, defl[c:d])
    res = s.run()
    plan = res[0]
    full, part, stats, na1, na2, (sst, idx) = res[-6:]
    assert plan[0] == 0 and plan[1] == t_max and plan[2] == n and abs(plan[3] - x0) <= 1e-13 * x0
    tol = 1e-9 if prec == 0 else 1e-6
    v_ref = ref.value if spin else ref.value + 0j
    for (st, v, var), sl in ((full, slice(0, npix)), (part, slice(a, b)), (na2, slice(c, d))):
        assert np.max(np.abs(v - v_ref[sl])) <= tol * sigma
        assert np.max(np.abs(var - ref.variance[sl])) <= tol * x0
    assert np.all(part[0] == 0) and np.all(na1[0] == 0) and np.all(na2[0] == 0)
    # the same per-tile code on the same inputs: identical results
    assert np.array_equal(full[1][a:b], part[1]) and np.array_equal(part[1], na1[1]) and np.array_equal(part[2], na1[2])
    assert np.array_equal(full[1][c:d], na2[1])
    assert stats[:2] == [0, npix + (b - a)] and stats[3:] == [0, 0, 0]
    ref_idx, key = kr.knn(nside, ref.target[c:d], K + 1)
    tie = (key[:, K] - key[:, K - 1]) <= 1e-11 * key[:, K]
    assert np.all(sst == 0) and np.all(np.all(idx == ref_idx[:, :K], axis=1) | tie)


def test_batches_equal_single_calls(exe):
    nside = 16
    npix = hp.npix(nside)
    specs = [(0, 16, 0, 0, 160), (2, 32, 1, 5, 130), (0, 48, 1, 2000, 96), (2, 24, 0, 100, 0)]
    s = Session(exe)
    maps = {}
    for spin in (0, 2):
        cl, bb, m, _ = _sky(spin, nside, 32, 50 + spin)
        maps[spin] = (cl, bb)
        s.map(spin + 1, nside, np.arange(npix), m)
    jobs = []
    for j, (spin, K, prec, first, count) in enumerate(specs):
        cl, bb = maps[spin]
        s.plan(10 + j, nside, cl, bb, spin, K, prec)
        d = wl.random_deflection(count, 60 + j) * 4
        jobs.append((10 + j, first, count, spin + 1, d))
    for pid, first, count, mid, d in jobs:
        s.lens(pid, first, count, mid, d)
    s.batch(jobs)
    s.batch(jobs, obj=(2, 7))  # batch objects, 2-warp blocks, 7-target tiles
    res = s.run()
    singles, conv, objs = res[-2 - len(jobs):-2], res[-2], res[-1]
    for (st, v, var), a, b in zip(singles, conv, objs):
        for other in (a, b):
            assert np.array_equal(st, other[0]) and np.array_equal(v, other[1]) and np.array_equal(var, other[2])


def test_nside_4096_band_and_supersampling(exe):
    """A band of the Nside 4096 spin-2 workload (mixed) through the range entry point, and
    supersampling of a small sky to its 2x grid, against the oracle."""
    W = wl.C3
    cl, bb = W.cl()
    first, count = 8_390_000, 48
    defl = wl.random_deflection(count, 77)
    tv = kr.displace(W.nside, np.arange(first, first + count), defl)
    idx, _ = kr.knn(W.nside, tv, 56)
    r = hp.pix2ring(W.nside, idx.ravel())[0]
    pix, P = sht.synth_rings(W.nside, np.arange(r.min() - 1, r.max() + 2), W.lmax, wl.draw_alm(cl, 9), spin=2)
    vals = np.stack([P.real, P.imag], 1)

    class Band:
        def __getitem__(self, key):
            i, c = key if isinstance(key, tuple) else (key, None)
            v = vals[np.searchsorted(pix, i)]
            return v if c is None else v[..., c]

    ref, x0, _, _ = _oracle(2, W.nside, W.K, cl, bb, Band(), defl, np.arange(first, first + count))
    sigma = float(np.sqrt(np.mean(np.sum(vals ** 2, 1))))
    nside, lmax = 16, 32
    c0, b0, m0, s0 = _sky(0, nside, lmax, 5)
    s = Session(exe)
    s.plan(1, W.nside, cl, bb, 2, W.K, 1)
    s.map(1, W.nside, pix, vals)
    s.lens(1, first, count, 1, defl)
    s.plan(2, nside, c0, None, 0, 32, 0)
    s.map(2, nside, np.arange(hp.npix(nside)), m0)
    s.super(2, 32, 100, 1500, 2)
    res = s.run()
    st, v, var = res[2]
    assert np.all(st == 0)
    assert np.max(np.abs(v - ref.value)) <= 1e-6 * sigma and np.max(np.abs(var - ref.variance)) <= 1e-6 * x0
    st, v, var = res[5]
    t_max, n = xi.grid_rule(np.abs(c0), 32, nside)
    tab, x00 = xi.spin0_table(c0, t_max, n)
    sref = kr.supersample(nside, 32, 32, 0, m0, np.arange(100, 1600), tab, x00)
    # supersampling targets sit between source pixels: about 20 % of stencils tie for the
    # last place, where any valid set is correct; the others must match
    tgt = hp.pix2vec(32, np.arange(100, 1600))
    _, key = kr.knn(nside, tgt, 33)
    tie = (key[:, 32] - key[:, 31]) <= 1e-11 * key[:, 32]
    ok = np.abs(v.real - sref.value) <= 1e-9 * s0
    assert np.all(ok | tie) and np.mean(ok) > 0.5


def test_spin1_and_augmented_plans_through_the_single_range_kernel(exe):
    """Spin-1 plans and augmented spin-2 plans launch the single-range kernel (its tile
    queue): a deflection field lensed as a spin-1 map and an E/B field with the widely
    linear estimator, against the oracle."""
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    first, count = 200, 150
    defl = wl.random_deflection(count, 91) * 8
    pix = np.arange(first, first + count)
    # spin 1: the gradient of a potential, spectrum l(l+1) C^phiphi
    ell = np.arange(lmax + 1.0)
    cl1 = ell * (ell + 1) * wl.cl_phiphi(lmax)
    g = sht.synth_map(nside, lmax, wl.draw_alm(wl.cl_phiphi(lmax), 92), gradient=True)
    t1, n1 = xi.grid_rule(np.abs(cl1), 32, nside)
    tab1, _, x01 = xi.spin1_tables(cl1, None, t1, n1)
    ref1 = kr.lens(nside, 32, 1, g, defl, pix, tab1, x01)
    # augmented spin 2
    cl2 = wl.cl_ee(lmax, 0.7 * lmax)
    bb = 0.3 * cl2
    P = sht.synth_map(nside, lmax, wl.draw_alm(cl2, 93), spin=2, blm=wl.draw_alm(bb, 94))
    qu = np.stack([P.real, P.imag], 1)
    t2, n2 = xi.grid_rule(np.abs(cl2) + np.abs(bb), 24, nside)
    tp, tm, x02 = xi.spin2_tables(cl2, bb, t2, n2)
    ref2 = kr.lens(nside, 24, 2, qu, defl, pix, tp, x02, f_minus=tm)
    s = Session(exe)
    s.plan(1, nside, cl1, None, 1, 32, 0)
    s.map(1, nside, np.arange(npix), g)
    s.lens(1, first, count, 1, defl)
    s.plan(2, nside, cl2, bb, 2, 24, 1, flags=1)  # FLINTS_SPIN2_AUGMENTED, mixed
    s.map(2, nside, np.arange(npix), qu)
    s.lens(2, first, count, 2, defl)
    res = s.run()
    for (st, v, var), ref, x0, m, tol in ((res[2], ref1, x01, g, 1e-9), (res[5], ref2, x02, qu, 1e-6)):
        sigma = float(np.sqrt(np.mean(np.sum(m ** 2, 1))))
        assert np.all(st == 0)
        assert np.max(np.abs(v - ref.value)) <= tol * sigma and np.max(np.abs(var - ref.variance)) <= tol * x0


def test_indefinite_covariances_take_the_nugget_steps(exe):
    """Sec. 2.4's nugget on covariances that are not positive definite (never met on the
    workloads, whose spectra are positive): a spectrum with a small negative multipole
    makes S + 1.49e-8 I indefinite on some stencils.  The kernel doubles the nugget
    until the factor exists (FLINTS_ST_NUGGET), at most 8 times (then FLINTS_ST_FAILED
    with NaN outputs), and the value is the estimate with that nugget; the mixed kernel
    re-solves those points on its FP64 path (FLINTS_ST_FALLBACK).  (The oracle's rule,
    n = -lambda_min + 1.49e-8, is a different reading of the same passage; here the
    oracle is run with the kernel's nugget.)"""
    nside, lmax, K = 8, 16, 16
    npix = hp.npix(nside)
    cl = wl.cl_tt(lmax, 11.0)
    cl[lmax] = -0.0043 * cl[2]
    m = sht.synth_map(nside, lmax, wl.draw_alm(np.abs(cl), 95))
    sigma = float(np.std(m))
    defl = wl.random_deflection(npix, 5) * 8
    pix = np.arange(npix)
    t_max, n = xi.grid_rule(np.abs(cl), K, nside)
    tab, x0 = xi.spin0_table(cl, t_max, n)
    tv = kr.displace(nside, pix, defl)
    idx, _ = kr.knn(nside, tv, K)
    X = hp.pix2vec(nside, idx)
    S = tab(kr._chord2(X[:, :, None, :], X[:, None, :, :]).reshape(-1)).reshape(npix, K, K)
    S[:, np.arange(K), np.arange(K)] = 1.0
    eps = kr.EPS_NUGGET
    # the first nugget eps 2^k (k = 0..8) whose Cholesky exists, as both sides factor in FP64
    first_ok = np.full(npix, -1)
    for k in range(8, -1, -1):
        _, ok = kr.cholesky_batched(S + eps * 2.0 ** k * np.eye(K))
        first_ok = np.where(ok, k, first_ok)
    s = Session(exe)
    s.plan(1, nside, cl, None, 0, K, 0)
    s.plan(2, nside, cl, None, 0, K, 1)
    s.map(1, nside, pix, m)
    s.lens(1, 0, npix, 1, defl)
    s.lens(2, 0, npix, 1, defl)
    s.stats(1)
    res = s.run()
    (st64, v64, var64), (stmx, vmx, varmx), stats = res[3], res[4], res[5]
    nug, failed = (st64 & 1) != 0, (st64 & 8) != 0
    assert np.array_equal(nug, first_ok != 0) and np.array_equal(failed, first_ok < 0)
    assert 0.05 < np.mean(nug) and np.any(failed)  # the case exercises both outcomes
    assert np.all(np.isnan(v64[failed])) and np.all(np.isfinite(v64[~failed]))
    assert stats[2] == np.sum(nug) and stats[5] == np.sum(failed)
    # values: the oracle's estimate with the nugget the kernel settled on.  Near the edge
    # of positive definiteness the weights are large (values of 100 sigma and more) and
    # rounding is amplified alike on both sides: the bound is relative to the value; a
    # wrong nugget would move it by a large fraction of itself
    for k in range(0, 9):
        rows = np.nonzero(first_ok == k)[0]
        if rows.size == 0:
            continue
        v, s2, _ = kr.estimate(nside, 0, m, tv[rows], idx[rows], tab, x0, eps=eps * 2.0 ** k)
        assert np.all(np.abs(v64[rows].real - v) <= 1e-6 * (sigma + np.abs(v))), k
        assert np.all(np.abs(var64[rows] - s2) <= 1e-6 * (x0 + np.abs(s2))), k
    # the mixed kernel: the indefinite points go to its FP64 path and end the same way
    assert np.all(((stmx & 2) != 0)[first_ok != 0])
    assert np.array_equal((stmx & (1 | 8)), (st64 & (1 | 8)))
    ok = ~failed
    assert np.all(np.abs(vmx[ok] - v64[ok]) <= 1e-6 * (sigma + np.abs(v64[ok])))


def test_targets_displaced_onto_a_pole(exe):
    """Targets displaced onto the north pole (to rounding), where the spin-2 frame at
    the displaced point is undefined: the kernel flags FLINTS_ST_POLE there and takes
    the frame of phi = 0, the oracle the frame of its displaced vector's rounding-level
    phi.  Transported back to the frame at the target pixel (FLINTS_ROTATE_TO_TARGET)
    the lensed value does not depend on that choice, so the two agree; K = 24 is the
    three northernmost rings at Nside 8, a stencil without ties at the pole.  Every
    other target lands 1e-3 rad from the pole instead and is not flagged."""
    nside, lmax, K = 8, 16, 24
    npix = hp.npix(nside)
    cl, bb, m, sigma = _sky(2, nside, lmax, 97)
    pix = np.arange(0, 12)  # the two northernmost rings
    z, s, _ = hp.pix2ang(nside, pix)
    defl = np.stack([-np.arctan2(s, z), np.zeros(pix.size)], 1)  # d_theta = -theta: onto the pole
    defl[1::2, 1] = 1e-3
    weight = np.abs(cl)
    t_max, n = xi.grid_rule(weight, K, nside)
    tab, x0 = xi.spin2_tables(cl, bb, t_max, n)[::2]
    ref = kr.lens(nside, K, 2, m, defl, pix, tab, x0, rotate=True)
    s_ = Session(exe)
    s_.plan(1, nside, cl, bb, 2, K, 0, 2)  # flags: FLINTS_ROTATE_TO_TARGET
    s_.map(1, nside, np.arange(npix), m)
    s_.lens(1, 0, pix.size, 1, defl)
    st, v, var = s_.run()[2]
    assert np.array_equal(st, np.where(np.arange(pix.size) % 2 == 0, 16, 0))
    assert np.max(np.abs(v - ref.value)) <= 1e-9 * sigma, np.max(np.abs(v - ref.value)) / sigma
    assert np.max(np.abs(var - ref.variance)) <= 1e-9 * x0


def test_invalid_calls_are_refused_before_any_launch(exe):
    """Every argument check of the K-nearest C API (null and out-of-range arguments,
    misaligned buffers, a plan of the wrong spin, launch shapes, batch jobs) returns
    FLINTS_EINVAL with a message naming the fault, writes no output and, for a batch
    stage refused at a later job, counts no points for the earlier ones.  Empty
    ranges (count 0, also at first = Npix, and empty batches) succeed with any
    buffers and write nothing."""
    nside, lmax = 8, 16
    s_ = Session(exe)
    s_.plan(1, nside, wl.cl_tt(lmax, 12.0), None, 0, 16, 0)
    s_.plan(2, nside, wl.cl_ee(lmax, 12.0), np.zeros(lmax + 1), 2, 16, 0)
    s_.plan(3, nside, wl.cl_phiphi(lmax), None, 1, 16, 0)
    s_.reject(1, 2, 3)
    res = s_.run()
    assert [r[0] for r in res[:3]] == [0, 0, 0]
    lines = res[3]
    assert lines[29] == "points 0", lines[29]  # the refused stages counted no points
    calls, tail = lines[:29] + lines[30:-1], lines[-1:]
    expect = ["plan is NULL", "target range", "target range", "defl is NULL", "map and out must not be NULL",
              "16-byte aligned", "16-byte aligned", "16-byte aligned", "8-byte aligned", "idx is NULL",
              "8-byte aligned", "called with a spin-2 plan", "called with a plan of spin 0", "nside_out",
              "target range", "warps_per_block 0..8", "warps_per_block 0..8", "warps_per_block 0..8",
              "bad table index", "NULL argument", "bad arguments", None, "capacity 2", "tile_points 0..16",
              "job 1: plan is NULL", "job 1: spin-1 and augmented", "job 1: target range outside", "job 1: NULL data",
              "job 1: misaligned", "warps_per_block 1..8", "bad job list", None, None, None, None, None, None]
    assert len(calls) == len(expect), calls
    for line, msg in zip(calls, expect):
        rc, text = line.split("|", 1)
        if msg is None:
            assert rc == "0", line
        else:
            assert rc == "1" and msg in text, (line, msg)
    assert tail == ["untouched 1"], tail


def test_invalid_no_allocation_calls_are_refused(exe):
    """Every check of the no-allocation entry point (sizes, spin, K, precision, range,
    null and misaligned buffers, a non-finite spectrum, a table above the fixed
    interval count, a spectrum with xi(0) = 0) returns FLINTS_EINVAL with its message
    and writes no output."""
    s_ = Session(exe)
    s_.nreject()
    lines = s_.run()[0]
    expect = ["nside outside", "lmax 9000 exceeds the fixed maximum 8192", "cl is NULL", "spin must be 0 or 2",
              "K must be", "bad precision", "target range outside", "NULL data pointer", "misaligned buffer",
              "misaligned buffer", "non-finite spectrum value at l = 5", "65536 intervals, above the fixed maximum",
              "is not positive", None]
    assert len(lines) == len(expect) + 1, lines
    for line, msg in zip(lines, expect):
        rc, text = line.split("|", 1)
        assert (rc == "0") if msg is None else (rc == "1" and msg in text), (line, msg)
    assert lines[-1] == "untouched 1"


@pytest.mark.parametrize("spin,prec", [(0, 0), (2, 1)], ids=["spin0-fp64", "spin2-mixed"])
def test_no_variance_and_forced_fallback_flags(spin, prec, exe):
    """FLINTS_NO_VARIANCE: the values and status are those of the default plan and
    the variance buffer is left as it was.  FLINTS_FORCE_FALLBACK (mixed plans):
    every point is re-solved on the FP64 path and carries FLINTS_ST_FALLBACK, its
    values within 1e-8 of the oracle, and the fallback counter equals the count."""
    nside, lmax, K = 8, 16, 16
    npix = hp.npix(nside)
    cl, bb, m, sigma = _sky(spin, nside, lmax, 55 + spin)
    pix = np.arange(100, 300)
    defl = wl.random_deflection(npix, 56 + spin, rms=0.5 * np.sqrt(4 * np.pi / npix))[pix]
    ref, x0, _, _ = _oracle(spin, nside, K, cl, bb, m, defl, pix)
    s_ = Session(exe)
    s_.plan(1, nside, cl, bb, spin, K, prec, 0)
    s_.plan(2, nside, cl, bb, spin, K, prec, 4)  # FLINTS_NO_VARIANCE
    s_.map(1, nside, np.arange(npix), m)
    s_.lens(1, pix[0], pix.size, 1, defl)
    s_.lens(2, pix[0], pix.size, 1, defl)
    if prec == 1:
        s_.plan(3, nside, cl, bb, spin, K, 1, 256)  # FLINTS_FORCE_FALLBACK
        s_.lens(3, pix[0], pix.size, 1, defl)
        s_.stats(3)
    res = s_.run()
    (st1, v1, var1), (st2, v2, var2) = res[3], res[4]
    assert np.array_equal(st1, st2) and np.array_equal(v1, v2)
    assert np.all(np.isnan(var2)) and not np.any(np.isnan(var1))
    if prec == 1:
        st3, v3, var3 = res[6]
        assert np.all(st3 == 2)  # FLINTS_ST_FALLBACK only
        ref_v = ref.value if spin else ref.value.real
        assert np.max(np.abs(v3 - ref_v)) <= 1e-8 * sigma
        assert np.max(np.abs(var3 - ref.variance)) <= 1e-8 * x0
        assert res[7][3] == pix.size  # fallback counter


@pytest.mark.parametrize("spin,prec", [(0, 0), (2, 1)], ids=["spin0-fp64", "spin2-mixed"])
def test_nonfinite_deflections_in_a_tile(spin, prec, exe):
    """NaN and infinite deflections among good ones in the same warp tiles: those
    points get FLINTS_ST_INPUT | FLINTS_ST_FAILED and NaN outputs, the failed counter
    counts them, and the other points of their tiles keep the oracle's values (the
    lanes of a bad point leave the warp's collective steps without stalling them)."""
    nside, lmax, K = 8, 16, 16
    npix = hp.npix(nside)
    cl, bb, m, sigma = _sky(spin, nside, lmax, 61 + spin)
    pix = np.arange(200, 296)
    defl = wl.random_deflection(npix, 62 + spin, rms=0.5 * np.sqrt(4 * np.pi / npix))[pix]
    bad = np.array([0, 5, 6, 17, 40, 95])
    d_bad = defl.copy()
    d_bad[bad[0], 0] = np.nan
    d_bad[bad[1], 1] = np.inf
    d_bad[bad[2]] = [-np.inf, 0.0]
    d_bad[bad[3]] = [np.nan, np.nan]
    d_bad[bad[4], 1] = -np.inf
    d_bad[bad[5], 0] = np.inf
    good = np.setdiff1d(np.arange(pix.size), bad)
    ref, x0, _, _ = _oracle(spin, nside, K, cl, bb, m, defl[good], pix[good])
    s_ = Session(exe)
    s_.plan(1, nside, cl, bb, spin, K, prec)
    s_.map(1, nside, np.arange(npix), m)
    s_.lens(1, pix[0], pix.size, 1, d_bad)
    s_.stats(1)
    res = s_.run()
    st, v, var = res[2]
    assert np.all(st[bad] == 32 | 8) and np.all(st[good] == 0)  # FLINTS_ST_INPUT | FLINTS_ST_FAILED
    assert np.all(np.isnan(v[bad].real)) and np.all(np.isnan(var[bad]))
    assert res[3][5] == bad.size
    tol = 1e-9 if prec == 0 else 1e-6
    ref_v = ref.value if spin else ref.value.real
    assert np.max(np.abs(v[good] - ref_v)) <= tol * sigma
    assert np.max(np.abs(var[good] - ref.variance)) <= tol * x0


def test_table_copy_and_stats_reset(exe):
    """flints_get_table copies the plan's xi table (values and slopes at the nodes,
    xi+ and xi- for spin 2) within the GPU test's bounds of the oracle's direct sums;
    flints_reset_stats clears the point count and the counters, which then count
    only the later calls."""
    nside, lmax = 8, 16
    npix = hp.npix(nside)
    cl0 = wl.cl_tt(lmax, 12.0)
    cl2 = wl.cl_ee(lmax, 12.0)
    bb = 0.1 * cl2
    s = Session(exe)
    s.plan(1, nside, cl0, None, 0, 16, 0)
    s.plan(2, nside, cl2, bb, 2, 32, 1)
    s.table(1, 0)
    s.table(2, 0)
    s.table(2, 1)
    s.map(1, nside, np.arange(npix), sht.synth_map(nside, lmax, wl.draw_alm(cl0, 3)))
    d = wl.random_deflection(npix, 4, rms=0.5 * np.sqrt(4 * np.pi / npix))
    s.lens(1, 0, 100, 1, d[:100])
    s.stats(1)
    s.reset(1)
    s.stats(1)
    s.lens(1, 100, 50, 1, d[100:150])
    s.stats(1)
    res = s.run()
    for k, (spin, cl, b, K) in enumerate([(0, cl0, None, 16), (2, cl2, bb, 32)]):
        weight = np.abs(cl) + (np.abs(b) if b is not None else 0.0)
        t_max, n = xi.grid_rule(weight, K, nside)
        nodes = np.arange(n + 1) * (t_max / n)
        if spin == 0:
            ref, dref = xi.xi0_direct(cl, nodes, deriv=True)
        else:
            ref, xm, dref, dxm = xi.xis_direct(2, cl, b, nodes, deriv=True)
            fm, gm = res[4]
            np.testing.assert_allclose(fm, xm / ref[0], rtol=0, atol=2e-11)
            np.testing.assert_allclose(gm * t_max, dxm / ref[0] * t_max, rtol=0, atol=1e-9)
        f, g = res[2 + k]
        assert f.size == n + 1
        np.testing.assert_allclose(f, ref / ref[0], rtol=0, atol=1e-13)
        np.testing.assert_allclose(g * t_max, dref / ref[0] * t_max, rtol=0, atol=1e-9)
    assert res[7][:2] == [0, 100] and res[8] == [0] and res[9] == [0, 0, 0, 0, 0, 0]
    assert res[11][:2] == [0, 50]


def test_plan_reports_the_device_memory_it_holds(exe):
    """flints_get_info's device_bytes equals what flints_plan allocated on the device
    (counted by the runtime stand-in) for spin 0, 1, 2 and augmented plans, and
    flints_free returns exactly that (the driver exits with an error otherwise); the
    serving loop charges this figure against its memory budget."""
    nside, lmax = 8, 16
    s = Session(exe)
    cases = [(0, 16, 0, 0, False), (2, 32, 1, 0, True), (2, 24, 0, 1, True), (1, 16, 1, 0, False),
             (2, 48, 0, 0, False)]
    for k, (spin, K, prec, flags, with_bb) in enumerate(cases, 1):
        cl = wl.cl_tt(lmax, 12.0) if spin == 0 else wl.cl_ee(lmax, 12.0)
        s.plan(k, nside, cl, 0.3 * cl if with_bb else None, spin, K, prec, flags)
    res = s.run()
    for r, case in zip(res, cases):
        assert r[0] == 0 and r[4] == r[5] > 0, (case, r)
