"""The double-float arithmetic of the mixed path (csrc/common.cuh: TwoSum,
TwoProduct, double-float add, multiply, square root, reciprocal, the Cholesky
pivot and the anchored accumulator) compiled for the host and checked against
exact rational arithmetic, without a GPU.

The section of common.cuh between ``struct df`` and the precision policy is
compiled as host C++ (tests/host_compile.py: correctly rounded stand-ins for
the rounding intrinsics; rsqrtf, which the device computes to 2 ulp, is the
correctly rounded value moved by 2 ulp).  The bounds asserted are the ones
the source states: error-free transforms are exact, general double-float
operations keep about 2^-44 relative error, the pivot's inverse square root
2^-47 typically and 2^-44 at most, and the anchored accumulator about
2^-46 2^e per multiply-add, 2^e being the power of two of its anchor
(B < 2^e <= 2B when the partial sums stay below B; measured worst 2^-46 2^e,
median 2^-49 2^e).
Each test draws from its own seeded generator.
"""
import random
from fractions import Fraction as Fr

import numpy as np
import pytest

from tests import host_compile as hc

DRIVER = r"""
static float rd(void) { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtof(b, nullptr); }
static double rdd(void) { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
static void pr(float x) { printf(" %a", (double)x); }
int main() {
    char op[32];
    while (scanf("%31s", op) == 1) {
        std::string o(op);
        if (o == "two_sum") { float a = rd(), b = rd(); df s = two_sum(a, b); pr(s.hi); pr(s.lo); }
        else if (o == "add" || o == "add_fast" || o == "mul") {
            df a{rd(), rd()}, b{rd(), rd()};
            df r = o == "add" ? df_add(a, b) : o == "mul" ? df_mul(a, b) : df_add_fast(a, b);
            pr(r.hi); pr(r.lo);
        } else if (o == "sqrt" || o == "rcp") {
            df a{rd(), rd()};
            df r = o == "sqrt" ? df_sqrt(a) : df_rcp(a);
            pr(r.hi); pr(r.lo);
        } else if (o == "pivot") {
            df d{rd(), rd()}, l, il;
            df_pivot(d, l, il);
            pr(l.hi); pr(l.lo); pr(il.hi); pr(il.lo);
        } else if (o == "from") { df r = df_from(rdd()); pr(r.hi); pr(r.lo); }
        else if (o == "grid") { double x = rdd(); float M = rd(); df r = df_on_grid(x, M); pr(r.hi); pr(r.lo); }
        else if (o == "anchor") { pr(anc_anchor(rd())); }
        else if (o == "anc") {  // anc C a.hi a.lo n then n terms: sign x.hi x.lo y.hi y.lo
            float C = rd();
            df a{rd(), rd()};
            int n = (int)rd();
            anc s = anc_init(a, C);
            for (int k = 0; k < n; ++k) {
                float sg = rd();
                df x{rd(), rd()}, y{rd(), rd()};
                if (sg > 0) anc_add_prod(s, x, y); else anc_sub_prod(s, x, y);
            }
            pr(s.h); pr(s.l);
        } else if (o == "sq") {  // anc C a.hi a.lo n then n pairs (h, l): the sum of (h + l)^2
            float C = rd();
            df a{rd(), rd()};
            int n = (int)rd();
            anc s = anc_init(a, C);
            for (int k = 0; k < n; ++k) { float h = rd(), l = rd(); anc_add_sq(s, h, l); }
            pr(s.h); pr(s.l);
        } else return 3;
        printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    text = hc.cut("common.cuh", "struct df {", "// Precision policy") + DRIVER
    exe = hc.build(tmp_path_factory.mktemp("dfloat"), "dfloat_host", text)

    def call(lines):
        out = hc.run(exe, "\n".join(lines) + "\n")
        return [[float.fromhex(t) for t in ln.split()] for ln in out.splitlines()]

    return call


def _h(x: float) -> str:
    return float(np.float32(x)).hex()


def _df(v: float):
    hi = float(np.float32(v))
    return hi, float(np.float32(v - hi))


def _rel(got: Fr, want: Fr) -> float:
    return abs(float((got - want) / want)) if want != 0 else abs(float(got))


def _rand_df(R, lo=-3.0, hi=3.0):
    return _df(R.uniform(lo, hi) * 2.0 ** R.randint(-6, 6))


def test_error_free_transforms_are_exact(run):
    R = random.Random(1)
    pairs = [(np.float32(R.uniform(-1, 1) * 2.0 ** R.randint(-30, 30)),
              np.float32(R.uniform(-1, 1) * 2.0 ** R.randint(-30, 30))) for _ in range(2000)]
    out = run([f"two_sum {_h(a)} {_h(b)}" for a, b in pairs])
    for (a, b), (s, e) in zip(pairs, out):
        assert Fr(s) + Fr(e) == Fr(float(a)) + Fr(float(b))
        assert s == float(np.float32(float(a) + float(b)))  # the high word is the rounded sum
    xs = [R.uniform(-1, 1) * 2.0 ** R.randint(-20, 20) for _ in range(500)]
    for x, (h, l) in zip(xs, run([f"from {x.hex()}" for x in xs])):
        assert abs(float(Fr(h) + Fr(l) - Fr(x))) <= 2.0 ** -47 * abs(x)


@pytest.mark.parametrize("op", ["add", "mul"])
def test_double_float_add_and_multiply_keep_44_bits(op, run):
    R = random.Random(2)
    ops = [(_rand_df(R), _rand_df(R)) for _ in range(3000)]
    out = run([f"{op} {_h(a[0])} {_h(a[1])} {_h(b[0])} {_h(b[1])}" for a, b in ops])
    worst = 0.0
    for (a, b), (h, l) in zip(ops, out):
        A, B = Fr(a[0]) + Fr(a[1]), Fr(b[0]) + Fr(b[1])
        want = A + B if op == "add" else A * B
        if op == "add":  # error relative to the larger operand (cancellation is exact)
            err = abs(float(Fr(h) + Fr(l) - want)) / max(abs(float(A)), abs(float(B)))
        else:
            err = _rel(Fr(h) + Fr(l), want)
        worst = max(worst, err)
        assert abs(l) <= 2.0 ** -23 * abs(h) or h == 0  # normalised result
    assert worst <= 2.0 ** -44, worst


def test_fast_add_of_same_sign_terms(run):
    R = random.Random(3)
    ops = [(_df(R.uniform(0, 4)), _df(R.uniform(0, 4))) for _ in range(2000)]
    out = run([f"add_fast {_h(a[0])} {_h(a[1])} {_h(b[0])} {_h(b[1])}" for a, b in ops])
    for (a, b), (h, l) in zip(ops, out):
        want = Fr(a[0]) + Fr(a[1]) + Fr(b[0]) + Fr(b[1])
        assert _rel(Fr(h) + Fr(l), want) <= 2.0 ** -44


def test_square_root_reciprocal_and_pivot(run):
    R = random.Random(4)
    vals = [_df(R.uniform(1e-6, 1.0) * 2.0 ** R.randint(-8, 8)) for _ in range(2000)]
    sq = run([f"sqrt {_h(h)} {_h(l)}" for h, l in vals])
    rc = run([f"rcp {_h(h)} {_h(l)}" for h, l in vals])
    pv = run([f"pivot {_h(h)} {_h(l)}" for h, l in vals])
    err_il = []
    for (h, l), (sh, sl), (rh, rl), (lh, ll, ih, il) in zip(vals, sq, rc, pv):
        d = h + l
        s = Fr(sh) + Fr(sl)
        assert abs(float(s * s / (Fr(h) + Fr(l))) - 1.0) <= 2.0 ** -43  # sqrt(d)
        assert _rel(Fr(rh) + Fr(rl), 1 / (Fr(h) + Fr(l))) <= 2.0 ** -43  # 1/d
        inv = Fr(ih) + Fr(il)
        err_il.append(abs(float(inv * inv * (Fr(h) + Fr(l))) - 1.0) / 2)  # rel. error of 1/sqrt(d)
        assert abs(float((Fr(lh) + Fr(ll)) * inv) - 1.0) <= 2.0 ** -43  # l = d / sqrt(d)
        assert d > 0
    # typically 2^-47, at most about 2^-44 (rounding of e and of the correction); without
    # the Newton step's second-order term the median would be 2^-44
    assert np.median(err_il) <= 2.0 ** -46 and max(err_il) <= 2.0 ** -43.5, (np.median(err_il), max(err_il))


def test_anchor_and_grid_split(run):
    R = random.Random(5)
    bs = [R.uniform(0, 1) * 2.0 ** R.randint(-20, 20) for _ in range(500)] + [0.0, 1.0, 2.0, 3.0]
    for b, (C,) in zip(bs, run([f"anchor {_h(b)}" for b in bs])):
        e = C / 6
        assert e == 2.0 ** round(np.log2(e)) and e > float(np.float32(b)) and (b == 0 or e <= 2 * float(np.float32(b)))
    # high words on the grid of [M, 2M): differences of two of them are exact in FP32
    M = 1.5 * 2.0 ** -5
    xs = [R.uniform(-1, 1) * 2.0 ** -6 for _ in range(400)]
    g = run([f"grid {x.hex()} {_h(M)}" for x in xs])
    for x, (h, l) in zip(xs, g):
        assert abs(float(Fr(h) + Fr(l) - Fr(x))) <= 2.0 ** (-5 - 47)
    for (h1, _), (h2, _) in zip(g[::2], g[1::2]):
        assert float(np.float32(h1 - h2)) == h1 - h2


@pytest.mark.parametrize("n", [8, 32, 96])
def test_anchored_accumulator_error_per_step(n, run):
    """Cholesky-row-like sums: unit-bounded operands whose partial sums stay below B;
    the error of (h - C) + l against the exact sum of the double-float products is
    about 2^-46 2^e per multiply-add (C = 6 2^e); asserted with a factor 4 margin."""
    R = random.Random(6 + n)
    lines, exact, bounds = [], [], []
    for _ in range(300):
        a = _df(R.uniform(0.5, 1.0))
        terms = [(R.choice((-1.0, 1.0)), _df(R.uniform(-1, 1) / np.sqrt(n)), _df(R.uniform(-1, 1) / np.sqrt(n)))
                 for _ in range(n)]
        s = Fr(a[0]) + Fr(a[1])
        B = abs(float(s))
        for sg, x, y in terms:
            s += int(sg) * (Fr(x[0]) + Fr(x[1])) * (Fr(y[0]) + Fr(y[1]))
            B = max(B, abs(float(s)))
        C = run([f"anchor {_h(B)}"])[0][0]
        lines.append(f"anc {_h(C)} {_h(a[0])} {_h(a[1])} {n} "
                     + " ".join(f"{sg} {_h(x[0])} {_h(x[1])} {_h(y[0])} {_h(y[1])}" for sg, x, y in terms))
        exact.append(s)
        bounds.append((B, C))
    worst = 0.0
    for (h, l), s, (B, C) in zip(run(lines), exact, bounds):
        got = (Fr(h) - Fr(C)) + Fr(l)
        assert B < C / 6 <= 2 * B
        worst = max(worst, abs(float(got - s)) / (C / 6 * n))
    assert worst <= 2.0 ** -44, worst


def test_anchored_sum_of_squares(run):
    """anc_add_sq adds (h + l)^2 of an unnormalised pair: the running norm |L^-1 c|^2."""
    R = random.Random(7)
    lines, exact = [], []
    for _ in range(300):
        n = 32
        pairs = [(float(np.float32(R.uniform(-1, 1) / 6)), float(np.float32(R.uniform(-1, 1) * 2.0 ** -26)))
                 for _ in range(n)]
        s = sum((Fr(h) + Fr(l)) ** 2 for h, l in pairs)
        C = run([f"anchor {_h(float(s))}"])[0][0]
        lines.append(f"sq {_h(C)} 0x0p+0 0x0p+0 {n} " + " ".join(f"{_h(h)} {_h(l)}" for h, l in pairs))
        exact.append((s, C))
    for (h, l), (s, C) in zip(run(lines), exact):
        assert abs(float((Fr(h) - Fr(C)) + Fr(l) - s)) <= 32 * 2.0 ** -45 * float(s)
