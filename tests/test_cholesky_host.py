"""The lens kernel's bordered Cholesky factorisations (csrc/lens.cuh:
factor_bordered and the three forms it chooses between: right-looking FP64
for N <= 32, split left-looking FP64 above, and the anchored double-float form
of the mixed path) run on a host warp of 32 threads and compared with numpy on
kriging systems built by the oracle from the paper's covariances (Eqs.
fundamental_variance, spins_correl; the nugget of Sec. 2.4) at Nside 4096
(spin 2, the c3 spectra) and Nside 2048 (spin 0, the c2 spectra), for every
stencil size the kernels are built for.

The factor works on the matrix bordered by two right-hand-side rows (the
target covariances c and the conjugated data y); the bordered rows come back
as conj(L^-1 conj(row)), from which the estimate is value = sum m_c conj(m_y)
and variance / xi(0) = 1 - sum |m_c|^2 (Eqs. major_eq, gaussvar_pol)."""
import numpy as np
import pytest

import workloads as wl
from oracle import healpix as hp
from oracle import kriging as kr
from oracle import xi
from tests import host_compile as hc

DRIVER = r"""
#include <type_traits>
using namespace flints;
static double rd() { char b[64]; if (scanf("%63s", b) != 1) exit(2); return strtod(b, nullptr); }
template <class R> static typename Ops<R>::T in(double x) { return Ops<R>::from(x); }
template <class R> static double out(typename Ops<R>::T x) { return Ops<R>::to(x); }

template <int N, class R, bool CPLX> static void one() {
    using T = typename Ops<R>::T;
    using Elem = typename std::conditional<CPLX, Cx<T>, T>::type;
    constexpr int M = N * (N + 1) / 2 + 2 * N;
    std::vector<Elem> mat(M);
    for (int e = 0; e < M; ++e) {
        if constexpr (CPLX) {
            const double re = rd(), im = rd();
            mat[e].re = in<R>(re);
            mat[e].im = in<R>(im);
        } else {
            mat[e] = in<R>(rd());
        }
    }
    bool ok = false;
    run_warp([&](int lane) {
        const bool r = factor_bordered<N, 2, R>(mat.data(), lane);
        if (lane == 0) ok = r;
    });
    printf("%d", ok ? 1 : 0);
    for (int e = N * (N + 1) / 2; e < M; ++e) {  // the two bordered rows
        if constexpr (CPLX) printf(" %a %a", out<R>(mat[e].re), out<R>(mat[e].im));
        else printf(" %a", out<R>(mat[e]));
    }
    printf("\n");
}

template <int N> static void dispatch(int prec, int cplx) {
    if (prec == 0) { if (cplx) one<N, double, true>(); else one<N, double, false>(); }
    else { if (cplx) one<N, df, true>(); else one<N, df, false>(); }
}

int main() {
    int N, cplx, prec;
    while (scanf("%d %d %d", &N, &cplx, &prec) == 3) {
        switch (N) {
            case 16: dispatch<16>(prec, cplx); break;
            case 24: dispatch<24>(prec, cplx); break;
            case 32: dispatch<32>(prec, cplx); break;
            case 48: dispatch<48>(prec, cplx); break;
            default: return 3;
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    if hc.compiler() is None:
        pytest.skip("no host C++ compiler")
    text = ("#include <vector>\n#include <type_traits>\n#include <math.h>\nnamespace flints {\n"
            "constexpr unsigned FULL = 0xffffffffu;\n"
            + hc.cut("common.cuh", "struct df {", "// HEALPix RING geometry")
            + hc.cut("lens.cuh", "template <class T>\nstruct Cx {", "template <int K>\nstruct Shape", False)
            + hc.cut("lens.cuh", "template <int K>\n__device__ __forceinline__ int tri(",
                     "// ------------------------------------------------------------------ helpers", False)
            + hc.cut("lens.cuh", "// Split left-looking Cholesky",
                     "// Returns false when a pivot of S + nugget I is not positive.", False)
            + "\n}\n" + DRIVER)
    exe = hc.build(tmp_path_factory.mktemp("chol"), "chol_host", text, warp="threads")

    def call(N, cplx, prec, packed):
        vals = np.stack([packed.real, packed.imag], -1).ravel() if cplx else packed.real
        out = hc.run(exe, f"{N} {int(cplx)} {prec} " + " ".join(float(x).hex() for x in vals) + "\n").split()
        nums = np.array([float.fromhex(t) for t in out[1:]])
        rows = nums[0::2] + 1j * nums[1::2] if cplx else nums
        return out[0] == "1", rows.reshape(2, N)

    return call


def _system(spin, K, seed):
    """S + nI, the target covariances c and a field realisation y on one stencil of
    the Nside 4096 (spin 2) or Nside 2048 (spin 0) workload."""
    W = wl.C3 if spin == 2 else wl.C2
    cl, bb = W.cl()
    weight = np.abs(cl) + (np.abs(bb) if bb is not None else 0.0)
    t_max, n = xi.grid_rule(weight, K, W.nside)
    tab = (xi.spin2_tables(cl, bb, t_max, n)[0] if spin == 2 else xi.spin0_table(cl, t_max, n)[0])
    rng = np.random.default_rng(seed)
    pix = wl.sample_pixels(W.npix, 1, seed)
    tv = kr.displace(W.nside, pix, rng.normal(size=(1, 2)) * wl.DEFLECTION_RMS / np.sqrt(2))
    idx, _ = kr.knn(W.nside, tv, K)
    X = hp.pix2vec(W.nside, idx)[0]
    S = tab(kr._chord2(X[:, None, :], X[None, :, :])).astype(complex)
    c = tab(kr._chord2(tv[0][None, :], X)).astype(complex)
    if spin == 2:
        S = S * kr.pair_phase(X[:, None, :], X[None, :, :], 2)
        c = c * kr.pair_phase(np.broadcast_to(tv[0], X.shape), X, 2)
    S[np.arange(K), np.arange(K)] = 1.0
    A = S + kr.EPS_NUGGET * np.eye(K)
    g = rng.normal(size=K) + (1j * rng.normal(size=K) if spin == 2 else 0)
    y = np.linalg.cholesky(A) @ (g / np.sqrt(2 if spin == 2 else 1))
    return A, c, y


def _pack(A, c, y):
    K = A.shape[0]
    tri = np.concatenate([A[i, :i + 1] for i in range(K)])
    return np.concatenate([tri, c, np.conj(y)])  # rows K and K + 1: c and conj(y)


def _estimate(rows, spin):
    m_c, m_y = rows
    value = np.sum(m_c * np.conj(m_y)) if spin == 2 else np.sum(m_c * m_y).real
    return value, 1.0 - np.sum(np.abs(m_c) ** 2)


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("K", [16, 24, 32, 48])
def test_factor_and_estimate_match_numpy(spin, K, run):
    for seed in range(2):
        A, c, y = _system(spin, K, 1000 * K + seed)
        L = np.linalg.cholesky(A)
        ref = np.conj(np.linalg.solve(L, np.conj(np.stack([c, np.conj(y)], 1)))).T  # conj(L^-1 conj(row))
        v_ref, q_ref = _estimate(ref, spin)
        for prec, tol in ((0, 1e-9), (1, 1e-7)):
            ok, rows = run(K, spin == 2, prec, _pack(A, c, y))
            assert ok
            v, q = _estimate(rows, spin)
            # in units of the field's standard deviation (1) and of xi(0) (1): the parity
            # tolerances are 1e-9 (FP64) and 1e-6 (mixed)
            assert abs(v - v_ref) <= tol and abs(q - q_ref) <= tol, (prec, abs(v - v_ref), abs(q - q_ref))
            # the target-covariance row itself, entry by entry
            assert np.max(np.abs(rows[0] - ref[0])) <= 1e3 * tol


def test_indefinite_matrix_is_reported(run):
    A, c, y = _system(0, 16, 5)
    A = A.copy()
    A[3, 3] = -1.0  # a negative pivot
    for prec in (0, 1):
        ok, _ = run(16, False, prec, _pack(A, c, y))
        assert not ok
