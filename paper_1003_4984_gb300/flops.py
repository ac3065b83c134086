"""Algorithmic operation counts and roofline peaks for the lens kernels.

Counting convention (used for every roofline fraction reported by the bench):

* a fused multiply-add counts 2 flops, any other add, subtract or multiply 1;
  square roots, reciprocals and the table index count 2 each;
* FP64 path: the arithmetic of the method itself, per target point, with K
  stencil members and P = K(K-1)/2 pairs:
    - left-looking Cholesky: (K^3 - K)/6 multiply-adds plus K pivots and P
      scalings; complex Hermitian (spin 2) multiply-adds are 4 real ones;
    - two forward solves (c and y): P multiply-adds each, K scalings each;
    - covariance assembly: per pair the squared chord (3 sub, 3 mul, 2 add)
      and the cubic table (index + 3 fma); spin 2 adds the parallel-transport
      phase (4 projections of 2 fma + 1 mul, squares and products: 48 flops;
      spin 1 is counted the same);
      the K target entries likewise (their chords come from the search);
    - value and variance: 2 dot products of length K;
* augmented spin 2: a real system of size N = 2K with three right-hand sides:
  (N^3 - N)/6 multiply-adds and N pivots, three forward solves of N(N-1)/2
  multiply-adds, per pair of stencil members the chord, two tables (xi+ and
  xi-), both phases (56 flops) and four entries (8), and three dot products of
  length N;
* mixed path: the same steps executed in double-float arithmetic on the FP32
  pipe, each double-float operation costed in FP32 flops: multiply-accumulate
  into an accumulator 15 (one TwoProduct with cross terms, one TwoSum, two
  adds), add 20, multiply 10, square root or reciprocal 35.  These are the
  costs of plain double-float operations: where the kernel accumulates onto
  an anchor (Cholesky rows, solves, covariance rows; about 6 FP32
  instructions per real multiply-add) it executes less, so the count is an
  upper estimate of the emulation's work, and the measured figure is the
  warp-instruction count of an ncu capture.
"""
from __future__ import annotations

# double-float operation costs in FP32 flops
DF_MAC, DF_ADD, DF_MUL, DF_SPECIAL = 15, 20, 10, 35


def fp64_flops(K: int, spin: int) -> float:
    P = K * (K - 1) / 2
    macs = (K ** 3 - K) / 6
    cm = 4 if spin != 0 else 1  # real multiply-adds per (complex) multiply-add
    chol = 2 * cm * macs + 2 * 2 * K + (2 if spin != 0 else 1) * P
    solve = 2 * (2 * cm * P + (2 if spin != 0 else 1) * K)
    pair = 8 + 8 + (48 + 2 if spin != 0 else 0)
    assembly = pair * P + (8 + (50 if spin != 0 else 0)) * K
    dots = 2 * 2 * K * (2 if spin != 0 else 1)
    return chol + solve + assembly + dots


def mixed_fp32_flops(K: int, spin: int) -> float:
    P = K * (K - 1) / 2
    macs = (K ** 3 - K) / 6
    cm = 4 if spin != 0 else 1
    chol = cm * macs * DF_MAC + K * 2 * DF_SPECIAL + P * (2 if spin != 0 else 1) * DF_MUL
    solve = 2 * (cm * P * DF_MAC + K * (2 if spin != 0 else 1) * DF_MUL)
    chord = 3 * DF_ADD + 3 * DF_MUL + 2 * DF_ADD
    table = DF_MUL + 3 * (DF_MUL + DF_ADD)
    phase = (27 * DF_MUL + 16 * DF_ADD + DF_SPECIAL) if spin != 0 else 0
    entry = 2 * DF_MUL if spin != 0 else 0
    assembly = P * (chord + table + phase + entry) + K * (table + phase + entry)
    return chol + solve + assembly


# peaks (TFLOP/s) derived from the unit counts and the 2070 MHz maximum SM clock:
# 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz; FP64 at the 1.25 TFLOP/s nominal rate.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def augmented_flops(K: int, mixed: bool) -> float:
    """Augmented spin-2 estimator: FP64 flops, or FP32 flops of its double-float form."""
    N = 2 * K
    P = K * (K - 1) / 2
    macs = (N ** 3 - N) / 6
    if not mixed:
        chol = 2 * macs + 2 * 2 * N + N * (N - 1) / 2
        solve = 3 * (2 * N * (N - 1) / 2 + N)
        assembly = P * (8 + 2 * 8 + 56 + 8) + K * (2 * 8 + 56 + 8)
        return chol + solve + assembly + 3 * 2 * N
    chol = macs * DF_MAC + N * 2 * DF_SPECIAL + N * (N - 1) / 2 * DF_MUL
    solve = 3 * (N * (N - 1) / 2 * DF_MAC + N * DF_MUL)
    chord = 3 * DF_ADD + 3 * DF_MUL + 2 * DF_ADD
    table = DF_MUL + 3 * (DF_MUL + DF_ADD)
    phases = 24 * DF_MUL + 14 * DF_ADD + DF_SPECIAL
    entries = 4 * DF_MUL + 4 * DF_ADD
    return chol + solve + P * (chord + 2 * table + phases + entries) + K * (2 * table + phases + entries)


def paper_fp64_flops(K: int, spin: int = 0) -> float:
    """FP64 flops per target of the tabulated-inverse route: the K covariances
    to the target (chord^2: 3 subtractions, 3 products, 2 additions; cubic table
    evaluation: 2 for the abscissa, 3 multiply-adds; spin 2: the transport
    phase, 34 flops, and 2 products), z_c = L^-1 conj(c) and z_y = L^-1 y
    (K (K + 1) / 2 multiply-adds each, complex for spin 2: 4 real ones), value
    and variance (2K multiply-adds, complex for spin 2)."""
    cm = 4 if spin else 1
    return K * (8 + 2 + 6 + (36 if spin else 0)) + cm * 2 * K * (K + 1) + cm * 2 * 2 * K


def paper_mixed_fp32_flops(K: int, spin: int = 0) -> float:
    """FP32 flops per target of the tabulated-inverse route in double-float: K
    chords (3 differences, 3 squares, 2 sums) and table lookups (a product and
    three multiply-adds), spin 2 also the member position (2 products) and the
    transport phase (27 products, 16 sums, a reciprocal) times the lookup (2
    products); K (K + 1) multiply-accumulates for z_c and z_y (4 real ones each
    for spin 2), and the two dots (2K products and sums, complex for spin 2)."""
    chord = 3 * DF_ADD + 3 * DF_MUL + 2 * DF_ADD
    table = DF_MUL + 3 * (DF_MUL + DF_ADD)
    cm = 4 if spin else 1
    phase = (2 * DF_MUL + 27 * DF_MUL + 16 * DF_ADD + DF_SPECIAL + 2 * DF_MUL) if spin else 0
    return K * (chord + table + phase) + cm * K * (K + 1) * DF_MAC + cm * 2 * K * (DF_MUL + DF_ADD)


def paper_augmented_fp64_flops(K: int) -> float:
    """FP64 flops per target of the augmented tabulated-inverse route: K member
    terms (chord 8, two table lookups 2 x 5, the two phases 40, the four
    real-form entries 8), three triangular products with the real 2K x 2K
    factor (3 x 2K (2K + 1) / 2 multiply-adds) and the dots (3 x 2K)."""
    N = 2 * K
    return K * (8 + 10 + 40 + 8) + 3 * 2 * N * (N + 1) / 2 + 3 * 2 * N
