"""Pins for the FP64 oracle: checks against what the paper and the mathematics fix.

Each pin is a plain function taking the loaded oracle library, so that the same pins can be
run against builds of the oracle with a mistake planted in them (test_oracle_mutants.py).
None of them re-types the oracle's own formula: they use closed forms, invariants, exact
rational arithmetic of the *other* form of the cost (Eq. (2)), dense-matrix formulations and
brute force.
"""

from __future__ import annotations

import math
from fractions import Fraction

import os

import numpy as np

import oracle
from synth import blurred_noise, make_pair

SIG_S, SIG_R = 20.0, 0.1


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------------------
# window sums (Sec. IV-B-1)

def pin_window_sums_routes(lib):
    """Method 1 (direct) and Method 2 (integral image) agree exactly, and both agree with a
    numpy edge-padded sliding-window sum, for several radii and an extended centre range."""
    rng = _rng(11)
    for (h, w, r, xb, xe) in [(7, 9, 1, 0, 9), (13, 17, 4, -20, 17), (5, 3, 3, -2, 5),
                              (1, 1, 2, 0, 1)]:
        img = rng.integers(0, 256, (h, w), dtype=np.uint8)
        S1, Q1 = oracle.window_sums(img, r, xb, xe, lib=lib)
        S2, Q2 = oracle.window_sums(img, r, xb, xe, lib=lib, integral=True)
        assert np.array_equal(S1, S2) and np.array_equal(Q1, Q2)
        pad_l = r + max(0, -xb)
        padded = np.pad(img.astype(np.int64), ((r, r), (pad_l, r + max(0, xe - w))),
                        mode="edge")
        l = 2 * r + 1
        win = np.lib.stride_tricks.sliding_window_view(padded, (l, l))
        cols = np.arange(xb, xe) + pad_l - r
        assert np.array_equal(S1, win.sum(axis=(2, 3))[:, cols])
        assert np.array_equal(Q1, (win ** 2).sum(axis=(2, 3))[:, cols])


def pin_window_sums_constant(lib):
    img = np.full((6, 8), 37, np.uint8)
    S, Q = oracle.window_sums(img, 2, lib=lib)
    assert (S == 25 * 37).all() and (Q == 25 * 37 * 37).all()


# ---------------------------------------------------------------------------------------
# ZNCC (Sec. III-A, Eq. (1)); Eq. (2) is the independent exact route

def _eq2_exact(L, R, r, x, y, d):
    """Eq. (2) in exact rationals: (sum Pi - l^2 mean_R mean_T) / (sigma_R sigma_T), with
    sigma^2 = sum I^2 - l^2 mean^2; only the final square root is taken in floating point."""
    H, W = L.shape
    l2 = (2 * r + 1) ** 2

    def px(img, u, v):
        return int(img[min(max(v, 0), H - 1), min(max(u, 0), W - 1)])

    wl = [px(L, x + i, y + j) for j in range(-r, r + 1) for i in range(-r, r + 1)]
    wr = [px(R, x - d + i, y + j) for j in range(-r, r + 1) for i in range(-r, r + 1)]
    mean_l, mean_r = Fraction(sum(wl), l2), Fraction(sum(wr), l2)
    num = sum(a * b for a, b in zip(wl, wr)) - l2 * mean_l * mean_r
    var_l = sum(a * a for a in wl) - l2 * mean_l * mean_l
    var_r = sum(b * b for b in wr) - l2 * mean_r * mean_r
    if var_l == 0 or var_r == 0:
        return 0.0
    # num / sqrt(var_l var_r), with num^2 / (var_l var_r) exact before the root
    sign = 1.0 if num >= 0 else -1.0
    return sign * math.sqrt(float(num * num / (var_l * var_r)))


def pin_zncc_eq2_exact(lib):
    rng = _rng(12)
    L = rng.integers(0, 256, (6, 8), dtype=np.uint8)
    R = rng.integers(0, 256, (6, 8), dtype=np.uint8)
    L[0:3, 0:3] = 90            # a flat patch: zero-variance windows exist
    for r, D in [(1, 4), (2, 5)]:
        C = oracle.zncc_volume(L, R, D, r, nthreads=2, lib=lib)
        for y in range(6):
            for x in range(8):
                for d in range(D):
                    ref = _eq2_exact(L, R, r, x, y, d)
                    assert abs(C[y, x, d] - ref) <= 1e-12, (r, x, y, d, C[y, x, d], ref)


def pin_zncc_identical_windows(lib):
    """right == left, d = 0: every window with non-zero variance correlates to exactly 1."""
    rng = _rng(13)
    L = blurred_noise(rng, 20, 30)
    C = oracle.zncc_volume(L, L, 3, 2, lib=lib)
    assert np.allclose(C[:, :, 0], 1.0, atol=1e-12)


def pin_zncc_affine_invariance(lib):
    """I_T -> a*I_T + b (a > 0, no clipping) leaves the cost unchanged; 255 - I_T negates it;
    every value lies in [-1, 1]."""
    rng = _rng(14)
    L = rng.integers(0, 256, (12, 20), dtype=np.uint8)
    R = rng.integers(0, 127, (12, 20), dtype=np.uint8)
    C = oracle.zncc_volume(L, R, 6, 2, lib=lib)
    C_aff = oracle.zncc_volume(L, (2 * R.astype(np.int32) + 3).astype(np.uint8), 6, 2, lib=lib)
    C_neg = oracle.zncc_volume(L, (255 - R).astype(np.uint8), 6, 2, lib=lib)
    assert np.allclose(C, C_aff, atol=1e-12)
    assert np.allclose(C, -C_neg, atol=1e-12)
    assert np.abs(C).max() <= 1.0 + 1e-12
    # also a gain on the reference side
    C_aff_l = oracle.zncc_volume((L // 2 + 60).astype(np.uint8), R, 6, 2, lib=lib)
    Lh = (L // 2).astype(np.uint8)
    C_half = oracle.zncc_volume(Lh, R, 6, 2, lib=lib)
    assert np.allclose(C_aff_l, C_half, atol=1e-12)


def pin_zncc_zero_variance(lib):
    rng = _rng(15)
    L = rng.integers(0, 256, (9, 12), dtype=np.uint8)
    R = rng.integers(0, 256, (9, 12), dtype=np.uint8)
    L[:, :] = 50                       # whole reference flat -> every cost is the fixed 0
    C = oracle.zncc_volume(L, R, 4, 1, lib=lib)
    assert (C == 0.0).all()
    R2 = R.copy()
    R2[3:6, 4:7] = 200                 # one flat target window centred at (5, 4)
    L2 = rng.integers(0, 256, (9, 12), dtype=np.uint8)
    C2 = oracle.zncc_volume(L2, R2, 4, 1, lib=lib)
    # centre of the flat target window is x - d = 5 at y = 4
    for d in range(4):
        assert C2[4, 5 + d, d] == 0.0


def pin_zncc_at_matches_volume(lib):
    rng = _rng(16)
    L = rng.integers(0, 256, (7, 11), dtype=np.uint8)
    R = rng.integers(0, 256, (7, 11), dtype=np.uint8)
    C = oracle.zncc_volume(L, R, 5, 2, lib=lib)
    for (x, y, d) in [(0, 0, 0), (10, 6, 4), (3, 2, 4), (5, 5, 1)]:
        assert oracle.zncc_at(L, R, 2, x, y, d, lib=lib) == C[y, x, d]


def pin_zncc_plane_subset(lib):
    rng = _rng(17)
    L = rng.integers(0, 256, (7, 11), dtype=np.uint8)
    R = rng.integers(0, 256, (7, 11), dtype=np.uint8)
    C = oracle.zncc_volume(L, R, 9, 1, lib=lib)
    Cs = oracle.zncc_volume(L, R, 9, 1, planes=[8, 0, 3], lib=lib)
    assert np.array_equal(Cs, C[:, :, [8, 0, 3]])


def pin_zncc_shift_recovery(lib):
    """A textured image shifted by a known disparity is recovered by WTA on the raw cost."""
    p = make_pair(40, 96, 16, seed=21, disp="const", const_disp=7, gain=1.0, offset=0.0,
                  noise=0.0)
    C = oracle.zncc_volume(p.left, p.right, 16, 3, lib=lib)
    disp, _, _ = oracle.wta(C, lib=lib)
    inner = disp[3:-3, 7 + 3 + 1:-3]
    assert (inner == 7).mean() >= 0.99


# ---------------------------------------------------------------------------------------
# DT (Sec. III-B, Eqs. (3)-(11))

def _K(sigma_s):
    return math.exp(-1.0 / sigma_s)


def pin_dt_weight_forms(lib):
    """Eq. (11) (K exp(-|dI|/sigma_r)) equals Eqs. (7)-(10) (a^(1 + sigma_s/sigma_r |dI|));
    a guide step of 255 with sigma_r = 0.1 gives K e^-10 across the edge; a flat guide gives
    K everywhere; undefined borders are 0."""
    g = np.zeros((4, 6), np.uint8)
    g[:, 3:] = 255
    w11 = oracle.dt_weights(g, SIG_S, SIG_R, form=0, lib=lib)
    w7 = oracle.dt_weights(g, SIG_S, SIG_R, form=1, lib=lib)
    assert np.allclose(w11, w7, rtol=1e-12, atol=0)
    K = _K(SIG_S)
    WL, WR, WU, WD = w11
    assert math.isclose(WL[0, 3], K * math.exp(-10.0), rel_tol=1e-12)
    assert math.isclose(WR[0, 2], K * math.exp(-10.0), rel_tol=1e-12)
    assert math.isclose(WL[0, 2], K, rel_tol=1e-12) and math.isclose(WR[0, 3], K, rel_tol=1e-12)
    assert (WL[:, 0] == 0).all() and (WR[:, -1] == 0).all()
    assert (WU[0, :] == 0).all() and (WD[-1, :] == 0).all()
    assert np.allclose(WU[1:, :], K) and np.allclose(WD[:-1, :], K)
    rng = _rng(18)
    g2 = rng.integers(0, 256, (5, 7), dtype=np.uint8)
    wl2, wr2, wu2, wd2 = oracle.dt_weights(g2, 5.0, 0.2, lib=lib)
    # the edge between (x, y) and (x+1, y) carries one weight: W_R(x) = W_L(x+1)
    assert np.array_equal(wr2[:, :-1], wl2[:, 1:])
    assert np.array_equal(wd2[:-1, :], wu2[1:, :])
    gd = g2.astype(np.float64) / 255.0
    assert np.allclose(wl2[:, 1:], _K(5.0) * np.exp(-np.abs(gd[:, 1:] - gd[:, :-1]) / 0.2),
                       rtol=1e-14, atol=0)


def _line_pair_closed(Wn, K, s, x0=None):
    """Flat guide, one line of length Wn: the response of L2R then R2L (scaled, factor s per
    pass) to a unit impulse at x0 (or to the all-ones line when x0 is None), in closed form
    from geometric sums."""
    out = np.zeros(Wn)
    for x in range(Wn):
        if x0 is None:
            # L2R of ones: 1 - K^(j+1); R2L: s * sum_{j>=x} K^(j-x) (1 - K^(j+1))
            out[x] = (1 - K ** (Wn - x)) - s * K ** (x + 1) * (1 - K ** (2 * (Wn - x))) / (1 - K * K)
        else:
            m = max(x, x0)
            out[x] = s * s * K ** (-x - x0) * (K ** (2 * m) - K ** (2 * Wn)) / (1 - K * K)
    return out


def pin_dt_impulse_closed_form(lib):
    """Flat guide: one DT iteration on an impulse is the outer product of the 1-D closed-form
    line-pair responses (rows, then columns); an H = 1 image reduces to the 1-D form times s^2
    (the vertical passes of a single row only scale)."""
    K = _K(SIG_S)
    s = 1 - K
    H, W = 9, 23
    g = np.full((H, W), 128, np.uint8)
    w = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    x0, y0 = 7, 3
    C = np.zeros((H, W, 1))
    C[y0, x0, 0] = 1.0
    out = oracle.dt_aggregate(C, w, SIG_S, 1, lib=lib)[:, :, 0]
    ref = np.outer(_line_pair_closed(H, K, s, y0), _line_pair_closed(W, K, s, x0))
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-300)
    g1 = np.full((1, W), 9, np.uint8)
    w1 = oracle.dt_weights(g1, SIG_S, SIG_R, lib=lib)
    C1 = np.zeros((1, W, 1))
    C1[0, x0, 0] = 1.0
    out1 = oracle.dt_aggregate(C1, w1, SIG_S, 1, lib=lib)[0, :, 0]
    assert np.allclose(out1, s * s * _line_pair_closed(W, K, s, x0), rtol=1e-12, atol=0)


def pin_dt_constant_closed_form(lib):
    """Flat guide, all-ones input, one iteration: the outer product of the 1-D closed forms
    (L2R of ones is 1 - K^(x+1) because s = 1 - K)."""
    K = _K(SIG_S)
    s = 1 - K
    H, W = 6, 31
    g = np.full((H, W), 3, np.uint8)
    w = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    out = oracle.dt_aggregate(np.ones((H, W, 1)), w, SIG_S, 1, lib=lib)[:, :, 0]
    ref = np.outer(_line_pair_closed(H, K, s), _line_pair_closed(W, K, s))
    assert np.allclose(out, ref, rtol=1e-12, atol=0)


def _pass_matrix(weights_line, s, forward):
    """Dense matrix of one recurrence along a line, from its closed form: output x receives
    input x' (x' <= x for a forward pass) with factor s * prod of the weights at the
    positions strictly between x' and x on the scan path, ending at x."""
    n = len(weights_line)
    M = np.zeros((n, n))
    for x in range(n):
        for xp in range(n):
            if forward and xp <= x:
                M[x, xp] = s * np.prod(weights_line[xp + 1:x + 1])
            elif not forward and xp >= x:
                M[x, xp] = s * np.prod(weights_line[x:xp])
    return M


def pin_dt_dense_matrix(lib):
    """On a textured 5x4 guide, iters = 2, several planes: the oracle equals the explicit
    operator built from the dense pass matrices, applied pass by pass in the paper's order
    (L2R, R2L, U2D, D2U), including linearity across planes."""
    rng = _rng(19)
    H, W, nd = 4, 5, 3
    g = rng.integers(0, 256, (H, W), dtype=np.uint8)
    sig_s, sig_r = 3.0, 0.3
    WL, WR, WU, WD = oracle.dt_weights(g, sig_s, sig_r, lib=lib)
    s = 1 - _K(sig_s)
    C = rng.uniform(-1, 1, (H, W, nd))
    out = oracle.dt_aggregate(C, (WL, WR, WU, WD), sig_s, 2, lib=lib)
    ref = C.copy()
    for _ in range(2):
        for y in range(H):
            ref[y] = _pass_matrix(WL[y], s, True) @ ref[y]
        for y in range(H):
            ref[y] = _pass_matrix(WR[y], s, False) @ ref[y]
        for x in range(W):
            ref[:, x] = _pass_matrix(WU[:, x], s, True) @ ref[:, x]
        for x in range(W):
            ref[:, x] = _pass_matrix(WD[:, x], s, False) @ ref[:, x]
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-15)
    # linearity: DT(aA + bB) = a DT(A) + b DT(B)
    A, B = rng.uniform(-1, 1, (2, H, W, nd))
    lhs = oracle.dt_aggregate(0.3 * A - 1.7 * B, (WL, WR, WU, WD), sig_s, 2, lib=lib)
    rhs = 0.3 * oracle.dt_aggregate(A, (WL, WR, WU, WD), sig_s, 2, lib=lib) - \
        1.7 * oracle.dt_aggregate(B, (WL, WR, WU, WD), sig_s, 2, lib=lib)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-14)


def pin_dt_scaled_vs_literal(lib):
    """The scaled chain equals the literal chain of Eqs. (3)-(6) times (1-K)^(4 iters)."""
    rng = _rng(20)
    g = blurred_noise(rng, 12, 17)
    w = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    C = rng.uniform(-1, 1, (12, 17, 2))
    for iters in (1, 3):
        a = oracle.dt_aggregate(C, w, SIG_S, iters, scaled=True, lib=lib)
        b = oracle.dt_aggregate(C, w, SIG_S, iters, scaled=False, lib=lib)
        assert np.allclose(a, b * (1 - _K(SIG_S)) ** (4 * iters), rtol=1e-11, atol=0)


def pin_dt_bounded_and_plane_independent(lib):
    """|scaled DT(C)| <= DT(1) = A_hat pointwise when |C| <= 1; changing one plane leaves the
    others bit-identical; iters = 0 is the identity."""
    rng = _rng(22)
    g = blurred_noise(rng, 10, 14)
    w = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    C = rng.uniform(-1, 1, (10, 14, 4))
    A = oracle.ones_response(g, SIG_S, SIG_R, 3, lib=lib)
    out = oracle.dt_aggregate(C, w, SIG_S, 3, lib=lib)
    assert (np.abs(out) <= A[:, :, None] * (1 + 1e-12)).all()
    assert (A <= 1 + 1e-12).all() and (A > 0).all()
    C2 = C.copy()
    C2[:, :, 2] = rng.uniform(-1, 1, (10, 14))
    out2 = oracle.dt_aggregate(C2, w, SIG_S, 3, lib=lib)
    assert np.array_equal(out2[:, :, [0, 1, 3]], out[:, :, [0, 1, 3]])
    assert np.array_equal(oracle.dt_aggregate(C, w, SIG_S, 0, lib=lib), C)


def pin_dt_edge_stop(lib):
    """Cost does not leak across a strong guide edge: with an impulse left of a 0/255 step,
    the first pixel past the edge receives at most K e^-10 / (1 - K^2) of the level of the
    last pixel before it (the edge weight, times the geometric R2L echo from the right)."""
    g = np.zeros((3, 20), np.uint8)
    g[:, 10:] = 255
    w = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    C = np.zeros((3, 20, 1))
    C[:, 5, 0] = 1.0
    out = oracle.dt_aggregate(C, w, SIG_S, 1, lib=lib)[:, :, 0]
    K = _K(SIG_S)
    assert out[1, 10] <= out[1, 9] * K * math.exp(-10.0) / (1 - K * K) * (1 + 1e-9)
    # without the edge the same pixel keeps a level of order K
    g[:, 10:] = 0
    w0 = oracle.dt_weights(g, SIG_S, SIG_R, lib=lib)
    out0 = oracle.dt_aggregate(C, w0, SIG_S, 1, lib=lib)[:, :, 0]
    assert out0[1, 10] >= 0.5 * K * out0[1, 9]


# ---------------------------------------------------------------------------------------
# WTA (Sec. III-C, Eq. (WTA1))

def pin_wta_bruteforce_and_ties(lib):
    rng = _rng(23)
    C = rng.uniform(-1, 1, (6, 7, 9))
    disp, best, gap = oracle.wta(C, lib=lib)
    assert np.array_equal(disp, np.argmax(C, axis=2))
    assert np.array_equal(best, C.max(axis=2))
    srt = np.sort(C, axis=2)
    assert np.allclose(gap, srt[:, :, -1] - srt[:, :, -2], atol=1e-15)
    T = np.zeros((2, 3, 5))
    T[0, 0, [1, 3]] = 0.5
    T[1, 2, :] = -0.25
    T[0, 1, [4, 2]] = 0.9
    dt, _, gt = oracle.wta(T, lib=lib)
    assert dt[0, 0] == 1 and dt[1, 2] == 0 and dt[0, 1] == 2 and gt[0, 0] == 0.0
    # a per-pixel offset (FastDT's d_arb argument) does not move the winner
    off = rng.uniform(-5, 5, (6, 7, 1))
    d2, _, _ = oracle.wta(C - off, lib=lib)
    assert np.array_equal(d2, disp)


# ---------------------------------------------------------------------------------------
# end to end

def pin_end_to_end_recovery(lib):
    """Constant disparity 7 on textured noise (no photometric change): >= 99% of interior
    pixels exact with 3 DT iterations; piecewise rectangles with gain/offset/noise: >= 95%
    exact on valid pixels away from rectangle edges."""
    p = make_pair(48, 120, 16, seed=31, disp="const", const_disp=7, gain=1.0, offset=0.0,
                  noise=0.0)
    disp, _ = oracle.run(p.left, p.right, 16, 4, SIG_S, SIG_R, 3, lib=lib)
    assert (disp[4:-4, 16:-4] == 7).mean() >= 0.99
    q = make_pair(96, 320, 32, seed=1, disp="rects")
    d0, _ = oracle.run(q.left, q.right, 32, 4, SIG_S, SIG_R, 0, lib=lib)
    gt = q.gt
    edge = np.zeros_like(q.valid)
    for dy in range(-4, 5):
        for dx in range(-4, 5):
            edge |= np.roll(np.roll(gt, dy, 0), dx, 1) != gt
    m = q.valid & ~edge
    m[:4], m[-4:], m[:, :32 + 4], m[:, -4:] = False, False, False, False
    assert m.sum() > 1000
    assert (d0[m] == gt[m]).mean() >= 0.95


# ---------------------------------------------------------------------------------------
# FastDT storage (Sec. IV-C): the 8-bit code and the near-zero-mean 16-bit store

def pin_fastdt_codec_examples(lib):
    """Codes worked out by hand from the encoding and decoding rules of Sec. IV-C: positive
    values and zero give code 0; 0x8000 keeps bits 14..9 (flag 01); -2048 = 0xF800 has bits
    14..11 all ones and keeps bits 10..5 (flag 10); -128 = 0xFF80 and -1 = 0xFFFF keep bits
    6..1 (flag 11); -2049 = 0xF7FF keeps 111011 from bits 14..9 and decodes to 0xF600."""
    enc = lambda v: oracle.fastdt_encode(v, lib=lib)
    dec = lambda c: oracle.fastdt_decode(c, lib=lib)
    for v in (0, 1, 100, 32767):
        assert enc(v) == 0
    assert dec(0) == 0
    cases = [(-32768, 0x01, -32768), (-2048, 0x02, -2048), (-128, 0x03, -128), (-1, 0xFF, -2),
             (-2, 0xFF, -2), (-2049, (0b111011 << 2) | 1, -2560), (-129, (0b111011 << 2) | 2, -160),
             (-3000, (0b111010 << 2) | 1, -3072)]
    for v, code, back in cases:
        assert enc(v) == code, (v, hex(enc(v)), hex(code))
        assert dec(code) == back, (hex(code), dec(code), back)


def golden_fastdt_codes():
    """(value, code, decoded) rows of tests/golden/fastdt_codes.txt (worked by hand from the
    rules of Sec. IV-C)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fastdt_codes.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v, c, d = line.split()
                rows.append((int(v), int(c, 16), int(d)))
    return rows


def pin_fastdt_codec_golden(lib):
    """The code table of tests/golden/fastdt_codes.txt (Sec. IV-C's rules by hand)."""
    rows = golden_fastdt_codes()
    assert len(rows) >= 20
    for v, code, back in rows:
        assert oracle.fastdt_encode(v, lib=lib) == code, (v, code)
        assert oracle.fastdt_decode(code, lib=lib) == back, (code, back)


def pin_fastdt_codec_properties(lib):
    """Over every 16-bit value: the decoded value never exceeds the original (the dropped low
    bits are zeroed, the kept bits and the leading ones are exact), its error is below the
    weight of the lowest kept bit (2^9, 2^5 or 2^1 for flags 01, 10, 11), non-negative values
    decode to 0, and encoding a decoded value gives its code back."""
    for v in range(-32768, 32768):
        c = oracle.fastdt_encode(v, lib=lib)
        d = oracle.fastdt_decode(c, lib=lib)
        if v >= 0:
            assert c == 0 and d == 0
            continue
        low = {1: 9, 2: 5, 3: 1}[c & 3]
        assert d <= v and v - d < (1 << low), (v, c, d)
        assert oracle.fastdt_encode(d, lib=lib) == c


def pin_fastdt_store(lib):
    """One store: the reference disparity comes back as 0, every value no better than it (under
    the argmax) as 0, and a better value as C(d) - C(d_arb) within the code's error (the
    dropped bits plus half a unit of rounding, in units of ahat / T)."""
    rng = _rng(91)
    C = rng.uniform(-1, 1, (6, 7, 9))
    ahat = rng.uniform(0.5, 1.5, (6, 7))
    C *= ahat[:, :, None]
    out = oracle.fastdt_store(C, ahat, lib=lib)
    T = oracle.FASTDT_T
    for y in range(6):
        for x in range(7):
            ref = C[y, x, 0]
            for d in range(9):
                if C[y, x, d] <= ref:
                    assert out[y, x, d] == 0.0
                else:
                    exact = (C[y, x, d] - ref) / ahat[y, x] * T
                    got = out[y, x, d] / ahat[y, x] * T
                    assert got >= exact - 0.5 - 1e-9 and got - exact < 512 + 0.5, (got, exact)


def pin_fastdt_chain_composition(lib):
    """The FastDT chain on a textured 5x4 guide equals its definition composed from pinned
    parts: each pass pair applied with the dense pass matrices (built from the closed form of
    the recurrences), the all-ones response A_hat_p after the same p pairs (the same matrices
    on a plane of ones), and the FastDT store (pinned by the codec and store pins) after every
    pair but the last, dividing by A_hat_p. One and two iterations; d_arb = 0."""
    rng = _rng(23)
    H, W, nd = 4, 5, 6
    g = rng.integers(0, 256, (H, W), dtype=np.uint8)
    sig_s, sig_r = 3.0, 0.3
    WL, WR, WU, WD = oracle.dt_weights(g, sig_s, sig_r, lib=lib)
    s = 1 - _K(sig_s)

    def pass_pair(X, horiz):
        X = X.copy()
        if horiz:
            for y in range(H):
                X[y] = _pass_matrix(WR[y], s, False) @ (_pass_matrix(WL[y], s, True) @ X[y])
        else:
            for x in range(W):
                X[:, x] = _pass_matrix(WD[:, x], s, False) @ (_pass_matrix(WU[:, x], s, True) @ X[:, x])
        return X

    for iters in (1, 2):
        C = rng.uniform(-1, 1, (H, W, nd))
        ref, ones = C.copy(), np.ones((H, W, 1))
        for pair in range(1, 2 * iters + 1):
            horiz = pair % 2 == 1
            ref, ones = pass_pair(ref, horiz), pass_pair(ones, horiz)
            if pair < 2 * iters:
                ref = oracle.fastdt_store(ref, ones[:, :, 0], d_arb=0, lib=lib)
        out = oracle.dt_aggregate_fastdt(C, g, sig_s, sig_r, iters, d_arb=0, lib=lib)
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-15), (iters, np.abs(out - ref).max())


def pin_fastdt_chain_accuracy(lib):
    """The chain with FastDT storage still recovers a constant disparity on textured noise
    (>= 99% of interior pixels) and agrees with the exact chain on most pixels of a
    slanted-plane pair."""
    p = make_pair(48, 120, 16, seed=31, disp="const", const_disp=7, gain=1.0, offset=0.0, noise=0.0)
    disp, _ = oracle.run_fastdt(p.left, p.right, 16, 4, SIG_S, SIG_R, 3, lib=lib)
    assert (disp[4:-4, 16:-4] == 7).mean() >= 0.99
    q = make_pair(64, 160, 24, seed=32, disp="planes", occlusion_frac=0.05)
    d8, _ = oracle.run_fastdt(q.left, q.right, 24, 4, SIG_S, SIG_R, 3, lib=lib)
    d64, _ = oracle.run(q.left, q.right, 24, 4, SIG_S, SIG_R, 3, lib=lib)
    assert (d8 == d64).mean() >= 0.9


ALL_PINS = [
    pin_window_sums_routes, pin_window_sums_constant,
    pin_zncc_eq2_exact, pin_zncc_identical_windows, pin_zncc_affine_invariance,
    pin_zncc_zero_variance, pin_zncc_at_matches_volume, pin_zncc_plane_subset,
    pin_zncc_shift_recovery,
    pin_dt_weight_forms, pin_dt_impulse_closed_form, pin_dt_constant_closed_form,
    pin_dt_dense_matrix, pin_dt_scaled_vs_literal, pin_dt_bounded_and_plane_independent,
    pin_dt_edge_stop,
    pin_wta_bruteforce_and_ties,
    pin_end_to_end_recovery,
    pin_fastdt_codec_examples, pin_fastdt_codec_golden, pin_fastdt_codec_properties, pin_fastdt_store,
    pin_fastdt_chain_composition, pin_fastdt_chain_accuracy,
]
