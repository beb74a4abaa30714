"""GPU parity: every step of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances:
  window sums S, Q          bit-exact (integer sums of uint8 pixels, exact in int32)
  ZNCC cost                 |gpu - oracle| <= 1e-5 absolute: the numerator n P - S_R S_T and
                            both variances are exact integers, so only the FP32 conversion,
                            1/sqrt and two products round (a few ulps of values in [-1, 1])
  aggregated cost (FP32)    |gpu - oracle| <= 1e-4 * A_hat(x, y), A_hat = DT of an all-ones
                            plane, the largest |aggregated cost| possible at (x, y): each of
                            the 4 * iters passes adds a few FP32 roundings relative to A_hat
  disparity                 exact, except pixels whose oracle best-vs-second gap is below
                            1e-5 (1e-5 * A_hat after aggregation); those are counted, not failed
"""

import numpy as np
import pytest

import oracle
from synth import config_pair, make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_00476_gb300 import zncc as Z  # noqa: E402

SIG_S, SIG_R = 20.0, 0.1
ZNCC_TOL = 1e-5
AGG_TOL = 1e-4
GAP_TOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_u16(t):
    return t.cpu().numpy().view(np.uint16)


def rand_pair(h, w, d, seed, disp="rects"):
    return make_pair(h, w, d, seed=seed, disp=disp)


def gpu_cost(ctx, left, right, dtype=Z.ZNCC_F32):
    H, W = left.shape
    tdt = torch.float32 if dtype == Z.ZNCC_F32 else torch.float16
    c = torch.empty((H, W, ctx.D), dtype=tdt, device="cuda")
    ctx.zncc_cost_volume(dev(left), dev(right), c, dtype)
    torch.cuda.synchronize()
    return c


def check_disp(gpu, ref, gap, scale, what):
    """Exact outside near-ties; returns the number of near-tie pixels skipped."""
    near = gap < GAP_TOL * scale
    bad = (gpu != ref) & ~near
    assert not bad.any(), f"{what}: {int(bad.sum())} disparities differ away from near-ties " \
                          f"(first at {np.argwhere(bad)[:5].tolist()})"
    return int(near.sum())


# ---------------------------------------------------------------------------------------
STATS_CASES = [(96, 320, 4), (17, 37, 1), (5, 3, 7), (1, 1, 2), (64, 1, 3), (1, 70, 5),
               (40, 2100, 6), (33, 129, 7)]


@pytest.mark.parametrize("h,w,r", STATS_CASES)
def test_window_stats_bit_exact(h, w, r):
    rng = np.random.default_rng(h * 1000 + w + r)
    img = rng.integers(0, 256, (h, w), dtype=np.uint8)
    img[: h // 2, : w // 3] = 77                          # flat region: inv_sigma = 0
    ctx = Z.ZnccContext(w, h, 4, 2 * r + 1)
    S = torch.empty((h, w), dtype=torch.int32, device="cuda")
    Q = torch.empty_like(S)
    I = torch.empty((h, w), dtype=torch.float32, device="cuda")
    ctx.zncc_window_stats(dev(img), S, Q, I)
    torch.cuda.synchronize()
    S_ref, Q_ref = oracle.window_sums(img, r)
    assert np.array_equal(S.cpu().numpy(), S_ref)
    assert np.array_equal(Q.cpu().numpy(), Q_ref)
    n = (2 * r + 1) ** 2
    var = n * Q_ref - S_ref * S_ref
    ref_is = np.where(var > 0, 1.0 / np.sqrt(np.maximum(var, 1)), 0.0)
    got = I.cpu().numpy().astype(np.float64)
    assert np.array_equal(got == 0, var == 0)
    assert np.allclose(got, ref_is, rtol=4e-7, atol=0)
    ctx.close()


def test_window_stats_pitched_image():
    rng = np.random.default_rng(5)
    big = rng.integers(0, 256, (20, 64), dtype=np.uint8)
    img_t = dev(big)                                      # pitch 64, width 50
    ctx = Z.ZnccContext(50, 20, 4, 5)
    S = torch.empty((20, 50), dtype=torch.int32, device="cuda")
    assert Z.lib().zncc_window_stats(ctx._h, img_t.data_ptr(), 64, S.data_ptr(), None,
                                     None) == Z.ZNCC_OK
    torch.cuda.synchronize()
    S_ref, _ = oracle.window_sums(big[:, :50], 2)
    assert np.array_equal(S.cpu().numpy(), S_ref)


# ---------------------------------------------------------------------------------------
COST_CASES = [(96, 320, 32, 9), (17, 37, 13, 3), (5, 7, 20, 5), (1, 1, 1, 3), (40, 100, 64, 15),
              (33, 70, 8, 11), (24, 50, 16, 13), (1, 64, 4, 7), (64, 1, 4, 7), (6, 2100, 8, 3),
              (20, 45, 33, 9)]


@pytest.mark.parametrize("h,w,d,win", COST_CASES)
def test_cost_volume_matches_oracle(h, w, d, win):
    p = rand_pair(h, w, max(d, 1), seed=h * 7 + w + d + win)
    ctx = Z.ZnccContext(w, h, d, win)
    c = gpu_cost(ctx, p.left, p.right).cpu().numpy().astype(np.float64)
    ref = oracle.zncc_volume(p.left, p.right, d, win // 2)
    err = np.abs(c - ref).max()
    assert err <= ZNCC_TOL, f"max |dC| = {err}"
    ctx.close()


@pytest.mark.parametrize("h,w,d,win", COST_CASES)
def test_progressive_scan_cost_equals_packed_cost(h, w, d, win):
    """The progressive-scan ablation kernel matches the FP64 oracle within ZNCC_TOL and gives
    the packed-column kernel's values bit for bit (exact integer numerator, same
    normalization)."""
    p = rand_pair(h, w, max(d, 1), seed=h * 7 + w + d + win)
    ctx = Z.ZnccContext(w, h, d, win)
    c = gpu_cost(ctx, p.left, p.right)
    s = torch.empty_like(c)
    ctx.zncc_cost_volume_scan(dev(p.left), dev(p.right), s)
    torch.cuda.synchronize()
    ref = oracle.zncc_volume(p.left, p.right, d, win // 2)
    err = np.abs(s.cpu().numpy().astype(np.float64) - ref).max()
    assert err <= ZNCC_TOL, f"max |dC| = {err}"
    assert torch.equal(c, s)
    s16 = torch.empty((h, w, d), dtype=torch.float16, device="cuda")
    ctx.zncc_cost_volume_scan(dev(p.left), dev(p.right), s16, Z.ZNCC_F16)
    torch.cuda.synchronize()
    assert torch.equal(c.half(), s16)
    ctx.close()


# (h, w, D, window): several 64-pixel tiles with a ragged last one, strips of 8 rows with a
# ragged last one, two and three 128-disparity chunks, D = 1 and 3, every window side
MMA_CASES = COST_CASES + [(19, 200, 300, 9), (9, 130, 129, 15), (12, 64, 3, 3), (17, 70, 1, 5),
                          (21, 150, 96, 11), (8, 65, 40, 13), (10, 100, 60, 7)]


@pytest.mark.parametrize("h,w,d,win", MMA_CASES)
def test_tensor_core_cost_equals_packed_cost(h, w, d, win):
    """The tensor-core ablation (window cross sums as a banded BF16 product, FP32 accumulation)
    matches the FP64 oracle within ZNCC_TOL and gives the packed-column kernel's values bit for
    bit: the products are exact integers."""
    p = rand_pair(h, w, max(d, 1), seed=h * 11 + w + d + win)
    ctx = Z.ZnccContext(w, h, d, win)
    c = gpu_cost(ctx, p.left, p.right)
    s = torch.empty_like(c)
    ctx.zncc_cost_volume_mma(dev(p.left), dev(p.right), s)
    torch.cuda.synchronize()
    ref = oracle.zncc_volume(p.left, p.right, d, win // 2)
    err = np.abs(s.cpu().numpy().astype(np.float64) - ref).max()
    assert err <= ZNCC_TOL, f"max |dC| = {err}"
    assert torch.equal(c, s), f"{int((c != s).sum())} of {c.numel()} values differ"
    s16 = torch.empty((h, w, d), dtype=torch.float16, device="cuda")
    ctx.zncc_cost_volume_mma(dev(p.left), dev(p.right), s16, Z.ZNCC_F16)
    torch.cuda.synchronize()
    assert torch.equal(c.half(), s16)
    ctx.close()


def test_tensor_core_cost_at_full_size_on_sampled_pixels():
    """1280x384, D = 128, 9x9 (the bench pair's shape, random texture): identical to the packed
    kernel everywhere and to the FP64 oracle on sampled pixels within ZNCC_TOL."""
    h, w, d, win = 384, 1280, 128, 9
    p = rand_pair(h, w, d, seed=5)
    ctx = Z.ZnccContext(w, h, d, win)
    c = gpu_cost(ctx, p.left, p.right)
    s = torch.empty_like(c)
    ctx.zncc_cost_volume_mma(dev(p.left), dev(p.right), s)
    torch.cuda.synchronize()
    assert torch.equal(c, s)
    rng = np.random.default_rng(0)
    sc = s.cpu().numpy()
    lib = oracle.load()
    for y, x, dd in zip(rng.integers(0, h, 512), rng.integers(0, w, 512), rng.integers(0, d, 512)):
        ref = oracle.zncc_at(p.left, p.right, win // 2, int(x), int(y), int(dd), lib=lib)
        assert abs(float(sc[y, x, dd]) - ref) <= ZNCC_TOL
    ctx.close()


def test_cost_volume_fp16_storage_is_rounded_fp32():
    p = rand_pair(30, 90, 24, seed=9)
    ctx = Z.ZnccContext(90, 30, 24, 9)
    c32 = gpu_cost(ctx, p.left, p.right, Z.ZNCC_F32)
    c16 = gpu_cost(ctx, p.left, p.right, Z.ZNCC_F16)
    assert torch.equal(c32.half(), c16)


def test_zero_variance_gives_zero_cost():
    left = np.full((12, 40), 100, np.uint8)
    right = np.random.default_rng(3).integers(0, 256, (12, 40), dtype=np.uint8)
    ctx = Z.ZnccContext(40, 12, 8, 5)
    c = gpu_cost(ctx, left, right)
    assert (c == 0).all()


# ---------------------------------------------------------------------------------------
DT_CASES = [(13, 37, 8, 1), (13, 37, 8, 3), (1, 50, 4, 2), (50, 1, 4, 2), (384, 40, 4, 1),
            (20, 1100, 4, 1), (3, 2100, 4, 1), (1030, 3, 4, 1), (16, 30, 5, 3), (7, 9, 70, 2)]


@pytest.mark.parametrize("h,w,d,iters", DT_CASES)
def test_dt_aggregate_matches_oracle(h, w, d, iters):
    rng = np.random.default_rng(h + 31 * w + d)
    guide = make_pair(h, w, 4, seed=h + w).left
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float32)
    ctx = Z.ZnccContext(w, h, d, 3)
    t = dev(C)
    ctx.dt_aggregate(dev(guide), t, SIG_S, SIG_R, iters)
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.float64)
    w4 = oracle.dt_weights(guide, SIG_S, SIG_R)
    ref = oracle.dt_aggregate(C.astype(np.float64), w4, SIG_S, iters)
    A = oracle.ones_response(guide, SIG_S, SIG_R, iters)
    rel = (np.abs(got - ref) / A[:, :, None]).max()
    assert rel <= AGG_TOL, f"max |dC|/A_hat = {rel}"


@pytest.mark.parametrize("iters", [1, 3])
def test_dt_aggregate_fp16_storage_error_is_small(iters):
    """dt_aggregate with half storage rounds the volume after every pass pair: 2*iters
    roundings, each below 2^-11 of |cost| <= A_hat in the normal half range and below the
    subnormal spacing 2^-24 under it; the DT carries an error field e to at most A_hat |e|."""
    h, w, d = 40, 90, 16
    rng = np.random.default_rng(1)
    guide = make_pair(h, w, 4, seed=2).left
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float16)
    ctx = Z.ZnccContext(w, h, d, 3)
    t = dev(C)
    ctx.dt_aggregate(dev(guide), t, SIG_S, SIG_R, iters, Z.ZNCC_F16)
    t32 = dev(C.astype(np.float32))
    ctx.dt_aggregate(dev(guide), t32, SIG_S, SIG_R, iters, Z.ZNCC_F32)
    torch.cuda.synchronize()
    got = t.float().cpu().numpy().astype(np.float64)
    got32 = t32.cpu().numpy().astype(np.float64)
    ref = oracle.dt_aggregate(C.astype(np.float64), oracle.dt_weights(guide, SIG_S, SIG_R),
                              SIG_S, iters)
    A = oracle.ones_response(guide, SIG_S, SIG_R, iters)[:, :, None]
    rel32 = (np.abs(got32 - ref) / A).max()
    err = np.abs(got - ref) / A
    where = np.unravel_index(np.argmax(err), err.shape)
    assert rel32 <= AGG_TOL, rel32
    bound = 2 * iters * (2.0 ** -11 * A + 2.0 ** -24)
    excess = np.abs(got - ref) / bound
    where = np.unravel_index(np.argmax(excess), excess.shape)
    assert excess.max() <= 1.0, (excess.max(), where, got[where], ref[where])


def test_dt_iters_zero_is_identity():
    C = np.random.default_rng(0).uniform(-1, 1, (8, 9, 4)).astype(np.float32)
    ctx = Z.ZnccContext(9, 8, 4, 3)
    t = dev(C)
    ctx.dt_aggregate(dev(np.zeros((8, 9), np.uint8)), t, SIG_S, SIG_R, 0)
    assert np.array_equal(t.cpu().numpy(), C)


# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("h,w,d", [(10, 12, 9), (33, 17, 64), (1, 1, 1), (5, 300, 130)])
def test_wta_disparity_matches_oracle(h, w, d):
    rng = np.random.default_rng(h * w + d)
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float32)
    C[0, 0, :] = 0.25                                   # all tied: smallest d wins
    if d > 3:
        C[-1, -1, [1, d - 1]] = 2.0                     # two-way tie
    ctx = Z.ZnccContext(w, h, d, 3)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.wta_disparity(dev(C), disp)
    ref, _, _ = oracle.wta(C.astype(np.float64))
    assert np.array_equal(host_u16(disp), ref)
    # the same through the half path
    disp16 = torch.empty_like(disp)
    ctx.wta_disparity(dev(C.astype(np.float16)), disp16, Z.ZNCC_F16)
    ref16, _, _ = oracle.wta(C.astype(np.float16).astype(np.float64))
    assert np.array_equal(host_u16(disp16), ref16)


# ---------------------------------------------------------------------------------------
RUN_CASES = [(96, 320, 32, 9, 0), (96, 320, 32, 9, 1), (96, 320, 32, 9, 3), (37, 61, 13, 5, 3),
             (20, 45, 33, 7, 2), (1, 40, 8, 3, 1), (40, 1, 8, 3, 1), (3, 2100, 8, 3, 1),
             (64, 200, 48, 15, 3)]


# (h, w, D): one disparity (every map entry is 0) and a disparity range wider than the image
# (target windows past the left edge read the clamped edge column)
DEGENERATE_D = [(24, 40, 1), (16, 20, 40)]


@pytest.mark.parametrize("h,w,d", DEGENERATE_D)
@pytest.mark.parametrize("storage", [Z.ZNCC_F32, Z.ZNCC_F16])
def test_degenerate_disparity_ranges(h, w, d, storage):
    """The fused run at D = 1 gives the map 0 everywhere, and at D > W (many disparities with
    equal, clamped target windows: ties go to the smallest d) matches the oracle away from
    near-ties: 1e-5 of A_hat for F32, 0.05 of A_hat for F16 (above the half rounding of the
    normalised stored pairs)."""
    p = rand_pair(h, w, d, seed=5, disp="planes")
    ctx = Z.ZnccContext(w, h, d, 5)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, storage)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 0
    got = host_u16(disp)
    if d == 1:
        assert (got == 0).all()
    ref, gap = oracle.run(p.left, p.right, d, 2, SIG_S, SIG_R, 3)
    A = oracle.ones_response(p.left, SIG_S, SIG_R, 3)
    if storage == Z.ZNCC_F32:
        check_disp(got, ref, gap, A, "degenerate D")
    else:
        bad = (got != ref) & ~(gap < 0.05 * A)
        assert not bad.any(), int(bad.sum())
    ctx.close()


@pytest.mark.parametrize("h,w,d,win,iters", RUN_CASES)
def test_fused_run_matches_oracle(h, w, d, win, iters):
    p = rand_pair(h, w, d, seed=h + w + d + win + iters)
    ctx = Z.ZnccContext(w, h, d, win)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, iters, Z.ZNCC_F32)
    got = host_u16(disp)
    ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, iters)
    scale = oracle.ones_response(p.left, SIG_S, SIG_R, iters) if iters else 1.0
    check_disp(got, ref, gap, scale, f"zncc_run {h}x{w} D={d} win={win} iters={iters}")


def test_unfused_chain_equals_oracle_and_fused():
    """cost volume -> dt_aggregate -> wta_disparity gives the oracle's map, like zncc_run."""
    h, w, d, win, iters = 48, 160, 32, 9, 3
    p = rand_pair(h, w, d, seed=77)
    ctx = Z.ZnccContext(w, h, d, win)
    L, R = dev(p.left), dev(p.right)
    c = torch.empty((h, w, d), dtype=torch.float32, device="cuda")
    ctx.zncc_cost_volume(L, R, c)
    ctx.dt_aggregate(L, c, SIG_S, SIG_R, iters)
    d1 = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.wta_disparity(c, d1)
    d2 = torch.empty_like(d1)
    ctx.zncc_run(L, R, d2, SIG_S, SIG_R, iters)
    ref, gap, Cref = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, iters, want_cost=True)
    A = oracle.ones_response(p.left, SIG_S, SIG_R, iters)
    rel = (np.abs(c.cpu().numpy() - Cref) / A[:, :, None]).max()
    assert rel <= AGG_TOL, rel
    check_disp(host_u16(d1), ref, gap, A, "unfused chain")
    check_disp(host_u16(d2), ref, gap, A, "fused run")


def test_run_host_equals_device_run():
    h, w, d = 50, 120, 24
    p = rand_pair(h, w, d, seed=5)
    ctx = Z.ZnccContext(w, h, d, 9)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3)
    host = np.zeros((h, w), np.uint16)
    ctx.zncc_run_host(p.left, p.right, host, SIG_S, SIG_R, 3)
    assert np.array_equal(host, host_u16(disp))
    # a page-locked map buffer takes the last kernel's stores directly (no download copy);
    # pinned image buffers still go up by copies
    for storage in (Z.ZNCC_F32, Z.ZNCC_F16, Z.ZNCC_I8):
        ref = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(dev(p.left), dev(p.right), ref, SIG_S, SIG_R, 3, storage)
        pinned = torch.full((h, w), -1, dtype=torch.int16).pin_memory()
        lp = torch.from_numpy(p.left).pin_memory().numpy()
        rp = torch.from_numpy(p.right).pin_memory().numpy()
        ctx.zncc_run_host(lp, rp, pinned.numpy().view(np.uint16), SIG_S, SIG_R, 3, storage)
        assert torch.equal(pinned, ref.cpu()), storage
    mref, gap = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
    check_disp(host, mref, gap, oracle.ones_response(p.left, SIG_S, SIG_R, 3), "host-buffer run")


def test_fp16_storage_run_mismatch_rate_small():
    h, w, d = 96, 320, 32
    p = rand_pair(h, w, d, seed=12)
    ctx = Z.ZnccContext(w, h, d, 9)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, Z.ZNCC_F16)
    ref, _ = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
    rate = (host_u16(disp) != ref).mean()
    assert rate < 0.01, rate


# (h, w, D): rows whose A_hat pass needs 15 KB of shared memory (automatic: pass by pass) and
# 1400-pixel rows that need 67 KB (automatic: one join)
@pytest.mark.parametrize("h,w,d", [(96, 320, 32), (40, 1400, 24)])
def test_ahat_join_modes_give_the_same_map(h, w, d):
    """ZNCC_TUNE_AHAT_JOIN: with F16 storage the line pairs wait for the A_hat chain on the
    second stream as a whole (1) or pass by pass (2); 0 picks by the passes' shared memory.
    Only the order of the launches differs, so the maps agree bit for bit, also when a
    host-buffer run is captured as a graph and replayed, and stay within the F16 mismatch rate
    of the oracle's."""
    p = rand_pair(h, w, d, seed=h + w + d, disp="planes")
    maps = []
    for join in (0, 1, 2):
        ctx = Z.ZnccContext(w, h, d, 9)
        ctx.set_tuning(Z.ZNCC_TUNE_AHAT_JOIN, join)
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, Z.ZNCC_F16)
        torch.cuda.synchronize()
        maps.append(host_u16(disp).copy())
        for _ in range(2):                          # issued, then replayed
            host = np.zeros((h, w), np.uint16)
            ctx.zncc_run_host(p.left, p.right, host, SIG_S, SIG_R, 3, Z.ZNCC_F16)
            assert np.array_equal(host, maps[-1]), join
        assert ctx.device_faults() == 0
        ctx.close()
    for m in maps[1:]:
        assert np.array_equal(maps[0], m), int((maps[0] != m).sum())
    ref, _ = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
    assert (maps[0] != ref).mean() < 0.01


def test_ahat_join_rejects_other_values():
    ctx = Z.ZnccContext(32, 16, 8, 3)
    for bad in (-1, 3, 7):
        with pytest.raises(Exception):
            ctx.set_tuning(Z.ZNCC_TUNE_AHAT_JOIN, bad)
    ctx.set_tuning(Z.ZNCC_TUNE_AHAT_JOIN, 2)
    ctx.close()


# (h, w): pixel counts that leave 0, 1, 2 and 3 pixels past the last group of four
@pytest.mark.parametrize("h,w", [(16, 48), (5, 7), (9, 26), (11, 27)])
def test_fused_map_into_an_unaligned_buffer(h, w):
    """The WTA finish converts four keys per thread and stores the four disparities at once
    where the map is 8-byte aligned; a map one element into its buffer (2-byte aligned) takes
    the element-wise stores, and the last pixels of a pair whose count is not a multiple of four
    take the element-wise path too. Both maps equal an aligned run's, the elements around the
    map keep their values, and the next run (the keys zeroed by the finish) gives the same map."""
    d = 24
    p = rand_pair(h, w, d, seed=900 + h * w, disp="planes")
    ctx = Z.ZnccContext(w, h, d, 9)
    ref = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), ref, SIG_S, SIG_R, 3, Z.ZNCC_F32)
    buf = torch.full((h * w + 3,), -7, dtype=torch.int16, device="cuda")
    view = buf[1:1 + h * w].view(h, w)
    assert view.data_ptr() % 8 != 0
    for _ in range(2):
        ctx.zncc_run(dev(p.left), dev(p.right), view, SIG_S, SIG_R, 3, Z.ZNCC_F32)
        torch.cuda.synchronize()
        assert torch.equal(view, ref)
    assert int(buf[0]) == -7 and int(buf[-1]) == -7 and int(buf[-2]) == -7
    hbuf = np.full(h * w + 1, 7, np.uint16)             # a host map one element in, likewise
    hview = hbuf[1:].reshape(h, w)
    for _ in range(2):
        ctx.zncc_run_host(p.left, p.right, hview, SIG_S, SIG_R, 3, Z.ZNCC_F32)
        assert np.array_equal(hview, host_u16(ref)) and hbuf[0] == 7
    assert ctx.device_faults() == 0
    mref, gap = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
    check_disp(host_u16(ref), mref, gap, oracle.ones_response(p.left, SIG_S, SIG_R, 3), "finish")
    ctx.close()


def test_run_host_repeated_calls_replay_the_same_work():
    """Repeated zncc_run_host calls with the same page-locked buffers and arguments are captured
    once as a CUDA graph and replayed; the replay reads the buffers' current contents, and a
    change of arguments, tuning or storage (which reallocates the context's volume) issues the
    call afresh. Every map equals a device-buffer run of the same inputs."""
    h, w, d = 48, 160, 32
    ctx = Z.ZnccContext(w, h, d, 9, stream=torch.cuda.Stream())
    lp = torch.empty((h, w), dtype=torch.uint8).pin_memory()
    rp = torch.empty_like(lp).pin_memory()
    mp = torch.empty((h, w), dtype=torch.int16).pin_memory()
    runs = [(1, 20.0, Z.ZNCC_F32, None), (2, 20.0, Z.ZNCC_F32, None), (3, 20.0, Z.ZNCC_F32, None),
            (4, 20.0, Z.ZNCC_F32, None), (4, 12.0, Z.ZNCC_F32, None), (5, 12.0, Z.ZNCC_F32, None),
            (5, 12.0, Z.ZNCC_F32, (Z.ZNCC_TUNE_LINE_LOADS, 1)), (6, 12.0, Z.ZNCC_F32, None),
            (6, 12.0, Z.ZNCC_F16, None), (7, 12.0, Z.ZNCC_F16, None), (8, 12.0, Z.ZNCC_F16, None),
            (9, 12.0, Z.ZNCC_F32, None), (10, 12.0, Z.ZNCC_F32, None)]
    for seed, sig_s, storage, tune in runs:
        if tune:
            ctx.set_tuning(*tune)
        p = rand_pair(h, w, d, seed=300 + seed, disp="planes")
        lp.copy_(torch.from_numpy(p.left))
        rp.copy_(torch.from_numpy(p.right))
        mp.fill_(-1)
        ctx.zncc_run_host(lp.numpy(), rp.numpy(), mp.numpy().view(np.uint16), sig_s, SIG_R, 3, storage)
        ref = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ld, rd = dev(p.left), dev(p.right)
        torch.cuda.synchronize()                    # the inputs, then the context's stream
        ctx.zncc_run(ld, rd, ref, sig_s, SIG_R, 3, storage)
        torch.cuda.synchronize()
        assert torch.equal(mp, ref.cpu()), (seed, storage)
    # buffers replaced between calls (new page-locked tensors, then a pageable map): each call
    # looks its buffers up afresh and never reaches an old one
    for k in range(4):
        lp, rp = torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory()
        out = np.zeros((h, w), np.uint16) if k == 3 else torch.full((h, w), -1, dtype=torch.int16).pin_memory()
        for _ in range(2):
            host = out if k == 3 else out.numpy().view(np.uint16)
            ctx.zncc_run_host(lp.numpy(), rp.numpy(), host, 12.0, SIG_R, 3, Z.ZNCC_F32)
            assert np.array_equal(host, host_u16(ref)), k
    assert ctx.device_faults() == 0
    mref, gap = oracle.run(p.left, p.right, d, 4, 12.0, SIG_R, 3)
    check_disp(host_u16(mp), mref, gap, oracle.ones_response(p.left, 12.0, SIG_R, 3), "replayed run")
    ctx.close()


@pytest.mark.parametrize("storage,loads", [(Z.ZNCC_F32, 0), (Z.ZNCC_F32, 1), (Z.ZNCC_F16, 2)])
def test_wait_drill_records_a_timeout_and_keeps_results(storage, loads):
    """ZNCC_TUNE_WAIT_DRILL makes a bounded device wait run out (an mbarrier nothing completes):
    the kernels record fault bit 2, which zncc_device_faults reports once and clears, the maps
    stay those of a normal run, and without the drill no fault is recorded. Nothing faults,
    traps or hangs."""
    h, w, d = 40, 192, 48
    p = rand_pair(h, w, d, seed=77, disp="planes")
    ld, rd = dev(p.left), dev(p.right)
    ctx = Z.ZnccContext(w, h, d, 9)
    ctx.set_tuning(Z.ZNCC_TUNE_LINE_LOADS, loads)
    ref = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(ld, rd, ref, SIG_S, SIG_R, 3, storage)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 0
    ctx.set_tuning(Z.ZNCC_TUNE_WAIT_DRILL, 1)
    got = torch.empty_like(ref)
    ctx.zncc_run(ld, rd, got, SIG_S, SIG_R, 3, storage)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 4
    assert ctx.device_faults() == 0                 # read and cleared
    assert torch.equal(got, ref)
    ctx.set_tuning(Z.ZNCC_TUNE_WAIT_DRILL, 0)
    ctx.zncc_run(ld, rd, got, SIG_S, SIG_R, 3, storage)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 0
    assert torch.equal(got, ref)
    ctx.close()


def test_invalid_arguments_report_einval():
    ctx = Z.ZnccContext(16, 8, 4, 3)
    img = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
    disp = torch.empty((8, 16), dtype=torch.int16, device="cuda")
    with pytest.raises(Z.ZnccError) as e:
        ctx.zncc_run(img, img, disp, -1.0, SIG_R, 1)
    assert e.value.status == Z.ZNCC_EINVAL
    with pytest.raises(Z.ZnccError):
        ctx.zncc_run(img, img, disp, SIG_S, 0.0, 1)
    with pytest.raises(Z.ZnccError):
        ctx.zncc_run(img, img, disp, SIG_S, SIG_R, -1)
    assert Z.lib().zncc_run(ctx._h, None, img.data_ptr(), 16, 1.0, 1.0, 1, 0,
                            disp.data_ptr()) == Z.ZNCC_EINVAL
    assert Z.lib().zncc_run(ctx._h, img.data_ptr(), img.data_ptr(), 15, 1.0, 1.0, 1, 0,
                            disp.data_ptr()) == Z.ZNCC_EINVAL
    assert Z.lib().zncc_cost_volume(ctx._h, img.data_ptr(), img.data_ptr(), 16,
                                    disp.data_ptr(), 7) == Z.ZNCC_EINVAL


# ---------------------------------------------------------------------------------------
def test_full_size_paper_workload_matches_oracle():
    """1280x384, D = 128, 9x9, sigma_s = 20, sigma_r = 0.1, 3 iterations, FP32: the launch
    configuration the benchmark times, against the full oracle."""
    p = config_pair("paper_1280x384")
    h, w = p.left.shape
    ctx = Z.ZnccContext(w, h, 128, 9)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    L, R = dev(p.left), dev(p.right)
    ctx.zncc_run(L, R, disp, SIG_S, SIG_R, 3, Z.ZNCC_F32)
    ref, gap, Cref = oracle.run(p.left, p.right, 128, 4, SIG_S, SIG_R, 3, want_cost=True)
    A = oracle.ones_response(p.left, SIG_S, SIG_R, 3)
    skipped = check_disp(host_u16(disp), ref, gap, A, "paper workload")
    assert skipped < 0.001 * h * w
    # aggregated cost at every element through the unfused calls
    c = torch.empty((h, w, 128), dtype=torch.float32, device="cuda")
    ctx.zncc_cost_volume(L, R, c)
    ctx.dt_aggregate(L, c, SIG_S, SIG_R, 3)
    rel = (np.abs(c.cpu().numpy() - Cref) / A[:, :, None]).max()
    assert rel <= AGG_TOL, rel
    # and accuracy against the synthetic ground truth (context for the method, not parity)
    v = p.valid
    assert (host_u16(disp)[v] == p.gt[v]).mean() > 0.5


# (h, w, D, window): widths that are multiples of 16 take the bulk-copy staging of the image rows
# (both S offsets of the 4-column groups occur across the windows); 3072-pixel rows; a width
# that is not a multiple of 16 takes the plain loads either way
BULK_CASES = [(96, 320, 32, 9), (40, 1280, 128, 9), (33, 208, 40, 15), (21, 48, 16, 3),
              (17, 2048, 24, 13), (9, 3072, 8, 11), (12, 64, 13, 5), (10, 100, 20, 7)]


@pytest.mark.parametrize("h,w,d,win", BULK_CASES)
@pytest.mark.parametrize("storage", [Z.ZNCC_F32, Z.ZNCC_F16, Z.ZNCC_I8])
def test_bulk_row_staging_equals_plain_loads(h, w, d, win, storage):
    """The cost kernel stages the image rows by bulk asynchronous copies (TMA unit) where the
    rows are 16-byte aligned, else with plain loads; both give the same maps bit for bit, the
    F32 map matches the oracle away from near-ties, and no kernel records a fault."""
    p = rand_pair(h, w, d, seed=h + 3 * w + d + win, disp="planes")
    maps = []
    for loads in (0, 1):
        ctx = Z.ZnccContext(w, h, d, win)
        ctx.set_tuning(Z.ZNCC_TUNE_ROW_LOADS, loads)
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, storage)
        torch.cuda.synchronize()
        assert ctx.device_faults() == 0
        maps.append(host_u16(disp).copy())
        ctx.close()
    assert np.array_equal(maps[0], maps[1]), int((maps[0] != maps[1]).sum())
    if storage == Z.ZNCC_F32:
        ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, 3)
        A = oracle.ones_response(p.left, SIG_S, SIG_R, 3)
        check_disp(maps[0], ref, gap, A, "bulk staging")


# (h, w, D): column groups of 1, 2 and 4 in the vertical store pairs, widths that are not a
# multiple of the group, and the paper's column height
V_LPC_CASES = [(384, 64, 128), (40, 37, 24), (130, 9, 40)]


@pytest.mark.parametrize("h,w,d", V_LPC_CASES)
@pytest.mark.parametrize("lpc", [1, 2, 4])
def test_vertical_column_groups_match_oracle(h, w, d, lpc):
    """ZNCC_TUNE_V_LPC puts up to 1, 2 or 4 adjacent columns in one block of the vertical pairs
    that store the volume: dt_aggregate stays within the aggregation tolerance of the oracle,
    and the fused map matches the oracle's away from near-ties."""
    rng = np.random.default_rng(7 * h + w + d + lpc)
    guide = make_pair(h, w, 4, seed=h + 2 * w).left
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float32)
    ctx = Z.ZnccContext(w, h, d, 9)
    ctx.set_tuning(Z.ZNCC_TUNE_V_LPC, lpc)
    t = dev(C)
    ctx.dt_aggregate(dev(guide), t, SIG_S, SIG_R, 2)
    torch.cuda.synchronize()
    ref = oracle.dt_aggregate(C.astype(np.float64), oracle.dt_weights(guide, SIG_S, SIG_R), SIG_S, 2)
    A = oracle.ones_response(guide, SIG_S, SIG_R, 2)
    rel = (np.abs(t.cpu().numpy().astype(np.float64) - ref) / A[:, :, None]).max()
    assert rel <= AGG_TOL, f"max |dC|/A_hat = {rel}"
    p = rand_pair(h, w, d, seed=50 + h + w + lpc, disp="planes")
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, Z.ZNCC_F32)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 0
    mref, gap = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
    check_disp(host_u16(disp), mref, gap, oracle.ones_response(p.left, SIG_S, SIG_R, 3), "column groups")
    ctx.close()


def test_vertical_column_groups_reject_other_values():
    ctx = Z.ZnccContext(32, 16, 8, 3)
    for bad in (-1, 3, 5, 8):
        with pytest.raises(Exception):
            ctx.set_tuning(Z.ZNCC_TUNE_V_LPC, bad)
    ctx.close()


# (h, w, D, storage): TMA staging of the DT pairs' slices where eligible (F32 rows and columns,
# F16 columns), ragged lines and disparity counts, and a half-precision pixel stride of 20 entries
# (40 bytes, not 16-byte aligned) that takes the cp.async path in both runs
TMA_CASES = [(96, 320, 64, Z.ZNCC_F32, {}), (40, 1280, 128, Z.ZNCC_F32, {}), (33, 208, 40, Z.ZNCC_F32, {}),
             (1030, 24, 12, Z.ZNCC_F32, {}), (50, 120, 24, Z.ZNCC_F16, {}), (64, 96, 20, Z.ZNCC_F16, {}),
             # four chunks per shared-memory wavefront: boxes 19 positions tall, shifted 0-3
             (40, 320, 64, Z.ZNCC_F16, {Z.ZNCC_TUNE_H_TQ: 4, Z.ZNCC_TUNE_V_TQ: 4}),
             (37, 208, 24, Z.ZNCC_F32, {Z.ZNCC_TUNE_H_TQ: 2, Z.ZNCC_TUNE_V_TQ: 2})]


@pytest.mark.parametrize("h,w,d,storage,tunings", TMA_CASES)
def test_tma_staging_equals_cp_async(h, w, d, storage, tunings):
    """ZNCC_TUNE_LINE_LOADS: the DT pairs stream their next slices by one TMA tensor copy per
    chunk in the horizontal pairs (0, automatic), by cp.async per thread everywhere (1), or by
    TMA in both directions (2). The arithmetic is the same, so maps and aggregated volumes agree
    bit for bit; the F32 map matches the oracle away from near-ties, and no copy times out."""
    p = rand_pair(h, w, d, seed=11 * h + w + d, disp="planes")
    rng = np.random.default_rng(h + w + d)
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float32)
    maps, vols = [], []
    for loads in (0, 1, 2):
        ctx = Z.ZnccContext(w, h, d, 9)
        for key, value in tunings.items():
            ctx.set_tuning(key, value)
        ctx.set_tuning(Z.ZNCC_TUNE_LINE_LOADS, loads)
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, storage)
        t = dev(C)
        ctx.dt_aggregate(dev(p.left), t, SIG_S, SIG_R, 2)
        torch.cuda.synchronize()
        assert ctx.device_faults() == 0
        maps.append(host_u16(disp).copy())
        vols.append(t.cpu().numpy())
        ctx.close()
    for m, v in zip(maps[1:], vols[1:]):
        assert np.array_equal(maps[0], m), int((maps[0] != m).sum())
        assert np.array_equal(vols[0], v)
    if storage == Z.ZNCC_F32:
        ref, gap = oracle.run(p.left, p.right, d, 4, SIG_S, SIG_R, 3)
        check_disp(maps[0], ref, gap, oracle.ones_response(p.left, SIG_S, SIG_R, 3), "TMA staging")


def _embedded(img, pad, offset):
    """The image as a row-strided view into a larger device buffer: rows `pad` bytes wider than
    the image, starting `offset` bytes past a 256-byte aligned base."""
    h, w = img.shape
    buf = torch.zeros(h * (w + pad) + offset + 64, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + h * (w + pad)].view(h, w + pad)[:, :w]
    view.copy_(torch.from_numpy(img).cuda())
    return view


@pytest.mark.parametrize("pad,offset", [(48, 0), (16, 32), (0, 1), (5, 0)])
def test_pitched_and_unaligned_images(pad, offset):
    """Images given as row-strided views: a pitch wider than the row that keeps 16-byte alignment
    takes the bulk-copy staging, an odd offset or pitch the plain loads; the maps equal those of
    contiguous images (and the oracle's away from near-ties), with no fault recorded."""
    h, w, d, win = 40, 320, 48, 9
    p = rand_pair(h, w, d, seed=900 + pad + offset, disp="planes")
    ctx = Z.ZnccContext(w, h, d, win)
    ref_map = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), ref_map, SIG_S, SIG_R, 3)
    got = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(_embedded(p.left, pad, offset), _embedded(p.right, pad, offset), got, SIG_S, SIG_R, 3)
    torch.cuda.synchronize()
    assert ctx.device_faults() == 0
    assert torch.equal(ref_map, got)
    ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, 3)
    check_disp(host_u16(got), ref, gap, oracle.ones_response(p.left, SIG_S, SIG_R, 3), "pitched")
    ctx.close()
