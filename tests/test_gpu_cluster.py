"""DT line pairs whose lines span the CTAs of a thread-block cluster (lines longer than one
block holds at the chosen lanes per chunk: F32 rows or columns beyond ~2048 pixels, F16 ones
beyond 1024, or 128-byte segments forced by the tuning knobs), against the oracle."""

import numpy as np
import pytest

import oracle
from synth import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_00476_gb300 import zncc as Z  # noqa: E402

SIG_S, SIG_R = 20.0, 0.1
AGG_TOL = 1e-4
GAP_TOL = 1e-5


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _dt_case(h, w, d, iters, seed):
    rng = np.random.default_rng(seed)
    guide = make_pair(h, w, 4, seed=seed).left
    C = rng.uniform(-1, 1, (h, w, d)).astype(np.float32)
    ref = oracle.dt_aggregate(C.astype(np.float64), oracle.dt_weights(guide, SIG_S, SIG_R), SIG_S, iters)
    A = oracle.ones_response(guide, SIG_S, SIG_R, iters)[:, :, None]
    return guide, C, ref, A


# (h, w, d, iters, tuning): rows of 3000 and 3072 pixels and columns of 3000 (two CTAs at 4
# lanes per chunk, forced), and 1280-pixel rows at 8 lanes per chunk (forced)
F32_CASES = [(6, 3000, 8, 1, {Z.ZNCC_TUNE_H_TQ: 4}), (3000, 6, 8, 1, {Z.ZNCC_TUNE_V_TQ: 4}),
             (5, 3072, 12, 2, {Z.ZNCC_TUNE_H_TQ: 4, Z.ZNCC_TUNE_V_TQ: 4}),
             (24, 1280, 40, 2, {Z.ZNCC_TUNE_H_TQ: 8}), (1280, 20, 24, 1, {Z.ZNCC_TUNE_V_TQ: 8})]


@pytest.mark.parametrize("h,w,d,iters,tuning", F32_CASES)
def test_clustered_dt_matches_oracle(h, w, d, iters, tuning):
    guide, C, ref, A = _dt_case(h, w, d, iters, seed=h * 7 + w)
    ctx = Z.ZnccContext(w, h, d, 3)
    for k, v in tuning.items():
        ctx.set_tuning(k, v)
    t = dev(C)
    ctx.dt_aggregate(dev(guide), t, SIG_S, SIG_R, iters)
    torch.cuda.synchronize()
    rel = (np.abs(t.cpu().numpy().astype(np.float64) - ref) / A).max()
    assert rel <= AGG_TOL, f"max |dC|/A_hat = {rel}"


# half storage: 8 lanes per chunk (64-byte segments, forced) need two CTAs beyond 1024 pixels
# and four at 3072
@pytest.mark.parametrize("h,w,d,iters", [(6, 1100, 16, 1), (4, 3072, 8, 1), (1100, 5, 16, 2)])
def test_clustered_dt_fp16_within_rounding_bound(h, w, d, iters):
    guide, C, ref, A = _dt_case(h, w, d, iters, seed=h + 3 * w)
    C16 = C.astype(np.float16)
    ref = oracle.dt_aggregate(C16.astype(np.float64), oracle.dt_weights(guide, SIG_S, SIG_R), SIG_S, iters)
    ctx = Z.ZnccContext(w, h, d, 3)
    ctx.set_tuning(Z.ZNCC_TUNE_H_TQ, 8)
    ctx.set_tuning(Z.ZNCC_TUNE_V_TQ, 8)
    t = dev(C16)
    ctx.dt_aggregate(dev(guide), t, SIG_S, SIG_R, iters, Z.ZNCC_F16)
    torch.cuda.synchronize()
    got = t.float().cpu().numpy().astype(np.float64)
    bound = 2 * iters * (2.0 ** -11 * A + 2.0 ** -24)
    assert (np.abs(got - ref) / bound).max() <= 1.0


@pytest.mark.parametrize("h,w,d,win,storage,tuning", [
    (1100, 64, 24, 9, Z.ZNCC_F32, {Z.ZNCC_TUNE_V_TQ: 8}),     # clustered V pairs, WTA in one
    (48, 1280, 32, 9, Z.ZNCC_F32, {Z.ZNCC_TUNE_H_TQ: 8}),     # clustered H pairs
    (1100, 80, 16, 7, Z.ZNCC_F16, {Z.ZNCC_TUNE_V_TQ: 8}),      # half: clustered V pairs + WTA
])
def test_clustered_fused_run_matches_oracle(h, w, d, win, storage, tuning):
    p = make_pair(h, w, d, seed=h + w + d)
    ctx = Z.ZnccContext(w, h, d, win)
    for k, v in tuning.items():
        ctx.set_tuning(k, v)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, 3, storage)
    got = disp.cpu().numpy().view(np.uint16)
    ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, 3)
    if storage == Z.ZNCC_F32:
        A = oracle.ones_response(p.left, SIG_S, SIG_R, 3)
        bad = (got != ref) & ~(gap < GAP_TOL * A)
        assert not bad.any(), int(bad.sum())
    else:
        assert (got != ref).mean() < 0.01
