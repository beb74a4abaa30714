"""GPU parity of the plane-resident fused path (F32 storage): each disparity plane stays in
shared memory for the ZNCC cost, every DT pass pair and the WTA, split over the CTAs of a
thread-block cluster by rows.

  disparity map     the FP64 oracle's, except where the oracle's best-vs-second gap is below
                    GAP_TOL * A_hat (as in test_gpu_parity.py)
  against streaming the streaming path's map (cost volume in device memory) on the same
                    input: identical except at such near-ties
  batch             a batch mixing plane-resident and streaming pairs equals the single runs

Cases span every cluster size (1, 2, 4, 8) and all three size classes of the kernel (row
segments per lane up to 11, 21 and 33 positions, bands up to 16, 24 and 32 rows), bands whose
last one is partial or empty, rows of more than one column group (W > 384 threads), the widest
rows (W = 1024) with the largest window, a single row, D = 1 and D not a multiple of 4.
"""

import numpy as np
import pytest

import oracle
from synth import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_00476_gb300 import zncc as Z  # noqa: E402

SIG_S, SIG_R = 20.0, 0.1
GAP_TOL = 1e-5

# (h, w, D, window, iterations, cluster size)
CASES = [(20, 64, 16, 5, 1, 1), (30, 100, 24, 7, 2, 1), (60, 133, 20, 9, 3, 2),
         (96, 320, 32, 9, 3, 4), (130, 200, 13, 3, 2, 8), (9, 50, 8, 3, 2, 8),
         (1, 150, 16, 3, 2, 1), (100, 1024, 16, 15, 1, 8), (64, 700, 40, 11, 2, 4),
         (5, 40, 1, 3, 1, 2), (96, 320, 48, 9, 3, 8)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_u16(t):
    return t.cpu().numpy().view(np.uint16)


def run(p, d, win, iters, plane, cs=0):
    """The fused F32 run with the plane-resident path on or off (off by default); also whether
    it ran."""
    h, w = p.left.shape
    ctx = Z.ZnccContext(w, h, d, win)
    ctx.set_tuning(Z.ZNCC_TUNE_PLANE, 1 if plane else 0)
    ctx.set_tuning(Z.ZNCC_TUNE_PLANE_CS, cs)
    ctx.profile_enable(True)
    disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, iters, Z.ZNCC_F32)
    torch.cuda.synchronize()
    ran = ctx.profile_read().get("zncc_plane", (0.0, 0))[1] > 0
    out = host_u16(disp)
    ctx.close()
    return out, ran


@pytest.mark.parametrize("h,w,d,win,iters,cs", CASES)
def test_plane_path_matches_oracle(h, w, d, win, iters, cs):
    p = make_pair(h, w, max(d, 2), seed=900 + h + w + d + iters)
    got, ran = run(p, d, win, iters, True, cs)
    assert ran, "the plane-resident path did not run"
    ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, iters)
    A = oracle.ones_response(p.left, SIG_S, SIG_R, iters)
    bad = (got != ref) & ~(gap < GAP_TOL * A)
    assert not bad.any(), f"{int(bad.sum())} disparities differ away from near-ties " \
                          f"(first at {np.argwhere(bad)[:5].tolist()})"


@pytest.mark.parametrize("h,w,d,win,iters", [(96, 320, 32, 9, 3), (192, 640, 64, 9, 3)])
def test_plane_path_agrees_with_streaming_path(h, w, d, win, iters):
    p = make_pair(h, w, d, seed=31 + w)
    plane, ran = run(p, d, win, iters, True)
    stream, ran_s = run(p, d, win, iters, False)
    assert ran and not ran_s
    diff = plane != stream
    if diff.any():
        _, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, iters)
        A = oracle.ones_response(p.left, SIG_S, SIG_R, iters)
        assert not (diff & ~(gap < GAP_TOL * A)).any()


def test_plane_path_not_taken_where_it_does_not_apply():
    """Rows longer than 1024 pixels, more than 8 x 32 rows, FP16 storage and runs without DT take
    the streaming path even with the plane-resident path enabled; it is off by default."""
    for (h, w, d, win, iters, storage) in [(8, 1100, 8, 3, 1, Z.ZNCC_F32), (16, 64, 8, 3, 1, Z.ZNCC_F16),
                                           (16, 64, 8, 3, 0, Z.ZNCC_F32), (300, 64, 8, 3, 1, Z.ZNCC_F32)]:
        p = make_pair(h, w, d, seed=5)
        ctx = Z.ZnccContext(w, h, d, win)
        ctx.set_tuning(Z.ZNCC_TUNE_PLANE, 1)
        ctx.profile_enable(True)
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(dev(p.left), dev(p.right), disp, SIG_S, SIG_R, iters, storage)
        torch.cuda.synchronize()
        assert ctx.profile_read().get("zncc_plane", (0.0, 0))[1] == 0
        ctx.close()


def test_mixed_batch_equals_single_runs():
    """Pairs of the plane-resident path (two cluster sizes) and a streaming pair in one batch."""
    sizes = [(40, 120, 16, 5), (96, 320, 32, 9), (8, 1100, 8, 3), (100, 200, 24, 7)]
    pairs = [make_pair(h, w, d, seed=700 + i) for i, (h, w, d, _) in enumerate(sizes)]
    ctxs = [Z.ZnccContext(w, h, d, win) for (h, w, d, win) in sizes]
    for c in ctxs:
        c.set_tuning(Z.ZNCC_TUNE_PLANE, 1)
        c.profile_enable(True)
    Ls = [dev(p.left) for p in pairs]
    Rs = [dev(p.right) for p in pairs]
    single = []
    for c, L, R, (h, w, _, _) in zip(ctxs, Ls, Rs, sizes):
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        c.zncc_run(L, R, disp, SIG_S, SIG_R, 2, Z.ZNCC_F32)
        single.append(host_u16(disp))
    disps = [torch.empty((h, w), dtype=torch.int16, device="cuda") for (h, w, _, _) in sizes]
    Z.zncc_run_batch(ctxs, Ls, Rs, disps, SIG_S, SIG_R, 2, Z.ZNCC_F32)
    torch.cuda.synchronize()
    for a, b in zip(single, disps):
        assert np.array_equal(a, host_u16(b))
    plane_launches = [c.profile_read().get("zncc_plane", (0.0, 0))[1] for c in ctxs]
    assert plane_launches[0] > 0 and plane_launches[1] > 0     # the launching contexts record them


def test_plane_cluster_size_rejects_other_values():
    ctx = Z.ZnccContext(32, 8, 8, 3)
    for v in (3, 16):
        with pytest.raises(Z.ZnccError):
            ctx.set_tuning(Z.ZNCC_TUNE_PLANE_CS, v)
    ctx.close()
