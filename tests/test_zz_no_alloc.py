"""dt_aggregate_noalloc: the context-free DT aggregation whose scratch is a static device
array, for callers that cannot allocate while they run. On the GPU it matches the FP64 oracle
within the DT tolerance and gives what dt_aggregate gives, call after call, without changing
the device's free memory; sizes beyond the static scratch and mismatched tensors are rejected
before any CUDA call.

This file is collected last on purpose: its GPU test must pass both alone and after every
other test of the suite has run in the same process."""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2212_00476_gb300 import build as zbuild
from paper_2212_00476_gb300 import zncc as Z
from synth import make_pair

SIG_S, SIG_R, ITERS = 20.0, 0.1, 3
MAX_PIXELS = 2_097_152            # 64 MiB of scratch at 32 bytes per pixel
# Both paths run the same kernels with the same launch shapes, so they agree to the last
# bit; the bound leaves room only for a different shape choice (a different association
# of the chunk carries), far below the 1e-4 * A_hat the DT kernels meet against the oracle.
TOL = 1e-6
AGG_TOL = 1e-4                    # against the FP64 oracle: |gpu - oracle| <= 1e-4 * A_hat(x, y)


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return Z.lib()


def test_noalloc_rejects_sizes_beyond_the_static_scratch(lib):
    # rejected before any CUDA call: the pointers are never used
    fake = ctypes.c_void_p(16)
    for w, h in [(2049, 1024), (3072, 683), (2048, 1025)]:
        st = lib.dt_aggregate_noalloc(fake, w, w, h, 8, fake, Z.ZNCC_F32, SIG_S, SIG_R, ITERS, None)
        assert st == Z.ZNCC_EUNSUPPORTED, (w, h, st)
        msg = lib.zncc_last_error(None).decode()
        assert str(MAX_PIXELS) in msg and "scratch" in msg, msg
    cases = [((None, 10, 10, 10, 4, fake, 0, SIG_S, SIG_R, 1, None), Z.ZNCC_EINVAL),
             ((fake, 9, 10, 10, 4, fake, 0, SIG_S, SIG_R, 1, None), Z.ZNCC_EINVAL),
             ((fake, 10, 10, 10, 4, fake, 2, SIG_S, SIG_R, 1, None), Z.ZNCC_EINVAL),
             ((fake, 10, 10, 10, 4, fake, 0, 0.0, SIG_R, 1, None), Z.ZNCC_EINVAL),
             ((fake, 10, 10, 10, 4, fake, 0, SIG_S, SIG_R, -1, None), Z.ZNCC_EINVAL),
             ((fake, 3073, 3073, 10, 4, fake, 0, SIG_S, SIG_R, 1, None), Z.ZNCC_EUNSUPPORTED),
             ((fake, 10, 10, 10, 1025, fake, 0, SIG_S, SIG_R, 1, None), Z.ZNCC_EUNSUPPORTED),
             ((fake, 10, 10, 10, 4, fake, 0, SIG_S, SIG_R, 0, None), Z.ZNCC_OK)]   # iters 0: no work
    for args, want in cases:
        assert lib.dt_aggregate_noalloc(*args) == want, args


def test_noalloc_wrapper_rejects_mismatched_tensors(lib):
    """The binding checks shapes, dtypes and devices before it passes pointers to the library
    (the call itself has no context that would catch a volume of the wrong size or type)."""
    torch = pytest.importorskip("torch")
    g = torch.zeros((6, 10), dtype=torch.uint8)
    bad = [(g, torch.zeros((6, 10, 4), dtype=torch.float16), Z.ZNCC_F32),    # half volume, F32 flag
           (g, torch.zeros((6, 10, 4), dtype=torch.float32), Z.ZNCC_F16),    # float volume, F16 flag
           (g, torch.zeros((5, 10, 4), dtype=torch.float32), Z.ZNCC_F32),    # fewer rows than the guide
           (g, torch.zeros((6, 10), dtype=torch.float32), Z.ZNCC_F32),       # not [H][W][D]
           (g.float(), torch.zeros((6, 10, 4), dtype=torch.float32), Z.ZNCC_F32),  # guide not uint8
           (g, torch.zeros((6, 10, 4), dtype=torch.float32), Z.ZNCC_F32)]    # host tensors
    for guide, cost, flag in bad:
        with pytest.raises(ValueError):
            Z.dt_aggregate_noalloc(guide, cost, SIG_S, SIG_R, ITERS, flag)


def _volume(torch, ctx, p, seed):
    """The guide on the device and a seeded synthetic cost volume in [-1, 1] (FP32), the same
    input for the oracle and both device paths."""
    left = torch.from_numpy(p.left).cuda()
    C = np.random.default_rng(seed).uniform(-1, 1, (ctx.H, ctx.W, ctx.D)).astype(np.float32)
    return left, torch.from_numpy(C).cuda(), C


def _oracle_error(p, C, out, iters):
    """max |out - oracle| / A_hat over the volume."""
    ref = oracle.dt_aggregate(C.astype(np.float64), oracle.dt_weights(p.left, SIG_S, SIG_R), SIG_S, iters)
    A = oracle.ones_response(p.left, SIG_S, SIG_R, iters)[:, :, None]
    return float((np.abs(out.float().cpu().numpy().astype(np.float64) - ref) / A).max())


@pytest.mark.gpu
def test_noalloc_matches_dt_aggregate_on_two_calls_in_a_row(lib):
    torch = pytest.importorskip("torch")
    H, W, D = 75, 203, 37                      # several chunks and slices, ragged tails
    p = make_pair(H, W, D, seed=4242)
    ctx = Z.ZnccContext(W, H, D, 9)
    left, cost, C = _volume(torch, ctx, p, 4243)
    ref = cost.clone()
    ctx.dt_aggregate(left, ref, SIG_S, SIG_R, ITERS)
    torch.cuda.synchronize()

    outs = [cost.clone(), cost.clone(), cost.clone()]
    Z.dt_aggregate_noalloc(left, outs[0], SIG_S, SIG_R, ITERS)     # set-up call
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    Z.dt_aggregate_noalloc(left, outs[1], SIG_S, SIG_R, ITERS)     # two calls in a row
    Z.dt_aggregate_noalloc(left, outs[2], SIG_S, SIG_R, ITERS)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    for i, out in enumerate(outs):
        err = (out - ref).abs().max().item()
        assert err <= TOL, (i, err)
        rel = _oracle_error(p, C, out, ITERS)
        assert rel <= AGG_TOL, (i, rel)
    assert free_after == free_before, (free_before, free_after)

    # half storage, on a stream of its own
    h_ref = cost.half()
    ctx.dt_aggregate(left, h_ref, SIG_S, SIG_R, ITERS, Z.ZNCC_F16)
    s = torch.cuda.Stream()
    h_out = cost.half()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Z.dt_aggregate_noalloc(left, h_out, SIG_S, SIG_R, ITERS, Z.ZNCC_F16, stream=s)
    s.synchronize()
    assert (h_out.float() - h_ref.float()).abs().max().item() <= TOL


@pytest.mark.gpu
def test_noalloc_at_the_size_limit_then_a_smaller_image(lib):
    torch = pytest.importorskip("torch")
    # the largest image the scratch holds, then a smaller one whose coefficients lie where
    # the larger one's were: nothing of the first call may leak into the second
    for (H, W, D, seed) in [(1024, 2048, 4, 77), (64, 100, 12, 78)]:
        assert W * H <= MAX_PIXELS
        p = make_pair(H, W, D, seed=seed)
        ctx = Z.ZnccContext(W, H, D, 5)
        left, cost, C = _volume(torch, ctx, p, seed + 1)
        ref = cost.clone()
        ctx.dt_aggregate(left, ref, SIG_S, SIG_R, 1)
        out = cost.clone()
        Z.dt_aggregate_noalloc(left, out, SIG_S, SIG_R, 1)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= TOL, ((H, W, D), err)
        assert np.isfinite(out.cpu().numpy()).all()
        rel = _oracle_error(p, C, out, 1)
        assert rel <= AGG_TOL, ((H, W, D), rel)
