"""Serving on the GPU: a mix of requests of uneven size, disparity range, window, DT
parameters and storage, submitted together, gives for every request exactly the map of a
single zncc_run on its own context, and the FP64 oracle's map within the disparity
tolerance; so does a one-pair-per-launch server and a server whose budget forces contexts to
be evicted and re-created. An injected device-allocation failure comes back through
serve_poll as ZNCC_ENOMEM and the server keeps serving. serve_poll_timed's latency breakdown
adds up to the request's total."""

import os

import numpy as np
import pytest

import oracle
from synth import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_00476_gb300 import zncc as Z  # noqa: E402

# (h, w, D, win, sigma_s, sigma_r, iters, storage, seed)
MIX = [(96, 320, 32, 9, 20.0, 0.1, 3, Z.ZNCC_F32, 600), (50, 130, 64, 7, 20.0, 0.1, 3, Z.ZNCC_F32, 601),
       (120, 200, 48, 11, 20.0, 0.1, 3, Z.ZNCC_F32, 602), (37, 61, 13, 5, 20.0, 0.1, 3, Z.ZNCC_F32, 603),
       (64, 97, 24, 9, 10.0, 0.2, 2, Z.ZNCC_F32, 604), (80, 160, 40, 9, 20.0, 0.1, 0, Z.ZNCC_F32, 605),
       (96, 320, 32, 9, 20.0, 0.1, 3, Z.ZNCC_F16, 606), (96, 320, 32, 9, 20.0, 0.1, 3, Z.ZNCC_F32, 607),
       (200, 384, 64, 9, 20.0, 0.1, 3, Z.ZNCC_F32, 608), (50, 130, 64, 7, 20.0, 0.1, 3, Z.ZNCC_F32, 609)]


def _pairs():
    return [make_pair(h, w, d, seed=seed, disp="planes", occlusion_frac=0.05)
            for (h, w, d, win, ss, sr, it, st, seed) in MIX]


def _alone(pairs):
    """Each request run by itself through zncc_run on a fresh context."""
    out = []
    for (h, w, d, win, ss, sr, it, st, seed), p in zip(MIX, pairs):
        ctx = Z.ZnccContext(w, h, d, win)
        disp = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctx.zncc_run(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda(), disp, ss, sr, it, st)
        torch.cuda.synchronize()
        out.append(disp.cpu().numpy().view(np.uint16).copy())
        ctx.close()
    return out


def _served(pairs, budget, max_slots):
    res = []
    with Z.ZnccServer(budget, max_slots) as srv:
        tickets = [srv.submit(p.left, p.right, d, win, ss, sr, it, st)
                   for (h, w, d, win, ss, sr, it, st, seed), p in zip(MIX, pairs)]
        for (h, w, *_), t in zip(MIX, tickets):
            disp = np.full((h, w), 0xFFFF, np.uint16)
            st = srv.poll(t, disp, 20_000_000)
            assert st == Z.ZNCC_OK, (Z.STATUS_NAMES[st], srv.last_error())
            res.append(disp)
    return res


@pytest.mark.parametrize("budget,max_slots", [(4 << 30, 32), (4 << 30, 1), (24 << 20, 32)])
def test_served_maps_equal_maps_computed_alone(budget, max_slots):
    pairs = _pairs()
    alone = _alone(pairs)
    served = _served(pairs, budget, max_slots)
    for i, (a, b) in enumerate(zip(alone, served)):
        assert np.array_equal(a, b), f"request {i} {MIX[i]} differs in the mix"


def test_served_maps_match_the_oracle():
    """Served maps against the FP64 oracle: F32 requests exact away from near-ties (best -
    second gap below 1e-5, times A_hat after aggregation); the half-storage request differs on
    fewer than 1% of its pixels."""
    pairs = _pairs()
    served = _served(pairs, 4 << 30, 32)
    for (h, w, d, win, ss, sr, it, st, seed), p, got in zip(MIX, pairs, served):
        ref, gap = oracle.run(p.left, p.right, d, win // 2, ss, sr, it)
        scale = oracle.ones_response(p.left, ss, sr, it) if it else 1.0
        bad = (got != ref) & (gap >= 1e-5 * scale)
        if st == Z.ZNCC_F32:
            assert not bad.any(), (h, w, d, win, it, int(bad.sum()))
        else:
            assert (got != ref).mean() < 0.01, (h, w, d, win, it, float((got != ref).mean()))


def test_poll_timed_breakdown_adds_up():
    """The server's latency breakdown of each request: every part is measured, the device work
    is positive, and the parts add up to the total (the stream wait is the remainder, so it may
    read a few microseconds below zero where host and device clocks differ)."""
    pairs = _pairs()
    with Z.ZnccServer(4 << 30, 32) as srv:
        tickets = [srv.submit(p.left, p.right, d, win, ss, sr, it, st)
                   for (h, w, d, win, ss, sr, it, st, seed), p in zip(MIX, pairs)]
        for (h, w, *_), t in zip(MIX, tickets):
            disp = np.zeros((h, w), np.uint16)
            st, tm = srv.poll_timed(t, disp, 20_000_000)
            assert st == Z.ZNCC_OK and tm is not None and tm["valid"] == 1, (st, tm)
            assert tm["h2d_ms"] > 0 and tm["run_ms"] > 0 and tm["d2h_ms"] > 0, tm
            assert tm["queue_ms"] >= 0 and tm["device_wait_ms"] > -0.05, tm
            parts = tm["queue_ms"] + tm["device_wait_ms"] + tm["h2d_ms"] + tm["run_ms"] + tm["d2h_ms"]
            assert abs(parts - tm["total_ms"]) < 1e-6, tm
            assert 1 <= tm["batch_pairs"] <= len(MIX), tm


def test_injected_allocation_failure_is_reported_and_recovered():
    p = make_pair(40, 90, 16, seed=700)
    disp = np.zeros((40, 90), np.uint16)
    with Z.ZnccServer(1 << 30, 8) as srv:
        os.environ["ZNCC_FAIL_DEVICE_ALLOC"] = "1"
        try:
            t = srv.submit(p.left, p.right, 16, 5, 20.0, 0.1, 2)
            assert srv.poll(t, disp, 20_000_000) == Z.ZNCC_ENOMEM
        finally:
            del os.environ["ZNCC_FAIL_DEVICE_ALLOC"]
        t = srv.submit(p.left, p.right, 16, 5, 20.0, 0.1, 2)
        assert srv.poll(t, disp, 20_000_000) == Z.ZNCC_OK
    ref = _alone_one(p, 16, 5, 2)
    assert np.array_equal(disp, ref)


def _alone_one(p, d, win, iters):
    h, w = p.left.shape
    ctx = Z.ZnccContext(w, h, d, win)
    out = torch.empty((h, w), dtype=torch.int16, device="cuda")
    ctx.zncc_run(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda(), out, 20.0, 0.1, iters)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy().view(np.uint16)


def test_poll_before_completion_keeps_the_ticket():
    p = make_pair(384, 1280, 128, seed=701)
    disp = np.zeros((384, 1280), np.uint16)
    with Z.ZnccServer(2 << 30, 4) as srv:
        t = srv.submit(p.left, p.right, 128, 9, 20.0, 0.1, 3)
        first = srv.poll(t, disp, 0)
        assert first in (Z.ZNCC_ENOTREADY, Z.ZNCC_OK)
        if first == Z.ZNCC_ENOTREADY:
            assert srv.poll(t, disp, 20_000_000) == Z.ZNCC_OK
    assert np.array_equal(disp, _alone_one(p, 128, 9, 3))
