"""Batched fused runs (zncc_run_batch): pairs of uneven size, disparity range and window in
one launch per step give exactly the maps of separate zncc_run calls, and the oracle's."""

import numpy as np
import pytest

import oracle
from synth import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2212_00476_gb300 import zncc as Z  # noqa: E402

SIG_S, SIG_R = 20.0, 0.1
SPECS = [(96, 320, 32, 9), (50, 130, 64, 7), (37, 61, 13, 11), (120, 200, 48, 9), (64, 97, 24, 5),
         (20, 1100, 16, 3)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _setup(specs, seed0=900):
    pairs, ctxs, L, R, D = [], [], [], [], []
    for i, (h, w, d, win) in enumerate(specs):
        p = make_pair(h, w, d, seed=seed0 + i)
        pairs.append(p)
        ctxs.append(Z.ZnccContext(w, h, d, win))
        L.append(dev(p.left))
        R.append(dev(p.right))
        D.append(torch.empty((h, w), dtype=torch.int16, device="cuda"))
    return pairs, ctxs, L, R, D


@pytest.mark.parametrize("iters,storage", [(3, Z.ZNCC_F32), (0, Z.ZNCC_F32), (2, Z.ZNCC_F16)])
def test_batch_equals_separate_runs(iters, storage):
    pairs, ctxs, L, R, D = _setup(SPECS)
    single = []
    for c, l, r, d in zip(ctxs, L, R, D):
        c.zncc_run(l, r, d, SIG_S, SIG_R, iters, storage)
        single.append(d.clone())
    for d in D:
        d.fill_(-1)
    Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, iters, storage)
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(single, D)):
        assert torch.equal(a, b), f"pair {i} {SPECS[i]} differs between batched and single runs"


def test_batch_matches_oracle():
    pairs, ctxs, L, R, D = _setup(SPECS[:4], seed0=950)
    Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, 3)
    torch.cuda.synchronize()
    for (h, w, d, win), p, disp in zip(SPECS[:4], pairs, D):
        got = disp.cpu().numpy().view(np.uint16)
        ref, gap = oracle.run(p.left, p.right, d, win // 2, SIG_S, SIG_R, 3)
        A = oracle.ones_response(p.left, SIG_S, SIG_R, 3)
        bad = (got != ref) & ~(gap < 1e-5 * A)
        assert not bad.any(), (h, w, d, win, int(bad.sum()))


def test_batch_rejects_bad_arguments():
    pairs, ctxs, L, R, D = _setup(SPECS[:2])
    with pytest.raises(Z.ZnccError) as e:
        Z.zncc_run_batch([ctxs[0], ctxs[0]], L, R, D, SIG_S, SIG_R, 1)
    assert e.value.status == Z.ZNCC_EINVAL
    many = [Z.ZnccContext(16, 8, 4, 3) for _ in range(33)]
    img = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
    out = [torch.empty((8, 16), dtype=torch.int16, device="cuda") for _ in range(33)]
    with pytest.raises(Z.ZnccError) as e:
        Z.zncc_run_batch(many, [img] * 33, [img] * 33, out, SIG_S, SIG_R, 1)
    assert e.value.status == Z.ZNCC_EINVAL


@pytest.mark.parametrize("storage", [Z.ZNCC_F32, Z.ZNCC_F16, Z.ZNCC_I8])
def test_batch_replayed_from_a_cuda_graph_equals_separate_runs(storage):
    """The batched run captured in a CUDA graph (with F16 and I8 storage the A_hat chain forks
    to a second stream and joins back inside the capture) and replayed gives the maps of
    separate runs."""
    specs = SPECS[:4]
    stream = torch.cuda.Stream()
    pairs, _, L, R, D = _setup(specs, seed0=950)
    ctxs = [Z.ZnccContext(w, h, d, win, stream=stream) for (h, w, d, win) in specs]
    single = []
    with torch.cuda.stream(stream):
        for c, l, r, d in zip(ctxs, L, R, D):
            c.zncc_run(l, r, d, SIG_S, SIG_R, 3, storage)
            single.append(d.clone())
        Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, 3, storage)     # buffers and plans first
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, 3, storage)
    for d in D:
        d.fill_(-1)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(zip(single, D)):
        assert torch.equal(a, b), f"pair {i} {specs[i]} differs between the graph and single runs"


def test_batch_mixing_bulk_and_plain_staging_equals_separate_runs():
    """Two pairs of one shape share the cost kernel's launch; the first one's images are 16-byte
    aligned (bulk-copy staging of its rows), the second's start one byte past alignment (plain
    loads): each gives the map of its own zncc_run, and no fault is recorded."""
    h, w, d, win = 48, 256, 40, 9
    ctxs, L, R, D, single = [], [], [], [], []
    for i, offset in enumerate((0, 1)):
        p = make_pair(h, w, d, seed=970 + i, disp="planes")
        ctxs.append(Z.ZnccContext(w, h, d, win))
        imgs = []
        for img in (p.left, p.right):
            buf = torch.zeros(h * w + 64, dtype=torch.uint8, device="cuda")
            v = buf[offset:offset + h * w].view(h, w)
            v.copy_(dev(img))
            imgs.append(v)
        L.append(imgs[0])
        R.append(imgs[1])
        D.append(torch.empty((h, w), dtype=torch.int16, device="cuda"))
        s = torch.empty((h, w), dtype=torch.int16, device="cuda")
        ctxs[-1].zncc_run(dev(p.left), dev(p.right), s, SIG_S, SIG_R, 3)
        single.append(s)
    Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, 3)
    torch.cuda.synchronize()
    assert ctxs[0].device_faults() == 0
    for a, b in zip(single, D):
        assert torch.equal(a, b)
