"""Serving calls without a GPU: argument checks, the budget rule, unknown tickets, bounded
destroy, and (on a machine without a CUDA device) a failing device call reported through
serve_poll instead of aborting. CPU only."""

import ctypes

import numpy as np
import pytest

from paper_2212_00476_gb300 import build as zbuild
from paper_2212_00476_gb300 import zncc as Z

SIG_S, SIG_R = 20.0, 0.1


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return Z.lib()


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except ImportError:
        return True


def test_serve_create_checks(lib):
    h = ctypes.c_void_p()
    assert lib.serve_create(0, 4, ctypes.byref(h)) == Z.ZNCC_EINVAL
    assert lib.serve_create(1 << 20, 0, ctypes.byref(h)) == Z.ZNCC_EINVAL
    assert lib.serve_create(1 << 20, 4, None) == Z.ZNCC_EINVAL
    assert lib.serve_destroy(None) == Z.ZNCC_EINVAL


def test_serve_submit_rejects_bad_requests(lib):
    img = np.zeros((32, 48), np.uint8)
    srv = Z.ZnccServer(64 << 20, 4)
    try:
        bad = [dict(max_disp=8, win=4), dict(max_disp=8, win=17), dict(max_disp=0, win=9)]
        for kw in bad:
            with pytest.raises(Z.ZnccError) as e:
                srv.submit(img, img, kw["max_disp"], kw["win"], SIG_S, SIG_R, 1)
            assert e.value.status == Z.ZNCC_EINVAL
        with pytest.raises(Z.ZnccError) as e:
            srv.submit(img, img, 8, 9, -1.0, SIG_R, 1)
        assert e.value.status == Z.ZNCC_EINVAL
        with pytest.raises(Z.ZnccError) as e:
            srv.submit(img, img, 2000, 9, SIG_S, SIG_R, 1)
        assert e.value.status == Z.ZNCC_EUNSUPPORTED
        # 1024 x 1024 x 64 F32 needs 256 MiB of volume alone: more than the whole budget
        big = np.zeros((1024, 1024), np.uint8)
        with pytest.raises(Z.ZnccError) as e:
            srv.submit(big, big, 64, 9, SIG_S, SIG_R, 3)
        assert e.value.status == Z.ZNCC_EINVAL
        assert "budget" in srv.last_error()
        # the same image without DT stores no volume and fits
        assert srv.submit(big, big, 64, 9, SIG_S, SIG_R, 0) > 0
        d = np.zeros((32, 48), np.uint16)
        assert srv.poll(12345, d, 0) == Z.ZNCC_EINVAL                 # unknown ticket
        assert lib.serve_poll(srv._h, 1, None, 0) == Z.ZNCC_EINVAL
        assert lib.serve_poll(srv._h, 1, d.ctypes.data, -1) == Z.ZNCC_EINVAL
        t = ctypes.c_uint64()
        assert lib.serve_submit(srv._h, None, img.ctypes.data, 48, 32, 8, 9, SIG_S, SIG_R, 1, 0,
                                ctypes.byref(t)) == Z.ZNCC_EINVAL
    finally:
        assert srv.close() == Z.ZNCC_OK


@pytest.mark.skipif(not _no_gpu(), reason="checks the no-device failure path")
def test_serve_reports_device_failure_through_poll(lib):
    img = np.full((16, 40), 7, np.uint8)
    d = np.zeros((16, 40), np.uint16)
    with Z.ZnccServer(64 << 20, 4) as srv:
        tickets = [srv.submit(img, img, 8, 5, SIG_S, SIG_R, it) for it in (0, 1, 3)]
        for t in tickets:
            assert srv.poll(t, d, 5_000_000) == Z.ZNCC_ECUDA
        assert "device" in srv.last_error()
        assert srv.poll(tickets[0], d, 0) == Z.ZNCC_EINVAL           # forgotten once polled


def test_serve_destroy_with_queued_requests_is_bounded(lib):
    img = np.full((16, 40), 7, np.uint8)
    srv = Z.ZnccServer(64 << 20, 1)
    for _ in range(5):
        srv.submit(img, img, 8, 5, SIG_S, SIG_R, 1)
    assert srv.close() == Z.ZNCC_OK
