"""ipp_bg_estimate_noalloc, the mesh background call for callers that cannot
allocate device memory (its scratch is an array inside the library), checked
through the C ABI against ipp_bg_estimate on two calls in a row: the second call
must not see anything left over from the first.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _params(mesh):
    from paper_2502_10783_gb300 import _abi
    return _abi.BgParams(mesh, mesh, 3, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5)


def _reference(L, img, mesh):
    """the existing entry point, with a caller workspace"""
    H, W = img.shape
    p = _params(mesh)
    nx, ny = -(-W // mesh), -(-H // mesh)
    bkg = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    rms = torch.empty_like(bkg)
    need = L.ipp_bg_estimate_workspace_size(W, H, p)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rc = L.ipp_bg_estimate(img.data_ptr(), 0, W, H, img.stride(0), None, None, p, bkg.data_ptr(),
                           rms.data_ptr(), None, None, None, ws.data_ptr(), ws.numel(), s)
    assert rc == 0
    return bkg, rms


def _noalloc(L, img, mesh):
    H, W = img.shape
    p = _params(mesh)
    nx, ny = -(-W // mesh), -(-H // mesh)
    bkg = torch.full((ny, nx), -7.0, dtype=torch.float32, device="cuda")
    rms = torch.full_like(bkg, -7.0)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rc = L.ipp_bg_estimate_noalloc(img.data_ptr(), 0, W, H, img.stride(0), None, None, p, bkg.data_ptr(),
                                   rms.data_ptr(), status.data_ptr(), s)
    assert rc == 0, L.ipp_last_error_detail()
    return bkg, rms, status


def test_noalloc_matches_workspace_call_twice(gpu):
    L = gpu.load()
    a, _ = synth.frame_gradient_1k(1001)
    b, _ = synth.tiny_frame(517, 389, 77, n_stars=40, sky=500.0)
    for img, mesh in ((a, 64), (b, 32)):   # two calls in a row, different grids
        t = torch.from_numpy(img).cuda()
        rb, rr = _reference(L, t, mesh)
        nb, nr, st = _noalloc(L, t, mesh)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        rb, rr, nb, nr = (x.cpu().numpy() for x in (rb, rr, nb, nr))
        assert np.all(np.abs(nb - rb) <= 1e-5 * np.abs(rb) + 1e-6)
        assert np.all(np.abs(nr - rr) <= 1e-5 * np.abs(rr) + 1e-6)


def test_noalloc_rejects_grid_above_limit(gpu):
    L = gpu.load()
    from paper_2502_10783_gb300 import _abi
    fake = C.c_void_p(0x1000)
    # 8192 x 8192 with 32 px meshes = 65,536 nodes > 16,384
    rc = L.ipp_bg_estimate_noalloc(fake, 0, 8192, 8192, 8192, None, None, _params(32), fake, fake, None, None)
    assert rc == _abi.IPP_ERR_NOT_SUPPORTED
    assert b"no-allocation limit" in L.ipp_last_error_detail()
