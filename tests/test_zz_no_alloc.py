"""rbf_soft_cost_noalloc, the soft cost for callers that cannot allocate
device memory while they run (deadline-bound scan-matching loops, processes
that reserve their GPU memory at start-up): its results must equal those of
rbf_soft_cost, through the C ABI, on consecutive calls that share its fixed
scratch array (a large call followed by a small one).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ptr(x):
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def test_noalloc_soft_cost_matches_regular_entry_point():
    from paper_2509_26222_gb300 import native as N, workloads as W
    lib = N.load(build_if_missing=True)
    P = ctypes.c_void_p
    lib.rbf_soft_cost_noalloc.argtypes = [P, P, P, P, ctypes.c_int64, P, P, P, P]
    lib.rbf_soft_cost_noalloc.restype = ctypes.c_int
    torch.cuda.set_device(0)
    cfg = W.config3(n=30_000)
    T = N.Terrain(rho=0.6, huber_delta=cfg["delta"])
    T.set_centers(torch.tensor(cfg["centers"], device="cuda"))
    T.set_weights(torch.tensor(cfg["w"], device="cuda"))
    pts_all = torch.tensor(cfg["body"].astype(np.float32), device="cuda")
    R = np.ascontiguousarray(cfg["R"], dtype=np.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a large call, then a much smaller one (a few blocks): the reduction of the
    # second must read only its own blocks, not slots the first one left
    for call, (dt, n) in enumerate(((0.0, pts_all.shape[0]), (0.07, 700))):
        pts = pts_all[:n].contiguous()
        t = np.ascontiguousarray(cfg["t"] + np.array([0.0, dt, -dt]), dtype=np.float64)
        ref = torch.empty(7, dtype=torch.float64, device="cuda")
        ref_r = torch.empty(n, dtype=torch.float32, device="cuda")
        st = lib.rbf_soft_cost(T._h, _ptr(R), _ptr(t), _ptr(pts), n, _ptr(ref),
                               ctypes.c_void_p(ref.data_ptr() + 8), _ptr(ref_r), stream)
        assert st == 0, lib.rbf_last_error()
        out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
        out_r = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.rbf_soft_cost_noalloc(T._h, _ptr(R), _ptr(t), _ptr(pts), n, _ptr(out),
                                       ctypes.c_void_p(out.data_ptr() + 8), _ptr(out_r), stream)
        assert st == 0, lib.rbf_last_error()
        torch.cuda.synchronize()
        ref, out = ref.cpu().numpy(), out.cpu().numpy()
        assert abs(out[0] - ref[0]) <= 1e-4 * abs(ref[0]), (call, out[0], ref[0])
        assert np.max(np.abs(out[1:] - ref[1:])) <= 1e-3 * np.max(np.abs(ref[1:])), call
        assert torch.allclose(out_r, ref_r, rtol=0, atol=1e-6), call
