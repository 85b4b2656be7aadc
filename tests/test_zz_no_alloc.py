"""The allocation-free MACE step (clamp_mace_step_noalloc).

It serves callers that cannot allocate device memory: it takes its reduction
scratch from a static device array inside the library instead of a caller
workspace.  This checks, through the C ABI, that it returns what the
allocating clamp_mace_step returns on the same inputs, on two calls in a row
(the second with a different volume, so stale scratch from the first call
would show).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    return clamp.load()


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("order", ["first", "second"])
def test_noalloc_mace_step_matches_allocating_step(lib, order):
    from paper_2406_13651_gb300 import clamp
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # the last shape gives the most reduction blocks the step ever uses (1216), filling the array's cap
    shapes = [(16, 32, 64, 5), (32, 64, 128, 3), (64, 128, 128, 2)]
    if order == "second":
        shapes = shapes[::-1]
    for call, (nz, ny, nx, L) in enumerate(shapes):
        rng = np.random.default_rng(100 + call)
        r = torch.from_numpy(rng.uniform(0.01, 1, (L + 1, nz, ny, nx)).astype(np.float32)).to(dev)
        w0 = torch.from_numpy(rng.uniform(0.01, 1, (L + 1, nz, ny, nx)).astype(np.float32)).to(dev)
        p = clamp.make_params(nx, ny, nz, L, 1e-3, 1e-4)
        ws = clamp.workspace(p)
        w_ref, w_new = w0.clone(), w0.clone()
        wbar_ref = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
        wbar_new = torch.empty_like(wbar_ref)
        ce_ref = torch.zeros(1, dtype=torch.float64, device=dev)
        ce_new = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        st = lib.clamp_mace_step(ctypes.byref(p), r.data_ptr(), w_ref.data_ptr(), wbar_ref.data_ptr(),
                                 ce_ref.data_ptr(), ws.data_ptr(), ws.numel(), stream)
        assert st == 0, lib.clamp_last_error()
        st = lib.clamp_mace_step_noalloc(ctypes.byref(p), r.data_ptr(), w_new.data_ptr(), wbar_new.data_ptr(),
                                         ce_new.data_ptr(), stream)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        assert _rel(w_new.cpu(), w_ref.cpu()) < 1e-6
        assert _rel(wbar_new.cpu(), wbar_ref.cpu()) < 1e-6
        assert ce_new.item() == pytest.approx(ce_ref.item(), rel=1e-6)


def test_noalloc_mace_step_allocates_nothing(lib):
    """After a first call on the device, further calls leave the device's free memory as it was."""
    from paper_2406_13651_gb300 import clamp
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nz, ny, nx, L = 64, 128, 128, 2
    rng = np.random.default_rng(7)
    r = torch.from_numpy(rng.uniform(0.01, 1, (L + 1, nz, ny, nx)).astype(np.float32)).to(dev)
    w = torch.from_numpy(rng.uniform(0.01, 1, (L + 1, nz, ny, nx)).astype(np.float32)).to(dev)
    wbar = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    ce = torch.zeros(1, dtype=torch.float64, device=dev)
    p = clamp.make_params(nx, ny, nz, L, 1e-3, 1e-4)
    assert lib.clamp_mace_step_noalloc(ctypes.byref(p), r.data_ptr(), w.data_ptr(), wbar.data_ptr(),
                                       ce.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.clamp_mace_step_noalloc(ctypes.byref(p), r.data_ptr(), w.data_ptr(), wbar.data_ptr(),
                                           ce.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
