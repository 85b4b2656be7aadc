"""C ABI checks that need no GPU: the library loads, exports every declared
symbol, and host-side validation rejects bad arguments before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    return clamp.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "clamp.h")).read()
    return sorted(set(re.findall(r"\b(clamp_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2406_13651_gb300 import clamp
    names = _declared()
    assert len(names) >= 18
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) <= set(clamp.EXPORTS) | set()


def test_params_struct_layout_matches_header():
    from paper_2406_13651_gb300 import clamp
    assert ctypes.sizeof(clamp.Params) == 64
    assert clamp.Params.tol.offset == 48
    assert clamp.Params.init_mu_steps.offset == 56


def test_supported_lengths(lib):
    assert [lib.clamp_supported_length(n) for n in (4, 8, 16, 24, 32, 64, 96, 128, 192, 256, 512)] == [0, 1, 1, 0, 1, 1, 1, 1, 1, 1, 0]


@pytest.mark.parametrize("field,value", [("nx", 48), ("nz", 4), ("nx", 8), ("looks", 0), ("noise_var", 0.0),
                                         ("prox_var", -1.0), ("rho", 1.0), ("prior_weight", 0.0),
                                         ("max_iters", -1), ("tol", -1.0)])
def test_param_validation(lib, field, value):
    from paper_2406_13651_gb300 import clamp
    p = clamp.make_params(32, 32, 16, 4, 1e-3, 1e-4)
    assert lib.clamp_check_params(ctypes.byref(p)) == 0
    setattr(p, field, value)
    st = lib.clamp_check_params(ctypes.byref(p))
    assert st in (1, 7)
    assert lib.clamp_workspace_size(ctypes.byref(p)) == 0
    assert len(lib.clamp_last_error()) > 0


def test_workspace_size_scales_with_voxel_looks(lib):
    from paper_2406_13651_gb300 import clamp
    p1 = clamp.make_params(128, 128, 64, 16, 1e-3, 1e-4)
    p2 = clamp.make_params(128, 128, 64, 32, 1e-3, 1e-4)
    s1, s2 = lib.clamp_workspace_size(ctypes.byref(p1)), lib.clamp_workspace_size(ctypes.byref(p2))
    n = 128 * 128 * 64
    assert 24 * n * 16 <= s1 < 26 * n * 16
    assert 24 * n * 32 <= s2 < 26 * n * 32


def test_null_pointers_rejected_without_launch(lib):
    from paper_2406_13651_gb300 import clamp
    p = clamp.make_params(32, 32, 16, 4, 1e-3, 1e-4)
    st = lib.clamp_forward_prox(ctypes.byref(p), 1, None, None, None, None, None, None, None, None, 0, None)
    assert st == 1
    st = lib.clamp_forward_prox(ctypes.byref(p), 0, 1, 1, 1, 1, 1, 1, None, None, 0, None)
    assert st == 1
    st = lib.clamp_fft3(48, 32, 16, 1, 1, 1, 0, None)
    assert st == 7


def test_prior_schedule_rule(lib):
    """The prior agent runs beside the forward agents up to 2^25 voxel-looks unless a flag
    forces a schedule; both flags together are rejected."""
    from paper_2406_13651_gb300 import clamp
    small = clamp.make_params(128, 128, 64, 16, 1e-3, 1e-4)          # 2^24 voxel-looks
    edge = clamp.make_params(128, 128, 64, 32, 1e-3, 1e-4)           # 2^25
    large = clamp.make_params(256, 256, 128, 32, 1e-3, 1e-4)         # 2^28
    assert lib.clamp_prior_concurrent(ctypes.byref(small)) == 1
    assert lib.clamp_prior_concurrent(ctypes.byref(edge)) == 1
    assert lib.clamp_prior_concurrent(ctypes.byref(large)) == 0
    large.flags = clamp.FLAG_PRIOR_CONCURRENT
    assert lib.clamp_prior_concurrent(ctypes.byref(large)) == 1
    small.flags = clamp.FLAG_PRIOR_SERIAL
    assert lib.clamp_prior_concurrent(ctypes.byref(small)) == 0
    small.flags = clamp.FLAG_PRIOR_SERIAL | clamp.FLAG_PRIOR_CONCURRENT
    assert lib.clamp_prior_concurrent(ctypes.byref(small)) == -1
    assert lib.clamp_check_params(ctypes.byref(small)) == 1


def test_l21_weight_validation(lib):
    """The l2,1 prior agent rejects a negative or non-finite weight before touching the GPU."""
    h = ctypes.c_void_p()
    for lam in (-1.0, float("nan"), float("inf")):
        assert lib.clamp_denoiser_create_l21(lam, ctypes.byref(h)) == 1
    assert lib.clamp_denoiser_create_l21(1.0, None) == 1


def test_product_build_reports_no_bounds_record(lib):
    """The product library is not the bounds-checking build: clamp_bounds_check returns 0 and
    reports no site without touching the device."""
    site = ctypes.c_uint32(123)
    assert lib.clamp_bounds_check(1, ctypes.byref(site)) == 0
    assert site.value == 0
    assert lib.clamp_bounds_check(0, None) < 0   # NULL site: CLAMP_EINVAL, negated


def test_host_alloc_rejects_bad_arguments(lib):
    out = ctypes.c_void_p(7)
    assert lib.clamp_host_alloc(0, ctypes.byref(out)) == 1   # CLAMP_EINVAL before any mapping
    assert out.value is None
    assert lib.clamp_host_alloc(64, None) == 1
    lib.clamp_host_free(None)
    lib.clamp_host_free(ctypes.c_void_p(4096))                # not from the allocator: ignored


def test_checked_build_exports_every_declared_symbol():
    """The bounds-checking variant (CLAMP_BOUNDS_CHECK) compiles from the same sources into its
    own library and exports the same ABI."""
    from paper_2406_13651_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libclamp_checked.so")
    chk = ctypes.CDLL(path)
    for nm in _declared():
        assert hasattr(chk, nm), nm
