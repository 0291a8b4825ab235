"""The allocation-free real-space entry point (se_real_space_apply_noalloc).

It serves callers that cannot allocate device memory (an application whose own
allocator reserves the device up front, or a latency-critical caller that cannot
accept the synchronisation of cudaMalloc / cudaFree).  Through the C ABI, two calls
in a row must reproduce the real-space part of the regular product
(se_mobility_apply with only the real-space term enabled) at the FP64 tolerance
of the other parity tests, and sizes beyond the fixed capacity are rejected.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1506_08481_b300 import api, inputs  # noqa: E402


def noalloc(lib, pos, rad, L, xi, rc, x):
    N, ncomp = x.shape
    y = torch.full_like(x, float("nan"))
    rc_ = lib.se_real_space_apply_noalloc(0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), N,
                                          float(L), float(xi), float(rc), 1.0,
                                          ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(rad.data_ptr()),
                                          ncomp, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    return rc_, y


def test_noalloc_matches_regular_real_space_part():
    lib = api.load()
    rng = np.random.default_rng(21)
    rad = rng.uniform(0.5, 1.2, 300)
    L = inputs.box_side(rad, 0.2)
    pos = inputs.positions_rsa(rad, L, rng)
    xi, rc = 0.7, 0.45 * L
    pos_d = torch.tensor(pos, device="cuda", dtype=torch.float64)
    rad_d = torch.tensor(rad, device="cuda", dtype=torch.float64)

    ctx = api.Context()
    ctx.set_params(xi, 32, 12, rc)
    ctx.set_option(api.SE_OPT_PRECISION, 1)
    ctx.set_option(api.SE_OPT_PARTS, 1)            # real-space term only
    ctx.set_config(pos, rad, L)
    for call in range(2):                          # two calls in a row share the scratch
        for ncomp in (12, 3):
            x = torch.tensor(rng.standard_normal((300, ncomp)), device="cuda", dtype=torch.float64)
            code, y = noalloc(lib, pos_d, rad_d, L, xi, rc, x)
            assert code == api.SE_OK, (call, ncomp, code)
            ref = ctx.apply(x).cpu().numpy()
            got = y.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12, (call, ncomp)


def test_noalloc_rejects_sizes_beyond_capacity():
    lib = api.load()
    N = api.SE_NOALLOC_MAX_N + 1
    pos = torch.zeros(N, 3, device="cuda", dtype=torch.float64)
    rad = torch.ones(N, device="cuda", dtype=torch.float64)
    x = torch.zeros(N, 3, device="cuda", dtype=torch.float64)
    code, _ = noalloc(lib, pos, rad, 100.0, 0.5, 5.0, x)
    assert code == api.SE_ERR_TOO_LARGE
    code, _ = noalloc(lib, pos[:10], rad[:10], 10.0, 0.5, 5.0, x[:10])   # rc >= L/2
    assert code == api.SE_ERR_CUTOFF
