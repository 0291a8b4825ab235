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


@pytest.mark.parametrize("case", ["cells_4", "cells_enlarged"])
def test_noalloc_cell_list_vs_oracle(oracle_mod, case):
    """The entry point's own cell-list pipeline (scan, scatter, per-cell order, wrapped cell
    offsets, the 27 neighbour cells) against the oracle's real-space part at the same xi
    and rc.  "cells_4": rc = L / 4.2, so 4^3 cells.  "cells_enlarged": L / rc = 17.5 asks
    for 17^3 > SE_NOALLOC_MAX_CELLS cells, which the entry point enlarges to 16^3.  The
    positions are shifted by whole periods, most of them out of [0, L), and every case is
    called twice in a row.  U, Omega and E equal the oracle's real-space sum; E_tr (whose
    harmonic pressure Faxen term the library splits between real and wave space in
    another way than the oracle) equals the regular product's real-space part."""
    lib = api.load()
    rng = np.random.default_rng(33)
    if case == "cells_4":
        rad = rng.uniform(0.5, 1.0, 600)
        L = inputs.box_side(rad, 0.1)
        xi, rc = 0.6, L / 4.2
    else:
        rad = np.full(3000, 0.5)
        L = inputs.box_side(rad, 0.05)
        xi, rc = 1.5, L / 17.5
    pos = inputs.positions_rsa(rad, L, rng)
    shifted = pos + L * rng.integers(-3, 4, size=pos.shape)
    N = rad.shape[0]
    x = rng.standard_normal((N, 12))
    ref = oracle_mod.mobility(pos, rad, L, x, xi=xi, rc=rc, kc=1.0, parts=1)
    ctx = api.Context()
    ctx.set_params(xi, 32, 12, rc)
    ctx.set_option(api.SE_OPT_PRECISION, 1)
    ctx.set_option(api.SE_OPT_PARTS, 1)
    ctx.set_config(pos, rad, L)
    xd = torch.tensor(x, device="cuda", dtype=torch.float64)
    lib_real = ctx.apply(xd).cpu().numpy()
    pos_d = torch.tensor(shifted, device="cuda", dtype=torch.float64)
    rad_d = torch.tensor(rad, device="cuda", dtype=torch.float64)
    for call in range(2):
        code, y = noalloc(lib, pos_d, rad_d, L, xi, rc, xd)
        assert code == api.SE_OK, (call, code)
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got[:, :11] - ref[:, :11]) / np.linalg.norm(ref[:, :11]) <= 1e-12, call
        assert np.linalg.norm(got[:, 11] - lib_real[:, 11]) / np.linalg.norm(lib_real[:, 11]) <= 1e-12, call
        # the forces-only prefix reads and writes 3 components per sphere
        code, y3 = noalloc(lib, pos_d, rad_d, L, xi, rc, xd[:, :3].contiguous())
        assert code == api.SE_OK
        x3 = np.zeros_like(x)
        x3[:, :3] = x[:, :3]
        ref3 = oracle_mod.mobility(pos, rad, L, x3, xi=xi, rc=rc, kc=1.0, parts=1)[:, :3] if call == 0 else ref3
        assert np.linalg.norm(y3.cpu().numpy() - ref3) / np.linalg.norm(ref3) <= 1e-12, call


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
