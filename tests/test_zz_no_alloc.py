"""The allocation-free projection entry point against the grid-based one.

whv_project_noalloc serves callers that may not allocate device memory (memory owned by a
host framework's pool, real-time loops that forbid allocation after start-up, work inside a
stream capture or a latency budget where cudaMalloc is not allowed).  Its scratch is a static
device array, so this file checks that two calls in a row -- the second one seeing the first
one's leftovers in that array -- both match whv_project on a grid, and that a size beyond the
static limit is refused.  The file is collected last (test_zz_ prefix).
"""
import numpy as np
import pytest
import torch

from paper_2606_31842_b300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


@pytest.mark.parametrize("npts,nd,speed", [((513, 513), 64, None), ((70, 45), 33, "c3"), ((21, 19, 17), 7, "c5")])
def test_noalloc_projection_matches_grid_projection_twice(npts, nd, speed):
    g = whv.Grid(npts)
    n = g.N
    c2 = None
    if speed is not None:
        c2 = I.speed_squared(speed, npts, 3)
        g.whv_set_speed(dev(c2))
    rng = np.random.default_rng(31)
    W = torch.from_numpy(rng.standard_normal((nd, n))).cuda()   # (nd, n) row-major = n x nd column-major
    g.whv_set_deflation_basis(whv.make_params(2.0), nd, whv.WHV_BASIS_USER, V=W,
                              lambda2=np.linspace(1.0, 2.0, nd))
    w = None if c2 is None else dev(1.0 / c2)
    for call, seed in enumerate([41, 42]):          # two calls in a row share the static scratch
        r = dev(I.random_field(g.shape, seed))
        ref = torch.zeros(nd, dtype=torch.float64, device="cuda")
        g.whv_project(r, ref)
        got = torch.full((nd,), float("nan"), dtype=torch.float64, device="cuda")
        whv.whv_project_noalloc(W, r, got, w)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, (call, err)
    g.close()


def test_noalloc_rejects_sizes_beyond_static_scratch():
    n, nd = 2048 * 300, 1024                         # ceil(n/2048) * nd = 307200 > 262144
    W = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    coef = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = whv.lib.whv_project_noalloc(n, nd, W.data_ptr(), r.data_ptr(), None, coef.data_ptr(), None)
    assert st == whv.WHV_ERR_INVALID
    assert b"static scratch" in whv.lib.whv_last_error(None)
