"""Batched solves (one persistent launch per CG iteration for all problems) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _problems(sizes, omegas, sources, nd, dim=2):
    probs = []
    for n in sizes:
        for om in omegas:
            for s in range(sources):
                npts = tuple([n] * dim)
                c = I.source_centers(n + s, 1, dim)[0]
                f = I.gaussian(npts, c, 2.0 / (n - 1) * 3, om ** 2)
                probs.append((npts, om, f, nd))
    return probs


@pytest.mark.parametrize("dim", [2, 3])
def test_batched_fixed_iterations_match_oracle(dim):
    """Uneven grids and frequencies, DEVD with closed-form bases, FP64: after k iterations every
    problem's iterate equals the oracle's DEVD-CG iterate."""
    sizes = (33, 47, 29) if dim == 2 else (13, 11)
    omegas = (9.0, 14.0) if dim == 2 else (6.0, 8.0)
    probs = _problems(sizes, omegas, 1, 5, dim)
    stream = torch.cuda.Stream()   # batched grids share one stream
    grids, params, fs = [], [], []
    k = 6
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
        prm = whv.make_params(om, method="cg", tol=0.0, maxit=k)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (npts, om, f, nd), u, info in zip(probs, us, infos):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        modes, lam2, _ = SP.select_modes(og, tg, nd)
        ref = K.devd_solve(og, tg, f, SP.basis(og, modes), lam2, "cg", 0.0, k).u
        assert info["iterations"] == k
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-12


def test_batched_fp32_converges_like_single_solves():
    """FP32 stepping, 12 problems (3 sizes x 2 frequencies x 2 sources) to 1e-6; each solution
    matches the FP64 oracle's converged one within the FP32 operator-error bound."""
    probs = _problems((65, 97, 129), (12.0, 18.0), 2, 8)
    stream = torch.cuda.Stream()
    grids, params, fs = [], [], []
    for npts, om, f, nd in probs:
        g = whv.Grid(npts, precision=whv.WHV_FP32_STEP, stream=stream)
        prm = whv.make_params(om, method="cg", tol=1e-6, maxit=2000)
        g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
        grids.append(g); params.append(prm); fs.append(dev(f))
    us, infos = whv.whv_solve_batched(grids, params, fs)
    its = [i["iterations"] for i in infos]
    assert all(i["status"] == "OK" for i in infos), infos
    assert len(set(its)) > 1        # problems stop independently
    for (npts, om, f, nd), u in zip(probs, us):
        og = O.Grid(npts)
        tg = WH.time_grid_for(og, om)
        U = IND.helmholtz_direct(npts, tg.omega_eff, f)
        assert IND.relmax(u.cpu().numpy(), U) < 1e-4


def test_batched_rejects_mixed_grids():
    s = torch.cuda.Stream()
    g1 = whv.Grid((33, 33), precision=whv.WHV_FP32_STEP, stream=s)
    g2 = whv.Grid((33, 33), precision=whv.WHV_FP64, stream=s)
    prm = whv.make_params(8.0, method="cg", tol=1e-6)
    f = dev(np.ones(g1.N))
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g2], [prm, prm], [f, f])
    with pytest.raises(whv.WhvError):
        whv.whv_solve_batched([g1, g1], [prm, prm], [f, f])
