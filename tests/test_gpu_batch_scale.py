"""Batched solves at the sizes the batched workload runs: more 64 x 64 tiles than resident CTAs,
so every CTA of the persistent launch takes several work items (the item loop, the switch between
problems inside one CTA and, in FP32, the load of the CTA's next tile while the current one is
stepped).  Checked against single-grid solves on the GPU and against the oracle (its DEVD-CG in
the sine eigenbasis, oracle/modal.py, at these sizes: pinned to the time-domain oracle).  Also:
problems that share one basis (whv_share_basis, contractions that read the basis once for all of
them), the batched wave solve on its own (whv_apply_pi_batched), and whv_solve_many's deflation of
all columns at once."""
import numpy as np
import pytest
import torch

from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K, modal as MD
from paper_2606_31842_b300 import inputs as I
from tests import _independent as IND

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

whv = pytest.importorskip("paper_2606_31842_b300.whv")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def tiles(npts, k, r=1):
    """Work items of one problem in the 2-D batched kernel: 64 x 64 regions with a (k r)-wide halo."""
    tw = 64 - 2 * k * r
    return -(-(npts[0] - 2) // tw) * -(-(npts[1] - 2) // tw)


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


# (nodes per side, omega, source seed): two large grids of each kind plus small ones, uneven
SPEC = [(513, 30.0, 0), (769, 40.0, 1), (513, 50.0, 2), (769, 20.0, 3), (257, 40.0, 4), (97, 12.0, 5), (33, 9.0, 6)]
ND = 8


def forcing(n, om, seed):
    npts = (n, n)
    return I.gaussian(npts, I.source_centers(1000 + seed, 1, 2)[0], 2.0 / (n - 1) * 3, om ** 2)


_modal_cache = {}


def modal_iterate(n, om, f, it):
    """The oracle's DEVD-CG iterate after `it` iterations (tol 0) on the n x n box."""
    key = (n, om)
    if key not in _modal_cache:
        g = O.Grid((n, n))
        _modal_cache[key] = MD.ModalSystem(g, WH.time_grid_for(g, om), ND)
    _, _, u = MD.devd_cg(_modal_cache[key], f, 0.0, it)
    return u


def build(precision, stream, k=None, tol=0.0, maxit=3, refine=False, df=False, share=False):
    grids, params, fs, spec = [], [], [], []
    shared = {}
    for n, om, seed in SPEC:
        npts = (n, n)
        prm = whv.make_params(om, method="cg", tol=tol, maxit=maxit, refine_fp64=refine, residual_df64=df)
        g = whv.Grid(npts, precision=precision, stream=stream)
        if share and (n, om) in shared:
            g.whv_share_basis(shared[(n, om)])
        else:
            g.whv_set_deflation_basis(prm, ND, whv.WHV_BASIS_CLOSED_FORM)
            shared[(n, om)] = g
        f = forcing(n, om, seed)
        grids.append(g); params.append(prm); fs.append(dev(f)); spec.append((n, om, f))
    if k is not None:
        grids[0].whv_set_steps_per_sweep(k)
    return grids, params, fs, spec


@pytest.mark.parametrize("k", [3, 8, 10])
def test_fp32_batch_with_several_items_per_cta(k):
    """FP32, fixed iterations: batched iterates equal single-grid FP32 iterates up to the rounding
    of the start step, and the oracle's within the FP32 operator error; the batch holds several
    times more tiles than the launch has CTAs."""
    assert sum(tiles((n, n), k) for n, _, _ in SPEC) > 2 * sms()
    stream = torch.cuda.Stream()
    it = 3
    grids, params, fs, spec = build(whv.WHV_FP32_STEP, stream, k=k, maxit=it)
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (n, om, f), u, info, prm in zip(spec, us, infos, params):
        assert info["iterations"] == it
        s1 = whv.Grid((n, n), precision=whv.WHV_FP32_STEP)
        s1.whv_set_steps_per_sweep(1)
        s1.whv_set_deflation_basis(prm, ND, whv.WHV_BASIS_CLOSED_FORM)
        u1 = s1.whv_solve(prm, dev(f))[0]
        s1.close()
        assert IND.relmax(u.cpu().numpy(), u1.cpu().numpy()) < 2e-5
        assert IND.relmax(u.cpu().numpy(), modal_iterate(n, om, f.reshape(n - 2, n - 2), it)) < 1e-4
    for g in grids:
        g.close()


@pytest.mark.parametrize("share", [False, True])
def test_fp64_batch_with_several_items_per_cta(share):
    """FP64 (k = 4 default), fixed iterations: every iterate equals the oracle's to 1e-12, with
    per-problem bases or with bases shared by the problems of one (grid, frequency)."""
    assert sum(tiles((n, n), 4) for n, _, _ in SPEC) > 2 * sms()
    stream = torch.cuda.Stream()
    it = 3
    grids, params, fs, spec = build(whv.WHV_FP64, stream, maxit=it, share=share)
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (n, om, f), u, info in zip(spec, us, infos):
        assert info["iterations"] == it
        assert IND.relmax(u.cpu().numpy(), modal_iterate(n, om, f.reshape(n - 2, n - 2), it)) < 1e-12
    for g in grids:
        g.close()


def test_double_float_correction_with_several_items_per_cta():
    """FP32 stepping inside the FP64 residual correction with double-float b and residual wave
    solves (4 sub-steps per sweep, several work items per CTA): every FP64 true residual meets
    tol = 1e-9 and every solution is the oracle's converged DEVD-CG solution within the residual
    times the deflated condition number."""
    assert sum(tiles((n, n), 4) for n, _, _ in SPEC) > 2 * sms()
    stream = torch.cuda.Stream()
    grids, params, fs, spec = build(whv.WHV_FP32_STEP, stream, tol=1e-9, maxit=3000, refine=True, df=True)
    us, infos = whv.whv_solve_batched(grids, params, fs)
    for (n, om, f), u, info in zip(spec, us, infos):
        assert info["status"] == "OK" and info["outer_iterations"] >= 1, info
        assert info["true_rel_residual"] <= 1e-9, info
        key = (n, om)
        if key not in _modal_cache:
            g = O.Grid((n, n))
            _modal_cache[key] = MD.ModalSystem(g, WH.time_grid_for(g, om), ND)
        _, conv, ref = MD.devd_cg(_modal_cache[key], f.reshape(n - 2, n - 2), 1e-13, 20000)
        assert np.all(conv)
        assert IND.relmax(u.cpu().numpy(), ref) < 1e-6
    for g in grids:
        g.close()


def test_shared_basis_batch_equals_copied_basis_batch():
    """Four sources on each of two (grid, frequency) classes: sharing the basis (one contraction
    per class reading it once) gives the same FP32 + FP64-correction solutions and iteration counts
    as per-problem copies of it."""
    out = {}
    for share in (False, True):
        stream = torch.cuda.Stream()
        grids, params, fs = [], [], []
        shared = {}
        for n, om in ((257, 30.0), (513, 40.0)):
            for s in range(4):
                prm = whv.make_params(om, method="cg", tol=1e-8, maxit=3000, refine_fp64=True, residual_df64=True)
                g = whv.Grid((n, n), precision=whv.WHV_FP32_STEP, stream=stream)
                if share and (n, om) in shared:
                    g.whv_share_basis(shared[(n, om)])
                else:
                    g.whv_set_deflation_basis(prm, 16, whv.WHV_BASIS_CLOSED_FORM)
                    shared[(n, om)] = g
                grids.append(g); params.append(prm); fs.append(dev(forcing(n, om, 10 + s)))
        us, infos = whv.whv_solve_batched(grids, params, fs)
        assert all(i["status"] == "OK" for i in infos), infos
        out[share] = ([u.cpu().numpy() for u in us], [(i["iterations"], i["outer_iterations"]) for i in infos])
        for g in grids:
            g.close()
    assert out[False][1] == out[True][1]
    for a, b in zip(out[False][0], out[True][0]):
        assert IND.relmax(a, b) < 1e-9


def test_shared_basis_survives_its_source_grid_and_refuses_mismatches():
    stream = torch.cuda.Stream()
    prm = whv.make_params(20.0, method="cg", tol=1e-10, maxit=2000)
    a = whv.Grid((65, 65), stream=stream)
    a.whv_set_deflation_basis(prm, 6, whv.WHV_BASIS_CLOSED_FORM)
    b = whv.Grid((65, 65), stream=stream)
    b.whv_share_basis(a)
    ref = a.whv_get_basis(want_vectors=True)
    a.close()                                   # the vectors live on with b
    got = b.whv_get_basis(want_vectors=True)
    assert torch.equal(ref["V"], got["V"])
    f = dev(forcing(65, 20.0, 0))
    u, info = b.whv_solve(prm, f)
    og = O.Grid((65, 65))
    U = IND.helmholtz_direct((65, 65), WH.time_grid_for(og, 20.0).omega_eff, forcing(65, 20.0, 0))
    assert info["status"] == "OK" and IND.relmax(u.cpu().numpy(), U) < 1e-8
    c = whv.Grid((65, 67), stream=stream)
    with pytest.raises(whv.WhvError):
        c.whv_share_basis(b)                     # other shape
    d = whv.Grid((65, 65), stream=stream)
    d.whv_set_speed(dev(I.speed_squared("c3", (65, 65), 3)))
    with pytest.raises(whv.WhvError):
        d.whv_share_basis(b)                     # other speed kind
    for g in (b, c, d):
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_pi_batched_matches_single_grids(precision):
    """out_p = Pi_h(v_p; f_p) of all problems in one launch equals the single-grid whv_apply_pi
    (FP64: and the oracle, to 1e-12; FP32: within the FP32 stepping bound)."""
    prec = whv.WHV_FP64 if precision == "fp64" else whv.WHV_FP32_STEP
    stream = torch.cuda.Stream()
    spec = [((129, 97), 12.0), ((257, 257), 30.0), ((65, 80), 20.0), ((33, 33), 9.0)]
    grids, params, vs, fs = [], [], [], []
    for i, (npts, om) in enumerate(spec):
        grids.append(whv.Grid(npts, precision=prec, stream=stream))
        params.append(whv.make_params(om))
        vs.append(dev(I.random_field(I.interior_shape(npts), 50 + i)))
        fs.append(dev(I.gaussian(npts, [0.4, 0.6], 0.1, om ** 2)) if i % 2 == 0 else None)
    outs = whv.whv_apply_pi_batched(grids, params, vs, fs)
    for i, ((npts, om), g, prm) in enumerate(zip(spec, grids, params)):
        single = whv.Grid(npts, precision=prec)
        ref = single.whv_apply_pi(prm, vs[i], fs[i])
        single.close()
        tolr = 1e-12 if prec == whv.WHV_FP64 else 2e-5
        assert IND.relmax(outs[i].cpu().numpy(), ref.cpu().numpy()) < tolr
        if prec == whv.WHV_FP64:
            og = O.Grid(npts)
            tg = WH.time_grid_for(og, om)
            f = None if fs[i] is None else fs[i].cpu().numpy()
            oref = WH.apply_pi(og, tg, vs[i].cpu().numpy(), f)
            assert IND.relmax(outs[i].cpu().numpy(), oref) < 1e-12
    for g in grids:
        g.close()


@pytest.mark.parametrize("method", ["cg", "gmres"])
def test_solve_many_deflates_all_columns_at_once(method):
    """whv_solve_many with DEVD on a dense basis (the projection, the deflated forcings and the
    inflation each read the basis once for all columns) equals column-by-column whv_solve."""
    npts, om, nd = (97, 81), 18.0, 10
    g = whv.Grid(npts)
    prm = whv.make_params(om, method=method, tol=1e-10, maxit=2000, restart=20)
    g.whv_set_deflation_basis(prm, nd, whv.WHV_BASIS_CLOSED_FORM)
    cols = [I.gaussian(npts, I.source_centers(70 + j, 1, 2)[0], 0.08, om ** 2) for j in range(5)]
    F = torch.stack([dev(c) for c in cols])
    U, infos = g.whv_solve_many(prm, F)
    for j in range(5):
        u1, i1 = g.whv_solve(prm, F[j].contiguous())
        assert infos[j]["iterations"] == i1["iterations"]
        assert IND.relmax(U[j].cpu().numpy(), u1.cpu().numpy()) < 1e-11
    g.close()


@pytest.mark.parametrize("k_tma,k_ref", [(8, 6), (4, 2), (12, 10)])
def test_tma_fed_sweeps_equal_staged_sweeps_bitwise(k_tma, k_ref):
    """FP32 f = 0 batched wave solves of the large and small problems: the TMA-fed kernel (k a
    multiple of 4: copies into double-buffered shared stages, 16-byte stores to row-padded state)
    and k_batch_block2d (other k: loads through registers) run the same four-cell operations, so
    their outputs are equal bit for bit; both match the single-grid FP32 wave solve."""
    stream = torch.cuda.Stream()
    grids, params, vs = [], [], []
    for i, (n, om, seed) in enumerate(SPEC):
        grids.append(whv.Grid((n, n), precision=whv.WHV_FP32_STEP, stream=stream))
        params.append(whv.make_params(om))
        vs.append(dev(I.random_field((n - 2, n - 2), 60 + i)))
    assert sum(tiles((n, n), k_tma) for n, _, _ in SPEC) > 2 * sms()
    out = {}
    for k in (k_tma, k_ref):
        grids[0].whv_set_steps_per_sweep(k)
        out[k] = whv.whv_apply_pi_batched(grids, params, vs)
    for (n, om, _), a, b, v, prm in zip(SPEC, out[k_tma], out[k_ref], vs, params):
        assert torch.equal(a, b), (n, om)
        single = whv.Grid((n, n), precision=whv.WHV_FP32_STEP)
        ref = single.whv_apply_pi(prm, v)
        single.close()
        assert IND.relmax(a.cpu().numpy(), ref.cpu().numpy()) < 2e-5
    for g in grids:
        g.close()


def test_forced_fp32_wavefront_equals_staged_sweeps_bitwise():
    """Forced FP32 batched wave solves (the b solve of the FP64 correction): at k = 8 the
    two-column wavefront kernel (eight levels per pass, the forcing of the rows in flight in a
    register ring) and k_batch_block2d at k = 6 run the same FP32 operations, so their outputs are
    equal bit for bit, with and without a forcing and with and without an initial state; both match
    the single-grid FP32 wave solve, and the forced FP64 batched solve matches the oracle."""
    stream = torch.cuda.Stream()
    grids, params, vs, fs = [], [], [], []
    for i, (n, om, seed) in enumerate(SPEC):
        grids.append(whv.Grid((n, n), precision=whv.WHV_FP32_STEP, stream=stream))
        params.append(whv.make_params(om))
        vs.append(dev(I.random_field((n - 2, n - 2), 80 + i)) if i % 3 != 1 else
                  torch.zeros((n - 2) * (n - 2), dtype=torch.float64, device="cuda"))
        fs.append(dev(I.gaussian((n, n), I.source_centers(90 + i, 1, 2)[0], 0.05, om ** 2))
                  if i % 3 != 2 else None)
    assert sum(tiles((n, n), 8) for n, _, _ in SPEC) > 2 * sms()
    out = {}
    for k in (8, 6):
        grids[0].whv_set_steps_per_sweep(k)
        out[k] = whv.whv_apply_pi_batched(grids, params, vs, fs)
    for i, ((n, om, _), a, b) in enumerate(zip(SPEC, out[8], out[6])):
        assert torch.equal(a, b), (n, om)
        single = whv.Grid((n, n), precision=whv.WHV_FP32_STEP)
        ref = single.whv_apply_pi(params[i], vs[i], fs[i])
        single.close()
        assert IND.relmax(a.cpu().numpy(), ref.cpu().numpy()) < 2e-5
    for g in grids:
        g.close()


@pytest.mark.parametrize("rows", [128, 256])
def test_wavefront_item_heights_equal_staged_sweeps_bitwise(rows, monkeypatch):
    """FP32 f = 0 batched wave solves at k = 8 with the wavefront kernel's work items fixed at 128
    or 256 rows (WHV_FRONT_ROWS; by default each launch picks one): both heights run the same
    operations per node, so the outputs equal k_batch_block2d's at k = 6 bit for bit."""
    stream = torch.cuda.Stream()
    grids, params, vs = [], [], []
    for i, (n, om, seed) in enumerate(SPEC):
        grids.append(whv.Grid((n, n), precision=whv.WHV_FP32_STEP, stream=stream))
        params.append(whv.make_params(om))
        vs.append(dev(I.random_field((n - 2, n - 2), 120 + i)))
    out = {}
    monkeypatch.setenv("WHV_FRONT_ROWS", str(rows))
    for k in (8, 6):
        grids[0].whv_set_steps_per_sweep(k)
        out[k] = whv.whv_apply_pi_batched(grids, params, vs)
    for (n, om, _), a, b in zip(SPEC, out[8], out[6]):
        assert torch.equal(a, b), (n, om, rows)
    for g in grids:
        g.close()


def test_fp32_batch_cg_with_tall_wavefront_items(monkeypatch):
    """Fixed-iteration batched FP32 CG at k = 8 with 256-row wavefront items (the per-item partial
    sums of p^T A p are grouped differently, the rest of the table zero-filled): iterates agree with
    the 128-row run to the rounding of those sums and with single-grid FP32 solves."""
    stream = torch.cuda.Stream()
    it = 3
    res = {}
    for rows in (128, 256):
        monkeypatch.setenv("WHV_FRONT_ROWS", str(rows))
        grids, params, fs, spec = build(whv.WHV_FP32_STEP, stream, k=8, maxit=it)
        us, infos = whv.whv_solve_batched(grids, params, fs)
        assert all(i["iterations"] == it for i in infos)
        res[rows] = [u.cpu().numpy() for u in us]
        for g in grids:
            g.close()
    for (n, om, f), a, b, prm in zip(spec, res[128], res[256], params):
        assert IND.relmax(b, a) < 1e-6, (n, om)
        s1 = whv.Grid((n, n), precision=whv.WHV_FP32_STEP)
        s1.whv_set_steps_per_sweep(1)
        s1.whv_set_deflation_basis(prm, ND, whv.WHV_BASIS_CLOSED_FORM)
        u1 = s1.whv_solve(prm, dev(f))[0]
        s1.close()
        assert IND.relmax(b, u1.cpu().numpy()) < 2e-5
