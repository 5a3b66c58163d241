"""romb_compliance_grad_noalloc (the compliance gradient kept in a fixed
static device array) against romb_compliance_grad on the same solved lattice,
on two calls in a row, plus its size limit.  Collected last so that it runs
both alone and after every other GPU test in one process."""
import numpy as np
import pytest

import lattice_inputs as LI

from romb_testutil import small_rom

pytestmark = pytest.mark.gpu
romb = pytest.importorskip("paper_2604_09113_gb300")
torch = pytest.importorskip("torch")


def _solved(ctx, lat, path):
    romb.romb_train_load(ctx.h, path)
    romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64)
    romb.romb_factor(ctx.h)
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=1000)


def test_noalloc_gradient_equals_allocating_call_twice():
    p = 4
    R, path = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    lat = LI.lattice(9, 7, p, 2, seed=43, mu_mode="uniform", mu_range=(0.22, 0.36), rho=5e-4)
    n_ctrl, cells = len(lat.ctrl), lat.ncells
    with romb.Context(0) as ctx:
        _solved(ctx, lat, path)
        ref = romb.romb_compliance_grad(ctx.h, n_ctrl, cells)
        assert np.isfinite(ref[0]) and ref[0] > 0
        for call in range(2):
            free_before = torch.cuda.mem_get_info(0)[0]
            got = romb.romb_compliance_grad_noalloc(ctx.h, n_ctrl, cells)
            free_after = torch.cuda.mem_get_info(0)[0]
            # same kernels and arithmetic on the same inputs: bitwise equal
            assert got[0] == ref[0], call
            for a, b in zip(got[1:], ref[1:]):
                assert np.array_equal(a, b), call
            if call == 1:   # the first call may load the library's static memory
                assert free_after == free_before
        # the allocating call still agrees after the no-allocation calls
        again = romb.romb_compliance_grad(ctx.h, n_ctrl, cells)
        assert again[0] == ref[0] and np.array_equal(again[1], ref[1])


def test_noalloc_gradient_rejects_lattices_beyond_its_scratch():
    # 80 x 80 cells at m = 2: 8 (6400 (277 + 18) + 2 * 161^2 + 64) B = 15.5 MB fits;
    # 90 x 90 cells: 8 (8100 * 295 + 2 * 181^2 + 64) B = 19.6 MB exceeds 16 MiB
    p = 4
    R, path = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    lat = LI.lattice(90, 90, p, 2, seed=44, mu_mode="uniform", mu_range=(0.22, 0.36), rho=5e-4)
    with romb.Context(0) as ctx:
        _solved(ctx, lat, path)
        with pytest.raises(romb.RombError) as e:
            romb.romb_compliance_grad_noalloc(ctx.h, len(lat.ctrl), lat.ncells)
        assert e.value.status == -11
        # the allocating call has no such limit
        c, dx, _, _ = romb.romb_compliance_grad(ctx.h, len(lat.ctrl), lat.ncells)
        assert np.isfinite(c) and np.isfinite(dx).all()


def _grad_device(fn, ctx, n_ctrl, cells, with_dmu):
    """Call a gradient entry point with device (CUDA tensor) outputs."""
    import ctypes
    dev = torch.device("cuda", 0)
    c = ctypes.c_double()
    dx = torch.zeros((n_ctrl, 2), dtype=torch.float64, device=dev)
    dR = torch.zeros(cells, dtype=torch.float64, device=dev)
    dmu = torch.zeros((cells, 4), dtype=torch.float64, device=dev) if with_dmu else None
    st = fn(ctx.h, ctypes.byref(c), ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dR.data_ptr()),
            None if dmu is None else ctypes.c_void_p(dmu.data_ptr()))
    assert st == 0, romb.STATUS.get(st, st)
    torch.cuda.synchronize()
    return c.value, dx.cpu().numpy(), dR.cpu().numpy(), None if dmu is None else dmu.cpu().numpy()


@pytest.mark.parametrize("with_dmu", [True, False])
def test_noalloc_two_families_device_outputs(with_dmu):
    # circle holes and crosses mixed (one node table per family in the scratch),
    # lattice arrays and outputs in device memory (outputs written in place),
    # with and without dc/dmu (dc/dR then comes from the scratch's own dmu)
    p = 4
    _, pc = small_rom(0, p, 0.18, 0.40, 20, 12, 1)
    _, px = small_rom(1, p, 0.07, 0.21, 20, 12, 1, seed=2)
    lat = LI.lattice(8, 6, p, 3, seed=47, mu_mode="uniform", mu_range=(0.22, 0.36), cross_range=(0.09, 0.19),
                     cross_fraction=0.5)
    assert 0 < lat.family.sum() < lat.ncells
    dev = torch.device("cuda", 0)
    darr = {"ctrl": torch.from_numpy(lat.ctrl).to(dev), "mu": torch.from_numpy(lat.mu).to(dev),
            "family": torch.from_numpy(lat.family).to(dev),
            "traction": torch.from_numpy(lat.traction.reshape(8).copy()).to(dev)}
    nodes = (lat.p * lat.nx + 1) * (lat.p * lat.ny + 1)
    n_ctrl, cells = len(lat.ctrl), lat.ncells
    with romb.Context(0) as ctx:
        romb.romb_train_load(ctx.h, pc)
        romb.romb_train_load(ctx.h, px)
        romb.romb_assemble(ctx.h, lat, romb.ROMB_FP64, device_arrays=darr)
        romb.romb_factor(ctx.h)
        u = torch.zeros((1, nodes, 2), dtype=torch.float64, device=dev)
        romb.romb_bddc_solve(ctx.h, nodes, rtol=1e-12, maxit=1000, out=u)
        ref = _grad_device(romb._lib.romb_compliance_grad, ctx, n_ctrl, cells, True)
        for call in range(2):
            got = _grad_device(romb._lib.romb_compliance_grad_noalloc, ctx, n_ctrl, cells, with_dmu)
            assert got[0] == ref[0], call
            assert np.array_equal(got[1], ref[1]), call
            assert np.array_equal(got[2], ref[2]), call
            if with_dmu:
                assert np.array_equal(got[3], ref[3]), call
    assert np.isfinite(ref[1]).all() and np.abs(ref[2]).max() > 0
