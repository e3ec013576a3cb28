"""qp_species_copy: the host <-> device copy of a species' FP64 state, one
strided copy when the arrays share one allocation, one copy per array
otherwise (GPU only)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import NAMES, DeviceSpecies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.mark.parametrize("dims", [2, 3])
def test_round_trip_of_the_strided_layout(ctx, dims):
    cap, n = 1000, 777
    sp = DeviceSpecies(ctx, Q.QP_ELECTRON, cap, dims, track_chi=False)
    rng = np.random.default_rng(dims)
    src = torch.from_numpy(rng.standard_normal(sp.block.shape)).pin_memory()
    sp.copy_state(src, n, True)
    torch.cuda.synchronize()
    got = sp.block.cpu()
    assert torch.equal(got[:, :n], src[:, :n])
    assert torch.count_nonzero(got[:, n:]) == 0  # slots past count untouched
    back = torch.zeros_like(src).pin_memory()
    sp.copy_state(back, n, False)
    torch.cuda.synchronize()
    assert torch.equal(back[:, :n], src[:, :n])
    assert torch.count_nonzero(back[:, n:]) == 0


def test_separately_allocated_arrays(ctx):
    # allocations of different sizes: the arrays do not share one pitch, so
    # the library copies them one by one
    cap, n = 500, 321
    arrays = {nm: torch.zeros(cap + 1024 * k, dtype=torch.float64, device="cuda:0")
              for k, nm in enumerate(NAMES)}
    n_live = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    d = Q.qp_species_desc()
    d.kind, d.dims, d.capacity = Q.QP_PHOTON, 3, cap
    for nm in NAMES:
        setattr(d, nm, C.c_void_p(arrays[nm].data_ptr()))
    d.n_live = C.c_void_p(n_live.data_ptr())
    h = Q.qp_create_species(ctx, d)
    host = torch.arange(len(NAMES) * 600, dtype=torch.float64).reshape(len(NAMES), 600)
    host = host.pin_memory()
    Q.qp_species_copy(ctx, h, host.data_ptr(), 600 * 8, n, True)
    torch.cuda.synchronize()
    for k, nm in enumerate(NAMES):
        assert torch.equal(arrays[nm][:n].cpu(), host[k, :n])
        assert torch.count_nonzero(arrays[nm][n:]) == 0
    Q.qp_destroy_species(ctx, h)


def test_arguments_are_checked(ctx):
    sp = DeviceSpecies(ctx, Q.QP_ELECTRON, 100, 3, track_chi=False)
    host = torch.zeros(sp.block.shape, dtype=torch.float64).pin_memory()
    L = Q.lib()
    assert L.qp_species_copy(ctx, sp.handle, None, 800, 10, 1, None) == Q.QP_ERR_INVALID_ARG
    assert L.qp_species_copy(ctx, sp.handle, host.data_ptr(), 800, 101, 1,
                             None) == Q.QP_ERR_INVALID_ARG
    assert L.qp_species_copy(ctx, sp.handle, host.data_ptr(), 8 * 9, 10, 1,
                             None) == Q.QP_ERR_INVALID_ARG
    assert L.qp_species_copy(ctx, sp.handle, host.data_ptr(), 804, 10, 1,
                             None) == Q.QP_ERR_INVALID_ARG
    assert L.qp_species_copy(ctx, 4095, host.data_ptr(), 800, 10, 1,
                             None) == Q.QP_ERR_NOT_INITIALIZED
