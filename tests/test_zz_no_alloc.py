"""qp_diagnostics_noalloc against qp_diagnostics (GPU only).

The allocation-free entry point serves callers that cannot allocate device
memory: a host application whose pool allocator owns the device memory.  It must give the same species
reductions as the context-based qp_diagnostics, call after call, although
every call shares one static scratch array.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

RTOL = 1e-12
FIELDS = ("weight", "energy", "px", "py", "pz", "chi_mean")


def _same(a, b):
    assert a.n_live == b.n_live and a.n_alive == b.n_alive
    for f in FIELDS:
        x, y = getattr(a, f), getattr(b, f)
        assert x == pytest.approx(y, rel=RTOL, abs=1e-12 * max(1.0, abs(y))), f
    np.testing.assert_allclose(np.array(a.hist), np.array(b.hist), rtol=RTOL, atol=1e-12)


@pytest.fixture(scope="module")
def sim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.beam_collision(n=3000, n_steps=120, buffer=200_000)
    s = Simulation(w)
    s.run(120)
    torch.cuda.synchronize()
    yield s
    s.close()


@pytest.mark.parametrize("name", ["electron", "photon"])
def test_noalloc_matches_context_diagnostics_twice(sim, name):
    sp = sim.species[name]
    assert sp.count() > 0
    ref = sim.diagnostics(name)
    first = Q.qp_diagnostics_noalloc(sp._desc)
    second = Q.qp_diagnostics_noalloc(sp._desc)
    _same(first, ref)
    _same(second, ref)
    assert first.n_emit == 0 and first.status == 0   # context data is not reported


def test_noalloc_alternating_species_share_the_scratch(sim):
    el, ph = sim.species["electron"], sim.species["photon"]
    ref_e, ref_p = sim.diagnostics("electron"), sim.diagnostics("photon")
    for _ in range(2):
        _same(Q.qp_diagnostics_noalloc(ph._desc), ref_p)
        _same(Q.qp_diagnostics_noalloc(el._desc), ref_e)


def test_noalloc_rejects_capacity_above_its_scratch(sim):
    d = Q.qp_species_desc.from_buffer_copy(sim.species["electron"]._desc)
    d.capacity = Q.QP_NOALLOC_MAX_SLOTS + 1
    out = Q.qp_diag()
    assert Q.lib().qp_diagnostics_noalloc(C.byref(d), C.byref(out), None) == Q.QP_ERR_INVALID_ARG


@pytest.mark.parametrize("n_live", [3000, Q.QP_NOALLOC_MAX_SLOTS])
def test_noalloc_at_the_largest_capacity(sim, n_live):
    # a species of exactly QP_NOALLOC_MAX_SLOTS slots uses every partial row
    # of the scratch and the final row right after them
    from paper_1311_1107_gb300.sim import DeviceSpecies
    cap = Q.QP_NOALLOC_MAX_SLOTS
    sp = DeviceSpecies(sim.ctx, Q.QP_ELECTRON, cap, 3, sim.dev)
    g = torch.Generator(device=sim.dev).manual_seed(n_live)
    src = sim.species["electron"].host()
    for nm, t in sp.t.items():
        if n_live <= len(src[nm]):
            t[:n_live].copy_(torch.as_tensor(src[nm][:n_live]))
        else:
            t.copy_(torch.rand(cap, generator=g, device=sim.dev, dtype=torch.float64) * 100.0)
    sp.chi.uniform_(0.0, 2.0, generator=g)
    sp.n_live.fill_(n_live)
    torch.cuda.synchronize()
    ref = Q.qp_diagnostics(sim.ctx, sp.handle, None)
    for _ in range(2):
        _same(Q.qp_diagnostics_noalloc(sp._desc), ref)
    Q.qp_destroy_species(sim.ctx, sp.handle)


def test_noalloc_refuses_a_stream_being_captured(sim):
    # the call synchronises its stream: during a capture it returns
    # QP_ERR_INVALID_ARG before anything is enqueued, and the capture stays
    # valid (it ends with an empty graph)
    sp = sim.species["electron"]
    Q.qp_diagnostics_noalloc(sp._desc)  # the scratch array looked up first
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(Q.QPError) as e:
            Q.qp_diagnostics_noalloc(sp._desc, C.c_void_p(s.cuda_stream))
    assert e.value.status == Q.QP_ERR_INVALID_ARG
    _same(Q.qp_diagnostics_noalloc(sp._desc), sim.diagnostics("electron"))
