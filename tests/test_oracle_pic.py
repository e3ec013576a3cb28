"""Pins of the oracle's PIC coupling (CPU only): the 2D Yee Maxwell solver
against the exact discrete plane wave of the scheme (its numerical
dispersion relation) and the conservation of div B and of the discrete
field energy; the current deposition against its totals and single-node
cases; the sort by cell against its definition (stable, a permutation)."""
import math

import numpy as np
import pytest

import oracle as O


def _zeros(nx, ny):
    return [np.zeros((ny, nx), np.float32) for _ in range(6)]


def test_discrete_plane_wave_is_exact():
    # E_y = sin(k x - w t) at (i, j+1/2, n), B_z the same at (i+1/2, j+1/2,
    # n-1/2) is an exact solution of the Yee scheme when
    # sin(w dt/2)/dt = sin(k dx/2)/dx; far enough from the grid's edges (the
    # scheme's signal moves at most one cell a step) it must stay so
    nx, ny, dx, dy = 128, 48, 0.2, 0.2
    dt = 0.9 * dx / math.sqrt(2)
    k = 2 * math.pi / (16 * dx)
    w = 2 / dt * math.asin(dt / dx * math.sin(k * dx / 2))
    F = _zeros(nx, ny)
    i = np.arange(nx)[None, :]
    F[1][:] = np.sin(k * i * dx).astype(np.float32) + 0 * np.zeros((ny, 1), np.float32)
    F[5][:] = np.sin(k * (i + 0.5) * dx + w * 0.5 * dt).astype(np.float32) + 0 * np.zeros(
        (ny, 1), np.float32)
    steps = 20
    for _ in range(steps):
        O.yee_advance_b(F, dx, dy, dt)
        O.yee_advance_e(F, None, dx, dy, dt)
    t = steps * dt
    ey = np.sin(k * i * dx - w * t)
    bz = np.sin(k * (i + 0.5) * dx - w * (t - 0.5 * dt))
    rows, cols = slice(22, 26), slice(30, 98)
    assert np.abs(F[1][rows, cols] - ey[:, cols]).max() < 2e-5
    assert np.abs(F[5][rows, cols] - bz[:, cols]).max() < 2e-5
    # the continuum wave (w = k) would be off by (w - k) t
    assert abs(w - k) * t > 1e-3
    for c in (0, 2, 3, 4):
        assert np.abs(F[c][rows, cols]).max() < 1e-6


def test_div_b_stays_zero_and_vacuum_energy_is_conserved():
    rng = np.random.default_rng(0)
    nx, ny, dx, dy = 96, 80, 0.3, 0.25
    dt = 0.5 * min(dx, dy)
    F = _zeros(nx, ny)
    # a smooth packet in the middle, far from the edges
    x = (np.arange(nx) - nx / 2)[None, :] * dx
    y = (np.arange(ny) - ny / 2)[:, None] * dy
    env = np.exp(-(x ** 2 + y ** 2) / 4.0)
    for c in (0, 1, 2):
        F[c][:] = (env * rng.uniform(-1, 1)).astype(np.float32)

    def div_b(F):
        bx, by = F[3].astype(np.float64), F[4].astype(np.float64)
        return (bx[:-1, 1:] - bx[:-1, :-1]) / dx + (by[1:, :-1] - by[:-1, :-1]) / dy

    energies = []
    for n in range(30):
        b_old = [F[c].astype(np.float64) for c in (3, 4, 5)]
        O.yee_advance_b(F, dx, dy, dt)
        b_new = [F[c].astype(np.float64) for c in (3, 4, 5)]
        e = [F[c].astype(np.float64) for c in (0, 1, 2)]
        # the scheme's conserved energy: E^n . E^n + B^(n-1/2) . B^(n+1/2)
        energies.append(sum((a * a).sum() for a in e) + sum((a * b).sum()
                                                            for a, b in zip(b_old, b_new)))
        O.yee_advance_e(F, None, dx, dy, dt)
        assert np.abs(div_b(F)).max() <= 1e-5 * max(1.0, np.abs(F[5]).max()) / dx
    assert max(energies) - min(energies) <= 2e-5 * energies[0]


def _lepton(xs, ys, us, w=1.0):
    n = len(xs)
    arr = {"x": np.asarray(xs, float), "y": np.asarray(ys, float), "z": np.zeros(n),
           "ux": np.array([u[0] for u in us]), "uy": np.array([u[1] for u in us]),
           "uz": np.array([u[2] for u in us]), "w": np.full(n, w)}
    return O.Species.from_arrays(arr, n, 2)


def test_current_deposition_totals_and_single_nodes():
    nx, ny, dx, dy, dt = 32, 24, 0.5, 0.4, 0.1
    rng = np.random.default_rng(1)
    n = 500
    us = rng.normal(0, 3, size=(n, 3))
    sp = _lepton(rng.uniform(4, 12, n), rng.uniform(3, 7, n), us, w=0.7)
    J = [np.zeros((ny, nx)) for _ in range(3)]
    O.deposit_current(sp, -1.0, dt, J, dx, dy)
    g = np.sqrt(1 + (us ** 2).sum(1))
    for c in range(3):
        # every stencil lies inside the grid: the grid total is the sum of q w v
        assert J[c].sum() * dx * dy == pytest.approx(-0.7 * (us[:, c] / g).sum(), rel=1e-12)
    # a particle whose mid-step position sits on a node of the E_z
    # staggering deposits its whole z current there
    u = np.array([0.0, 0.0, 2.0])
    sp1 = _lepton([5 * dx], [7 * dy], [u], w=2.0)
    J1 = [np.zeros((ny, nx)) for _ in range(3)]
    O.deposit_current(sp1, 1.0, dt, J1, dx, dy)
    vz = 2.0 / math.sqrt(5.0)
    assert J1[2][7, 5] == pytest.approx(2.0 * vz / (dx * dy), rel=1e-15)
    assert np.count_nonzero(J1[2]) == 1 and not J1[0].any() and not J1[1].any()
    # the mid-step position is x^(n+1) - v dt/2: a particle that ends the
    # step half a step past a node of the E_x staggering deposits there only
    ux = 3.0
    vx = ux / math.sqrt(1 + ux * ux)
    sp2 = _lepton([6.5 * dx + 0.5 * dt * vx], [4 * dy], [np.array([ux, 0.0, 0.0])])
    J2 = [np.zeros((ny, nx)) for _ in range(3)]
    O.deposit_current(sp2, -1.0, dt, J2, dx, dy)
    assert np.count_nonzero(np.abs(J2[0]) > 1e-9 * np.abs(J2[0]).max()) == 1
    assert J2[0][4, 6] == pytest.approx(-vx / (dx * dy), rel=1e-9)
    # at rest: nothing
    sp0 = _lepton([3.0], [3.0], [np.zeros(3)])
    J0 = [np.zeros((ny, nx)) for _ in range(3)]
    O.deposit_current(sp0, -1.0, dt, J0, dx, dy)
    assert not any(j.any() for j in J0)


def test_sort_by_cell_is_a_stable_permutation():
    rng = np.random.default_rng(2)
    n, nx, ny, dx, dy = 3000, 20, 10, 1.0, 1.0
    xs = rng.uniform(-2, 22, n)
    ys = rng.uniform(-1, 11, n)
    sp = _lepton(xs, ys, rng.normal(size=(n, 3)))
    sp.tau[:n] = np.arange(n)  # the original slot, carried along
    O.sort_by_cell(sp, nx, ny, dx, dy)
    cx, cy = np.floor(sp.x[:n] / dx), np.floor(sp.y[:n] / dy)
    inside = (cx >= 0) & (cx < nx) & (cy >= 0) & (cy < ny)
    key = np.where(inside, cy * nx + cx, nx * ny)
    assert np.all(np.diff(key) >= 0)
    orig = sp.tau[:n].astype(int)
    for k in np.unique(key):  # stable: slot order within a cell
        assert np.all(np.diff(orig[key == k]) > 0)
    assert sorted(orig) == list(range(n))
    np.testing.assert_array_equal(sp.x[:n], xs[orig])
    np.testing.assert_array_equal(sp.ux[:n] ** 2 >= 0, True)


def test_pic_twin_field_kicks_are_rounding_level():
    # the twin runs of the PIC parity test kick every grid value by a
    # relative +-eps after every cycle: without the kick a run repeats bit
    # for bit, with it the grid moves by about eps per cycle and no more
    from paper_1311_1107_gb300 import workloads as W
    from tests.parity import run_oracle

    w = W.laser_on_foil(nx=64, ny=32, ppc=2, foil_cells=2, n_steps=8,
                        photon_capacity=1 << 12, pair_capacity=1 << 8, pic=True)
    a, _ = run_oracle(w, 4)
    b, _ = run_oracle(w, 4)
    c, _ = run_oracle(w, 4, field_noise=2e-7, noise_key=0)
    d, _ = run_oracle(w, 4, field_noise=2e-7, noise_key=1)
    for k in range(6):
        fa, fb = a.field._keep[k], b.field._keep[k]
        assert np.array_equal(fa, fb)
    ey_a, ey_c, ey_d = a.field._keep[1], c.field._keep[1], d.field._keep[1]
    scale = np.abs(ey_a).max()
    assert scale > 0
    dc = np.abs(ey_c - ey_a).max() / scale
    assert 0 < dc < 1e-5
    assert not np.array_equal(ey_c, ey_d)  # the key picks the kick pattern
