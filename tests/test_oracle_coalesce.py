"""Pins of the oracle's super-photon compaction and coalescence (CPU only).

The paper names a coalescence that conserves energy and momentum on average
and gives no algorithm; the reading (two photons replace a group of at
least min_group photons of one cell, log2-energy bin and direction bin)
is pinned here by what it must conserve and by inputs whose groups are
known by construction, not by re-deriving its formulas."""
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle as O


def _photons(arr, cap=None, dims=3):
    n = len(arr["x"])
    sp = O.Species.from_arrays(arr, cap or n, dims)
    sp.tau[:n] = arr["tau"]
    return sp


def _totals(sp):
    n = sp.n
    w = sp.w[:n]
    u = np.stack([sp.ux[:n], sp.uy[:n], sp.uz[:n]], 1)
    e = np.linalg.norm(u, axis=1)
    return w.sum(), (w * e).sum(), (w[:, None] * u).sum(0)


def _random_photons(n, seed, dead_frac=0.2, dims=3):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3)) * [0.15, 0.15, 0.15] + [1.0, 0.0, 0.0]
    d /= np.linalg.norm(d, axis=1)[:, None]
    e = np.exp(rng.uniform(np.log(3.0), np.log(3000.0), n))
    arr = {"x": rng.uniform(0, 8, n), "y": rng.uniform(0, 8, n), "z": rng.uniform(0, 8, n),
           "ux": e * d[:, 0], "uy": e * d[:, 1], "uz": e * d[:, 2],
           "w": rng.uniform(0.5, 2.0, n),
           "tau": np.where(rng.uniform(size=n) < dead_frac, -1.0, rng.exponential(size=n))}
    return arr


BOX = (0.0, 0.0, 0.0, 2.0, 2.0, 2.0)
CELLS = (4, 4, 4)


def test_compaction_removes_decayed_photons_in_slot_order():
    arr = _random_photons(500, 1)
    arr["tau"][[3, 4]] = [0.0, -1e-300]  # tau = 0 is alive (the sentinel is < 0)
    sp = _photons(arr)
    alive = arr["tau"] >= 0
    assert alive[3] and not alive[4]
    stats = O.coalesce(sp, None)
    assert stats["n_dead"] == (~alive).sum() and sp.n == alive.sum()
    for k in ("x", "y", "z", "ux", "uy", "uz", "tau", "w"):
        np.testing.assert_array_equal(getattr(sp, k)[:sp.n], arr[k][alive])
    # nothing dead: nothing changes
    before = {k: getattr(sp, k)[:sp.n].copy() for k in ("x", "ux", "tau")}
    O.coalesce(sp, None)
    for k, v in before.items():
        np.testing.assert_array_equal(getattr(sp, k)[:sp.n], v)


def test_coalescence_conserves_weight_energy_momentum():
    arr = _random_photons(20000, 2)
    sp = _photons(arr)
    alive = arr["tau"] >= 0
    w = arr["w"][alive]
    u = np.stack([arr["ux"], arr["uy"], arr["uz"]], 1)[alive]
    W0, E0, P0 = w.sum(), (w * np.linalg.norm(u, axis=1)).sum(), (w[:, None] * u).sum(0)
    stats = O.coalesce(sp, O.coalesce_params(BOX, CELLS, 2, 2, 3))
    assert stats["groups_merged"] > 100 and sp.n < alive.sum()
    W1, E1, P1 = _totals(sp)
    assert W1 == pytest.approx(W0, rel=1e-13)
    assert E1 == pytest.approx(E0, rel=1e-13)
    np.testing.assert_allclose(P1, P0, rtol=1e-13, atol=1e-13 * E0)
    # every photon stays massless and carries a positive weight
    assert np.all(sp.w[:sp.n] > 0) and np.all(sp.tau[:sp.n] >= 0)


def _grouped_input(groups, seed, dims=3):
    """Photons in separate cells, each cell's photons inside one energy bin
    (8 per octave: [1, 1.125) of the octave) and one direction bin (near
    +x, 8 bins per face axis), so the groups are the cells."""
    rng = np.random.default_rng(seed)
    rows = []
    for g, n in enumerate(groups):
        cx, cy, cz = g % 4, (g // 4) % 4, g // 16
        for _ in range(n):
            e = 2.0 ** (3 + g % 5) * rng.uniform(1.01, 1.11)
            t = rng.uniform(0.01, 0.2, 2)  # transverse over axial: one bin
            d = np.array([1.0, t[0], t[1]])
            d /= np.linalg.norm(d)
            rows.append((2 * cx + rng.uniform(0.1, 1.9), 2 * cy + rng.uniform(0.1, 1.9),
                         (2 * cz + rng.uniform(0.1, 1.9)) if dims == 3 else 0.0,
                         *(e * d), rng.uniform(0.5, 3.0), rng.exponential(), g))
    rng.shuffle(rows)
    a = np.array(rows)
    return {"x": a[:, 0], "y": a[:, 1], "z": a[:, 2], "ux": a[:, 3], "uy": a[:, 4],
            "uz": a[:, 5], "w": a[:, 6], "tau": a[:, 7]}, a[:, 8].astype(int)


@pytest.mark.parametrize("dims", [3, 2])
def test_groups_known_by_construction_merge_into_conserving_pairs(dims):
    sizes = [1, 2, 3, 4, 7, 20, 2, 5]
    arr, gid = _grouped_input(sizes, 3, dims)
    n = len(gid)
    sp = _photons(arr, dims=dims)
    if dims == 2:
        sp.z = None
    cells = CELLS if dims == 3 else (4, 4, 1)
    stats = O.coalesce(sp, O.coalesce_params(BOX, cells, 8, 8, 3, dims=dims, seed=7))
    merged = [k for k, s in enumerate(sizes) if s >= 3]
    assert stats["groups_merged"] == len(merged)
    assert sp.n == sum(2 if s >= 3 else s for s in sizes)
    # survivors in slot order: each group's output sits at its first slot
    first = {g: int(np.flatnonzero(gid == g)[0]) for g in range(len(sizes))}
    order = []
    for i in range(n):
        g = gid[i]
        if sizes[g] < 3:
            order.append(("kept", i))
        elif first[g] == i:
            order += [("pair", g), ("pair", g)]
    assert len(order) == sp.n
    for k, (kind, v) in enumerate(order):
        if kind == "kept":
            assert sp.x[k] == arr["x"][v] and sp.ux[k] == arr["ux"][v]
            assert sp.tau[k] == arr["tau"][v]
            continue
        m = gid == v
        w, u = arr["w"][m], np.stack([arr["ux"][m], arr["uy"][m], arr["uz"][m]], 1)
        W, E, P = w.sum(), (w * np.linalg.norm(u, axis=1)).sum(), (w[:, None] * u).sum(0)
        if order[k - 1] == ("pair", v):
            continue  # checked with its partner
        a = np.array([sp.ux[k], sp.uy[k], sp.uz[k]])
        b = np.array([sp.ux[k + 1], sp.uy[k + 1], sp.uz[k + 1]])
        assert sp.w[k] == sp.w[k + 1] == pytest.approx(W / 2, rel=1e-15)
        # the group's energy and momentum, exactly; both photons massless
        assert sp.w[k] * (np.linalg.norm(a) + np.linalg.norm(b)) == pytest.approx(E, rel=1e-13)
        np.testing.assert_allclose(sp.w[k] * (a + b), P, rtol=1e-13, atol=1e-13 * E)
        assert np.linalg.norm(a) == pytest.approx(E / W, rel=1e-13)
        assert np.linalg.norm(b) == pytest.approx(E / W, rel=1e-13)
        # at the weighted mean position of the group
        X = np.array([(w * arr[c][m]).sum() / W for c in ("x", "y", "z")])
        assert sp.x[k] == pytest.approx(X[0], rel=1e-14)
        assert sp.y[k] == pytest.approx(X[1], rel=1e-14)
        if dims == 3:
            assert sp.z[k] == pytest.approx(X[2], rel=1e-14)
        # symmetric about P / W, in the plane of P and the group's first photon
        f = np.flatnonzero(m)[0]
        r = np.array([arr["ux"][f], arr["uy"][f], arr["uz"][f]])
        assert abs(np.dot(np.cross(P, r), a - b)) <= 1e-9 * np.linalg.norm(P) * \
            np.linalg.norm(r) * np.linalg.norm(a - b)
        assert sp.tau[k] > 0 and sp.tau[k + 1] > 0


def test_weighted_spectra_are_invariant_on_its_energy_bins_and_close_in_angle():
    # a merged pair carries its group's weight at the group's mean energy,
    # which lies in the group's energy bin: the weighted energy spectrum on
    # the coalescence's own log2 bins (and on any coarser power-of-two
    # grid) is unchanged.  Directions move within about a direction bin:
    # the weighted polar-angle spectrum on bins four times wider agrees
    # within the sampling noise (chi2 with the weighted variances).
    arr = _random_photons(30000, 4, dead_frac=0.0)
    sp = _photons(arr)
    B = 4

    def spectrum(e, w, per_octave):
        m, ex = np.frexp(e)  # e = m 2^ex, m in [0.5, 1)
        b = ex * per_octave + np.floor((2 * m - 1) * per_octave).astype(int)
        return np.bincount(b - 0, weights=w, minlength=2000)

    u0 = np.stack([arr["ux"], arr["uy"], arr["uz"]], 1)
    e0, w0 = np.linalg.norm(u0, axis=1), arr["w"]
    stats = O.coalesce(sp, O.coalesce_params(BOX, CELLS, B, 8, 3))
    assert stats["photons_merged"] > 5000
    u1 = np.stack([sp.ux[:sp.n], sp.uy[:sp.n], sp.uz[:sp.n]], 1)
    e1, w1 = np.linalg.norm(u1, axis=1), sp.w[:sp.n]
    for per_octave in (B, B // 2, 1):
        s0, s1 = spectrum(e0, w0, per_octave), spectrum(e1, w1, per_octave)
        np.testing.assert_allclose(s1, s0, rtol=1e-12, atol=1e-12 * s0.max())
    # polar angle about +x; direction bins span 2/8 of tan on a face
    th0 = np.arccos(u0[:, 0] / e0)
    th1 = np.arccos(u1[:, 0] / e1)
    edges = np.linspace(0.0, th0.max() * 1.001, 9)
    h0 = np.histogram(th0, edges, weights=w0)[0]
    h1 = np.histogram(np.minimum(th1, edges[-1] * 0.9999), edges, weights=w1)[0]
    v0 = np.histogram(th0, edges, weights=w0 * w0)[0]
    v1 = np.histogram(np.minimum(th1, edges[-1] * 0.9999), edges, weights=w1 * w1)[0]
    chi2 = ((h1 - h0) ** 2 / (v0 + v1)).sum()
    assert st.chi2.sf(chi2, len(h0) - 1) > 1e-3, (h0, h1)


def test_merged_optical_depths_are_exponential():
    arr = _random_photons(40000, 5, dead_frac=0.0)
    sp = _photons(arr)
    O.coalesce(sp, O.coalesce_params(BOX, CELLS, 2, 2, 3, seed=11, step=5))
    n0 = 40000
    # the merged photons are those whose weight is not an input weight
    merged = ~np.isin(sp.w[:sp.n], arr["w"])
    t = sp.tau[:sp.n][merged]
    assert len(t) > 2000
    assert st.kstest(t, "expon").pvalue > 1e-3
    assert sp.n < n0


def test_photons_outside_the_box_are_kept():
    arr = _random_photons(3000, 6, dead_frac=0.0)
    arr["x"] = arr["x"] + 100.0  # every photon outside the grid
    sp = _photons(arr)
    stats = O.coalesce(sp, O.coalesce_params(BOX, CELLS, 2, 2, 3))
    assert stats["groups_merged"] == 0 and sp.n == 3000
    np.testing.assert_array_equal(sp.ux[:3000], arr["ux"])


def test_bad_parameters_are_rejected():
    sp = _photons(_random_photons(10, 7))
    for kw in ({"min_group": 2}, {"ebins_per_octave": 0}, {"dir_bins": 65}):
        p = O.coalesce_params(BOX, CELLS, **{"ebins_per_octave": 2, "dir_bins": 2,
                                             "min_group": 3, **kw})
        with pytest.raises(ValueError):
            O.coalesce(sp, p)


def test_large_groups_merge_in_runs_of_max_group():
    # one group of 1000 photons (one cell, energy bin and direction bin),
    # max_group 256: runs of 256, 256, 256 and 232 slots in slot order, each
    # replaced by its own conserving pair
    arr, gid = _grouped_input([1000], 8)
    order = np.argsort(np.arange(1000))  # slot order = input order
    sp = _photons(arr)
    stats = O.coalesce(sp, O.coalesce_params(BOX, CELLS, 8, 8, 3, max_group=256))
    assert stats["groups_merged"] == 4 and stats["photons_merged"] == 1000 and sp.n == 8
    for r, (a, b) in enumerate(((0, 256), (256, 512), (512, 768), (768, 1000))):
        m = order[a:b]
        w, u = arr["w"][m], np.stack([arr["ux"][m], arr["uy"][m], arr["uz"][m]], 1)
        W, P = w.sum(), (w[:, None] * u).sum(0)
        k = 2 * r
        np.testing.assert_allclose(sp.w[k] * (np.array([sp.ux[k], sp.uy[k], sp.uz[k]])
                                              + np.array([sp.ux[k + 1], sp.uy[k + 1],
                                                          sp.uz[k + 1]])), P, rtol=1e-13)
        assert sp.w[k] == pytest.approx(W / 2, rel=1e-15)
    # a tail run shorter than min_group is kept as it is
    arr2, _ = _grouped_input([258], 9)
    sp2 = _photons(arr2)
    st2 = O.coalesce(sp2, O.coalesce_params(BOX, CELLS, 8, 8, 3, max_group=256))
    assert st2["groups_merged"] == 1 and sp2.n == 2 + 2
