"""Pins of the oracle's random streams, lattices and window.

Each check compares the oracle with something other than itself: published
known-answer vectors, crystallographic distances computed here from the
textbook site lists, exact moments of the normal distribution, and a
brute-force enumeration of lattice sites around the ion.
"""
import os

import numpy as np
import pytest
from scipy import stats

from conftest import GOLDEN
from paper_0810_4737_gb300.workloads import workload


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(O):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert O.philox(ctr, key).tolist() == expect


def _textbook_sites(kind, a, lo, hi):
    """Lattice sites written from the crystallography (not from the oracle):
    fcc translations, diamond = fcc + fcc shifted by a/4 (1,1,1); fluorite =
    cations on fcc, anions on the 8 tetrahedral holes (a/4)(+-1,+-1,+-1)."""
    fcc = np.array([[0, 0, 0], [0, 2, 2], [2, 0, 2], [2, 2, 0]], dtype=float) / 4.0
    if kind == "diamond":
        basis = np.vstack([fcc, fcc + 0.25])
        spec = np.zeros(8, dtype=int)
    else:
        anions = np.array([[i, j, k] for i in (1, 3) for j in (1, 3) for k in (1, 3)], dtype=float) / 4.0
        basis = np.vstack([fcc, anions])
        spec = np.array([0] * 4 + [1] * 8)
    pts, sp = [], []
    for ix in range(lo, hi):
        for iy in range(lo, hi):
            for iz in range(lo, hi):
                pts.append((basis + [ix, iy, iz]) * a)
                sp.append(spec)
    return np.vstack(pts), np.concatenate(sp)


@pytest.mark.parametrize("kind,a", [("diamond", 5.431), ("fluorite", 5.411)])
def test_cell_sites_match_crystallography(O, kind, a):
    w = workload("b1kev_si_0k_zbl", lattice=kind, a=a,
                 species=[{"Z": 58.0, "M": 140.116}, {"Z": 8.0, "M": 15.999}] if kind == "fluorite" else
                 [{"Z": 14.0, "M": 28.0855}])
    p = O.params(w)
    ref, ref_sp = _textbook_sites(kind, a, 0, 2)
    got, got_sp = [], []
    for ix in range(2):
        for iy in range(2):
            for iz in range(2):
                x, s = O.cell_atoms(p, 12345, ix, iy, iz)
                got.append(x)
                got_sp.append(s)
    got, got_sp = np.vstack(got), np.concatenate(got_sp)
    assert got.shape == ref.shape
    key = lambda X: np.lexsort(np.round(X, 9).T)
    np.testing.assert_allclose(got[key(got)], ref[key(ref)], atol=1e-12)
    assert sorted(got_sp.tolist()) == sorted(ref_sp.tolist())
    # cells above the surface are empty
    x, s = O.cell_atoms(p, 1, 0, 0, -1)
    assert x.shape[0] == 0


def test_nearest_neighbour_shells(O):
    """Si: 4 neighbours at a*sqrt(3)/4 = 2.3517 A; CeO2: 8 O around Ce at
    a*sqrt(3)/4 = 2.3430 A, O-O at a/2."""
    for kind, a, species in [("diamond", 5.431, [{"Z": 14.0, "M": 28.0855}]),
                             ("fluorite", 5.411, [{"Z": 58.0, "M": 140.116}, {"Z": 8.0, "M": 15.999}])]:
        p = O.params(workload("b1kev_si_0k_zbl", lattice=kind, a=a, species=species))
        xs, ss = [], []
        for ix in range(-1, 2):
            for iy in range(-1, 2):
                for iz in range(0, 3):
                    x, s = O.cell_atoms(p, 7, ix, iy, iz)
                    xs.append(x)
                    ss.append(s)
        X, S = np.vstack(xs), np.concatenate(ss)
        centre = np.array([0.5, 0.5, 1.5]) * a
        i0 = np.argmin(np.linalg.norm(X - centre, axis=1) + 100 * (S != 0))
        d = np.linalg.norm(X - X[i0], axis=1)
        d[i0] = np.inf
        nn = np.sort(d)
        if kind == "diamond":
            assert abs(nn[0] - a * np.sqrt(3) / 4) < 1e-12
            assert np.sum(np.abs(d - a * np.sqrt(3) / 4) < 1e-9) == 4
            assert abs(a * np.sqrt(3) / 4 - 2.3517) < 1e-4
        else:
            assert np.sum((np.abs(d - a * np.sqrt(3) / 4) < 1e-9) & (S == 1)) == 8
            io = np.argmin(np.linalg.norm(X - centre, axis=1) + 100 * (S != 1))
            do = np.linalg.norm(X - X[io], axis=1)
            do[io] = np.inf
            assert abs(np.min(do[S == 1]) - a / 2) < 1e-12
            assert abs(a * np.sqrt(3) / 4 - 2.3430) < 1e-4


def test_thermal_offsets_are_iid_normal(O):
    """Offsets from the Box-Muller stream: 0 mean, sigma^2 variance, normal
    kurtosis, no x-y-z correlation, normal CDF (KS)."""
    sigma = 0.076
    p = O.params(workload("b1kev_si_0k_zbl", sigma=sigma))
    p0 = O.params(workload("b1kev_si_0k_zbl", sigma=0.0))
    offs = []
    for ix in range(40):
        for iy in range(40):
            for iz in range(25):
                x, _ = O.cell_atoms(p, 99, ix, iy, iz)
                x0, _ = O.cell_atoms(p0, 99, ix, iy, iz)
                offs.append(x - x0)
    g = np.vstack(offs) / sigma
    n = g.size
    assert n >= 1_000_000 - 100_000
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(stats.kurtosis(g.ravel(), fisher=False) - 3) < 5 * np.sqrt(24 / n)
    c = np.corrcoef(g.T)
    assert np.max(np.abs(c - np.eye(3))) < 5 / np.sqrt(g.shape[0])
    assert stats.kstest(g.ravel()[:200_000], "norm").pvalue > 1e-3
    # re-entered cells reproduce the same offsets; another key does not
    a1, _ = O.cell_atoms(p, 99, 3, 4, 5)
    a2, _ = O.cell_atoms(p, 99, 3, 4, 5)
    a3, _ = O.cell_atoms(p, 100, 3, 4, 5)
    assert np.array_equal(a1, a2)
    assert not np.allclose(a1, a3)


def test_launch_positions_uniform_and_direction(O):
    w = workload("b1kev_si_0k_zbl", rot=(0.0, 45.0))
    p = O.params(w)
    xs, vs = [], []
    for i in range(4000):
        x, v = O.launch_state(p, 0, i)
        xs.append(x)
        vs.append(v)
    X, V = np.array(xs), np.array(vs)
    assert np.all(X[:, 2] == -w["rc"])
    for d in range(2):
        assert stats.kstest(X[:, d] / w["a"], "uniform").pvalue > 1e-3
    sp = np.linalg.norm(V, axis=1)
    np.testing.assert_allclose(0.5 * w["ion"]["M"] * sp ** 2, w["energy"], rtol=1e-12)
    tilt = np.degrees(np.arccos(V[:, 2] / sp))
    np.testing.assert_allclose(tilt, 7.0, atol=1e-9)
    rot = np.degrees(np.arctan2(V[:, 1], V[:, 0]))
    assert rot.min() >= 0 and rot.max() < 45
    assert stats.kstest(rot / 45.0, "uniform").pvalue > 1e-3
    # cone mode: uniform in solid angle within 10 degrees of [001]
    pc = O.params(workload("b1kev_si_0k_zbl", beam_mode="cone", tilt=10.0))
    ct = []
    for i in range(4000):
        _, v = O.launch_state(pc, 0, i)
        ct.append(v[2] / np.linalg.norm(v))
    ct = np.array(ct)
    cmax = np.cos(np.radians(10.0))
    assert ct.min() >= cmax - 1e-12
    assert stats.kstest((1 - ct) / (1 - cmax), "uniform").pvalue > 1e-3


@pytest.mark.parametrize("n,kind", [(3, "diamond"), (5, "diamond"), (4, "fluorite")])
def test_window_holds_every_site_near_the_ion(O, n, kind):
    """Along a random walk of the ion, the window (after re-anchoring) holds
    exactly the home-cell sites of an n^3 block, and every lattice site within
    the ion-target cutoff of the ion (brute-force enumeration)."""
    a = 5.431 if kind == "diamond" else 5.411
    species = ([{"Z": 14.0, "M": 28.0855}] if kind == "diamond"
               else [{"Z": 58.0, "M": 140.116}, {"Z": 8.0, "M": 15.999}])
    w = workload("b1kev_si_0k_zbl", n=n, lattice=kind, a=a, species=species)
    p = O.params(w)
    rng = np.random.default_rng(3)
    steps = rng.normal(size=(3000, 3)) * 0.05
    steps[:, 2] += 0.03
    path = np.array([3.0, 2.0, 1.0]) + np.cumsum(steps, axis=0)
    anc, cells, bas, xyz = O.window_replay(p, 777, path)
    nb = 8 if kind == "diamond" else 12
    # sites present are whole cells
    uc = np.unique(cells, axis=0)
    for c in uc:
        k = np.all(cells == c, axis=1)
        assert k.sum() == (nb if c[2] >= 0 else 0)
    # every site within rc of the final ion position is present
    lo = int(np.floor(path[-1].min() / a)) - 3
    hi = int(np.floor(path[-1].max() / a)) + 4
    sites, _ = _textbook_sites(kind, a, lo, hi)
    sites = sites[sites[:, 2] >= -1e-12]
    near = sites[np.linalg.norm(sites - path[-1], axis=1) < w["rc"]]
    assert len(near) > 5
    for s in near:
        assert np.min(np.linalg.norm(xyz - s, axis=1)) < 1e-9
    # anchors change by at most one cell per axis per point, and follow the ion
    h = 0.5 if n % 2 == 0 else 0.0
    np.testing.assert_array_equal(anc, np.floor(path / a + h).astype(int))
