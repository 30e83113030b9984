"""Pins of the oracle's bulk target and recoil beam (the paper's UO2 runs:
ions starting on a lattice site in a random direction, Sec. 4.1, 4.2).

* launch: every recoil starts on the origin site with |v| = sqrt(2 E / M) and
  a direction uniform on the sphere (cos theta and phi uniform, KS);
* lattice: a bulk target fills space (cells above z = 0 are populated) and
  lacks exactly the recoil's own site; the atoms within rc of that site are
  the fluorite shells 8 O at a sqrt(3)/4, 12 U at a/sqrt(2), 24 O at
  a sqrt(11)/4, and the force on the ion there vanishes (inversion symmetry);
* stopping acts everywhere in a bulk target: with no atoms the drag ODE gives
  the closed-form range M (v0 - v_stop) / gamma in any direction, also
  upwards, where a surface target has no stopping;
* the range is the distance from the start: records equal |x| of the last
  traced position, and the histogram equals the binned records; the stops
  are symmetric about the start (mean position 0 within its error);
* energy balance of a recoil track with the damage map centred on the start,
  and the map receives deposits on both sides of z = 0;
* adaptive cloning on the distance: weights sum to the primaries exactly;
* 85 MeV Kr: with the energy term of the time step the energy balance of a
  track holds (0.5 %) and its range stays below the drag-only bound; without
  it, unresolved close collisions create energy (the same track gains
  several times E0 and overshoots the bound);
* the energy term (with its 1e-4 A floor on the step) resolves an 85 MeV
  Kr-O collision at impact parameters 1e-3-0.1 A: the O recoil energy equals
  T_max sin^2(theta/2) from the classical deflection integral within 1e-3,
  while 0.05 A steps alone miss it by a factor 2 to 250.
"""
import numpy as np
import pytest
from scipy import stats

from paper_0810_4737_gb300.workloads import workload, KR, U235

A_UO2 = 5.4704


def _w(**kw):
    return workload("u85kev_uo2_300k_recoil", **kw)


def test_recoil_launch_is_isotropic(O):
    p = O.params(_w())
    n = 20000
    v = np.array([O.launch_state(p, 3, i)[1] for i in range(n)])
    x = np.array([O.launch_state(p, 3, i)[0] for i in range(0, n, 97)])
    assert np.all(x == 0.0)
    sp = np.linalg.norm(v, axis=1)
    np.testing.assert_allclose(sp, np.sqrt(2 * 85000.0 / U235["M"]), rtol=1e-13)
    u = v / sp[:, None]
    assert stats.kstest(u[:, 2], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    phi = np.mod(np.arctan2(u[:, 1], u[:, 0]), 2 * np.pi)
    assert stats.kstest(phi, stats.uniform(loc=0, scale=2 * np.pi).cdf).pvalue > 1e-3
    # isotropy: the mean direction is zero and the second moment is I/3
    assert np.all(np.abs(u.mean(axis=0)) < 4 * np.sqrt(1 / 3 / n))
    np.testing.assert_allclose(u.T @ u / n, np.eye(3) / 3, atol=4 * np.sqrt(2 / 15 / n))


def test_bulk_cells_fill_space_with_a_vacancy_at_the_origin(O):
    pb = O.params(_w(sigma=0.0))
    ps = O.params(_w(sigma=0.0, target="surface", beam_mode="cone"))
    for key in (1, 77):
        xb, sb = O.cell_atoms(pb, key, 0, 0, 0)
        xs, ss = O.cell_atoms(ps, key, 0, 0, 0)
        assert len(xs) == 12 and len(xb) == 11
        assert np.min(np.linalg.norm(xb, axis=1)) > 1.0          # nothing on the recoil's site
        np.testing.assert_array_equal(xb, xs[1:])                  # the other 11 sites unchanged
        np.testing.assert_array_equal(sb, ss[1:])
        for c in [(0, 0, -1), (2, -3, -5), (-1, 1, 0)]:
            xb, _ = O.cell_atoms(pb, key, *c)
            assert len(xb) == 12
        assert len(O.cell_atoms(ps, key, 0, 0, -1)[0]) == 0       # surface target: above z = 0 empty
    # thermal offsets of the other sites are unchanged by the vacancy
    pt = O.params(_w())
    pts = O.params(_w(target="surface", beam_mode="cone"))
    np.testing.assert_array_equal(O.cell_atoms(pt, 5, 0, 0, 0)[0], O.cell_atoms(pts, 5, 0, 0, 0)[0][1:])


def _window_atoms(p, key, lo=-1, hi=1):
    xs, ss = [], []
    for i in range(lo, hi + 1):
        for j in range(lo, hi + 1):
            for k in range(lo, hi + 1):
                x, s = O_cell(p, key, i, j, k)
                xs.append(x)
                ss.append(s)
    return np.vstack(xs), np.concatenate(ss)


def O_cell(p, key, i, j, k):
    from oracle import oracle
    return oracle.cell_atoms(p, key, i, j, k)


def test_shells_and_zero_force_at_the_recoil_site(O):
    w = _w(sigma=0.0)
    p = O.params(w)
    x, s = _window_atoms(p, 0)
    r = np.linalg.norm(x, axis=1)
    near = r < w["rc"]
    a = A_UO2
    shells = {(1, a * np.sqrt(3) / 4): 8, (0, a / np.sqrt(2)): 12, (1, a * np.sqrt(11) / 4): 24}
    assert near.sum() == sum(shells.values())
    for (spc, d), cnt in shells.items():
        sel = np.abs(r - d) < 1e-9
        assert sel.sum() == cnt and np.all(s[sel] == spc)
    _, fi, _, _ = O.forces(p, np.zeros(3), x, s)
    # a single nearest-neighbour U-O pair pushes with a few eV/A; the shells cancel
    _, f1, _, _ = O.forces(p, np.zeros(3), x[np.argmin(r)][None], s[np.argmin(r)][None])
    assert np.linalg.norm(f1) > 1.0
    assert np.linalg.norm(fi) < 1e-9 * np.linalg.norm(f1)


@pytest.mark.parametrize("direction", [(0.0, 0.0, -1.0), (0.48, -0.6, 0.64)])
def test_drag_range_closed_form_in_every_direction(O, direction):
    w = workload("kr85mev_uo2_300k_recoil", energy=2.0e5)
    p = O.params(w)
    gam = O.gamma_ls(p)
    M = KR["M"]
    v0 = np.sqrt(2 * 2.0e5 / M)
    vs = np.sqrt(2 * 5.0 / M)
    d = np.array(direction) / np.linalg.norm(direction)
    none = (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0, dtype=np.int32))
    xi, *_ = O.md_explicit(p, [0.0, 0.0, 0.0], v0 * d, *none, nsteps=20_000_000)
    expect = M * (v0 - vs) / gam
    assert abs(np.linalg.norm(xi) - expect) < 1e-3 * expect + 0.05
    np.testing.assert_allclose(xi / np.linalg.norm(xi), d, atol=1e-12)
    if d[2] < 0:   # a surface target has no stopping above z = 0: the ion keeps its speed
        ps = O.params(workload("kr85mev_uo2_300k_recoil", energy=2.0e5, target="surface", beam_mode="cone"))
        _, vi, *_ = O.md_explicit(ps, [0.0, 0.0, -1.0], v0 * d, *none, nsteps=1000)
        np.testing.assert_allclose(np.linalg.norm(vi), v0, rtol=1e-14)


def test_range_is_the_distance_from_the_start(O):
    w = _w(n_bins=100, bin_w=8.0, thresholds=[])
    p = O.params(w)
    n = 24
    r = O.run(p, n, seed=7, threads=8)
    rec = r["records"]
    assert np.all(rec["status"] == 1) and len(rec) == n
    ends = []
    for tid in range(n):
        tr, _ = O.trace(p, 7, tid, int(rec["steps"][rec["id"] == tid][0]) + 10)
        x = tr[-1, :3]
        ends.append(x)
        z = rec["z"][rec["id"] == tid][0]
        assert abs(z - np.sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2])) < 1e-12 * z
    hist = np.zeros(w["n_bins"] + 1)
    for z in rec["z"]:
        hist[min(int(z // w["bin_w"]), w["n_bins"])] += 1.0
    np.testing.assert_array_equal(r["hist"], hist[:-1])
    assert r["over"] == hist[-1] and r["under"] == 0 and r["back"] == 0
    ends = np.array(ends)
    se = ends.std(axis=0) / np.sqrt(n)
    assert np.all(np.abs(ends.mean(axis=0)) < 4.5 * se)
    assert np.any(ends[:, 2] < -20.0) and np.any(ends[:, 2] > 20.0)   # stops on both sides of z = 0
    # with cloning on the distance, the weighted histogram equals the binned records
    wc = _w(n_bins=100, bin_w=8.0)
    r = O.run(O.params(wc), n, seed=7, threads=8)
    rec = r["records"]
    assert r["clones"] > 0 and len(rec) == n + r["clones"]
    hist = np.zeros(wc["n_bins"] + 1)
    for z, lv in zip(rec["z"], rec["level"]):
        hist[min(int(z // wc["bin_w"]), wc["n_bins"])] += 2.0 ** -lv
    np.testing.assert_array_equal(r["hist"], hist[:-1])
    assert np.sum(2.0 ** -rec["level"].astype(float)) == n


def test_recoil_energy_balance_and_centred_damage_map(O):
    w = _w(damage_n=32, damage_voxel=20.0)
    p = O.params(w)
    for tid in range(4):
        e = O.track_energy(p, 0, tid)
        rest = e["ke_ion"] + e["pe"] + e["e_elec"] + e["deposited"] + e["below_threshold"] + e["ke_window"]
        assert abs(rest / e["E0"] - 1.0) < 1e-2, (tid, e)
    r = O.run(p, 48, seed=2, threads=8)
    d = r["damage"]
    assert d[:, :, :16].sum() > 0 and d[:, :, 16:].sum() > 0
    assert r["damage_overflow"] < 0.05 * d.sum()


def test_adaptive_cloning_on_the_distance(O):
    w = _w()
    p = O.params(w)
    r = O.run_adaptive(p, 400, 50, 175, seed=4, threads=8)
    total = r["hist"].sum() + r["under"] + r["over"] + r["back"] + r["w_trunc"]
    assert total == 400.0
    assert r["back"] == 0 and r["under"] == 0
    th = r["thresholds"]
    assert th.shape[1] == 8 and np.all(np.diff(th, axis=1) > 0)
    assert r["clones"] > 0


def test_energy_term_keeps_85_mev_tracks_conservative(O):
    from concurrent.futures import ThreadPoolExecutor
    base = dict(thresholds=[], damage_n=64, damage_voxel=5000.0)
    wk = workload("kr85mev_uo2_300k_recoil", **base)
    w0 = workload("kr85mev_uo2_300k_recoil", de_max=0.0, **base)
    assert wk["de_max"] > 0

    def balance(w):
        e = O.track_energy(O.params(w), 0, 0)
        rest = e["ke_ion"] + e["pe"] + e["e_elec"] + e["deposited"] + e["below_threshold"] + e["ke_window"]
        return rest / e["E0"] - 1.0

    def rng(w):
        return O.run(O.params(w), 1, seed=0, threads=1)["records"]["z"][0]

    with ThreadPoolExecutor(4) as ex:     # the oracle releases the GIL
        b1, b0, z1, z0 = ex.map(lambda f: f[0](f[1]), [(balance, wk), (balance, w0), (rng, wk), (rng, w0)])
    M, E = KR["M"], wk["energy"]
    bound = M * (np.sqrt(2 * E / M) - np.sqrt(2 * wk["e_stop"] / M)) / O.gamma_ls(O.params(wk))
    assert abs(b1) < 5e-3 and z1 < bound
    assert b0 > 0.5 and z0 > bound


@pytest.mark.parametrize("b", [1e-3, 0.02, 0.1])
def test_energy_term_resolves_mev_close_collisions(O, b):
    from test_oracle_potentials import deflection_angle
    from paper_0810_4737_gb300.workloads import O16
    M1, M2, E = KR["M"], O16["M"], 85.0e6
    mu = M1 * M2 / (M1 + M2)
    v0 = np.sqrt(2 * E / M1)
    T = {}
    for de in (100.0, 0.0):
        w = workload("kr85mev_uo2_300k_recoil", de_max=de, s_e=0.0, e_stop=0.0, lattice="explicit")
        p = O.params(w)
        rc = w["rc"]
        z0 = -np.sqrt(rc ** 2 - b ** 2) - 1e-6
        _, _, _, va, k, _ = O.md_explicit(p, [b, 0.0, z0], [0.0, 0.0, v0], [[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0]],
                                          np.array([1], dtype=np.int32), nsteps=1_000_000, stop_sep=rc + 1e-3)
        assert k < 1_000_000
        T[de] = 0.5 * M2 * np.sum(va[0] ** 2)
    th = deflection_angle(lambda r: O.ion_pair(p, O16["Z"], r)[0] if r < rc else 0.0, 0.5 * mu * v0 ** 2, b)
    exact = 4 * M1 * M2 / (M1 + M2) ** 2 * E * np.sin(th / 2) ** 2
    assert abs(T[100.0] / exact - 1) < 1e-3, (T, exact)
    if b < 0.05:
        assert abs(T[0.0] / exact - 1) > 0.5
