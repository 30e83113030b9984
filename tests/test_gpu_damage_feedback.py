"""GPU parity of the damage feedback (a new cell is amorphous with a
probability from the cumulative damage map) against the oracle, through
the C ABI.

* cell creation with a given map: the amorphous decision of every cell and
  the atom positions agree with the oracle (decisions bit-exact, positions
  1e-12 A in FP64);
* the window along a prescribed path with a given map: anchors, cells and
  positions as without feedback (bit-exact / 1e-12 A FP64 / 4e-6 A mixed);
* whole tracks: an amorphous surface layer shortens channelled B ranges on
  the GPU as in the oracle (same mean within statistics, KS p > 0.01);
* feedback between runs: a second run reads the damage the first deposited,
  and the two-run sequence is reproducible.
"""
import numpy as np
import pytest
from scipy import stats

from paper_0810_4737_gb300.workloads import workload

pytestmark = pytest.mark.gpu

DN, VOX = 8, 10.0


@pytest.fixture(scope="module")
def R():
    from paper_0810_4737_gb300 import build, reed
    build.build()
    return reed


def _w(**kw):
    base = dict(sigma=0.076, damage_n=DN, damage_voxel=VOX, dose_scale=1.0, e_crit=1.0, sigma_amorphous=0.5)
    base.update(kw)
    return workload("b1kev_si_0k_zbl", **base)


def _map(kind):
    m = np.zeros((DN, DN, DN))
    if kind == "saturated":
        m[:, :, :2] = 1e9
    else:   # e = ln 2 e_crit everywhere near the surface: half the cells amorphous
        m[:, :, :3] = np.log(2.0) * 8 * (VOX / 5.431) ** 3
    return np.append(m.ravel(), 0.0)


@pytest.mark.parametrize("kind", ["saturated", "ln2"])
def test_cell_creation_with_a_map(R, O, kind):
    w = _w()
    dmap = _map(kind)
    p = O.set_feedback_map(O.params(w), dmap)
    amorph = 0
    with R.Reed(w) as ctx:
        ctx.set_damage_map(dmap)
        for key in range(60):
            for c in [(0, 0, 0), (1, -1, 1), (-2, 3, 2), (3, 3, 4), (0, 0, 9)]:
                xg, sg = ctx.cell_atoms(key, *c)
                xo, so = O.cell_atoms(p, key, *c)
                assert np.array_equal(sg, so)
                np.testing.assert_allclose(xg, xo, rtol=0, atol=1e-12)
                site = O.cell_atoms(O.params(workload("b1kev_si_0k_zbl")), key, *c)[0]
                amorph += np.sqrt(np.mean((xg - site) ** 2)) > 0.25
    assert amorph > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_window_with_a_map(R, O, prec):
    w = _w()
    dmap = _map("ln2")
    p = O.set_feedback_map(O.params(w), dmap)
    rng = np.random.default_rng(11)
    steps = rng.normal(size=(3000, 3)) * 0.06
    steps[:, 2] += 0.02
    path = np.array([2.5, 1.5, -4.0]) + np.cumsum(steps, axis=0)
    with R.Reed(w) as ctx:
        ctx.set_damage_map(dmap)
        ag, cg, bg, xg = ctx.window_replay(77, path, precision=prec)
    ao, co, bo, xo = O.window_replay(p, 77, path)
    assert np.array_equal(ag, ao)
    kg, ko = np.lexsort(np.c_[cg, bg].T), np.lexsort(np.c_[co, bo].T)
    assert np.array_equal(cg[kg], co[ko]) and np.array_equal(bg[kg], bo[ko])
    np.testing.assert_allclose(xg[kg], xo[ko], rtol=0, atol=1e-12 if prec == 1 else 4e-6)


def test_amorphous_layer_shortens_channelled_ranges(R, O):
    w = _w(tilt=0.0, rot=(0.0, 0.0), sigma=0.0, n_bins=100, bin_w=5.0, sigma_amorphous=0.4)
    m = np.zeros((DN, DN, DN))
    m[:, :, :4] = 1e9
    dmap = np.append(m.ravel(), 0.0)
    n = 1024
    with R.Reed(w) as ctx:
        ctx.run(n_ions=n, seed=3, damage=False)
        plain = ctx.records()
    with R.Reed(w) as ctx:
        ctx.set_damage_map(dmap)
        ctx.run(n_ions=n, seed=3, damage=False)
        amor = ctx.records()
    zp = plain["z"][plain["status"] == 1]
    za = amor["z"][amor["status"] == 1]
    assert np.mean(za) < 0.9 * np.mean(zp)
    ref = O.run(O.params(w), n, seed=3, damage_init=dmap)["records"]
    zo = ref["z"][ref["status"] == 1]
    assert stats.ks_2samp(za, zo).pvalue > 0.01
    assert abs(np.mean(za) / np.mean(zo) - 1) < 4 * np.std(zo) / np.mean(zo) * np.sqrt(2.0 / len(zo))


def test_second_run_reads_the_first_runs_damage(R):
    # 1 keV B deposits a few hundred eV per ion in the top nanometres; with a
    # dose scale that makes the first run's damage amorphise the surface,
    # the second (otherwise identical) run channels less
    w = _w(tilt=0.0, rot=(0.0, 0.0), sigma=0.0, dose_scale=2e3, e_crit=1.0, sigma_amorphous=0.4)
    n = 2048
    out = []
    for _ in range(2):
        with R.Reed(w) as ctx:
            ctx.run(n_ions=n, seed=5, record_capacity=4 * n)   # room for both runs' records
            r1 = ctx.records()
            ctx.run(n_ions=n, seed=5, first_id=n)
            r2 = ctx.records()[len(r1):]
            d, ov = ctx.damage_map()
        out.append((r1, r2, d))
    (r1, r2, d), (s1, s2, e) = out
    assert d.sum() > 0
    z1, z2 = r1["z"][r1["status"] == 1], r2["z"][r2["status"] == 1]
    assert np.mean(z2) < np.mean(z1)
    # reproducible: each launch reads the map as it stood when it started
    for a, b in ((r1, s1), (r2, s2)):
        assert np.array_equal(np.sort(a, order="id"), np.sort(b, order="id"))
    assert np.allclose(d, e, rtol=1e-12, atol=0)
