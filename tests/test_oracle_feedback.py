"""Pins of the oracle's damage feedback (the reading: a new cell is amorphous
with probability 1 - exp(-e / e_crit), e = dose_scale * D / N the energy per
target atom of its voxel; amorphous cells take the larger thermal offset).

* an empty map changes nothing, bit for bit;
* a saturated map makes every cell in it amorphous: the offsets of created
  atoms have the amorphous width, cells outside the map keep the lattice's;
* at e = ln 2 e_crit half of the cells are amorphous (binomial bounds), and
  the voxel a cell belongs to is the one holding its centre;
* an amorphous surface layer shortens channelled ranges (B along [001]).
"""
import numpy as np

from paper_0810_4737_gb300.workloads import workload

DN, VOX = 8, 10.0


def _w(**kw):
    base = dict(sigma=0.076, damage_n=DN, damage_voxel=VOX, dose_scale=1.0, e_crit=1.0, sigma_amorphous=0.5)
    base.update(kw)
    return workload("b1kev_si_0k_zbl", **base)


def _offsets(O, p, key, cell):
    xyz, sp = O.cell_atoms(p, key, *cell)
    site = O.cell_atoms(O.params(workload("b1kev_si_0k_zbl", sigma=0.0)), key, *cell)[0]
    return xyz - site


def _cells_in_voxel(vx, vy, vz, a=5.431):
    # cells whose centres lie in voxel (vx, vy, vz) of an 8^3 x 10 A map
    half = 0.5 * DN * VOX
    out = []
    for ix in range(-12, 12):
        for iy in range(-12, 12):
            for iz in range(0, 16):
                c = np.array([(ix + 0.5) * a + half, (iy + 0.5) * a + half, (iz + 0.5) * a])
                if tuple(np.floor(c / VOX).astype(int)) == (vx, vy, vz):
                    out.append((ix, iy, iz))
    return out


def test_empty_map_changes_nothing(O):
    p0 = O.params(workload("b1kev_si_0k_zbl", sigma=0.076))
    p1 = O.set_feedback_map(O.params(_w()), np.zeros(DN ** 3 + 1))
    for key in (1, 99, 12345):
        for cell in [(0, 0, 0), (-3, 2, 5), (4, -4, 1)]:
            a, _ = O.cell_atoms(p0, key, *cell)
            b, _ = O.cell_atoms(p1, key, *cell)
            assert np.array_equal(a, b)


def test_saturated_map_amorphises_every_cell_in_it(O):
    m = np.zeros((DN, DN, DN))
    m[:, :, :2] = 1e9                       # top 20 A: saturated
    p = O.set_feedback_map(O.params(_w()), np.append(m.ravel(), 0.0))
    inside, outside = [], []
    for key in range(40):
        for cell in [(0, 0, 0), (1, -1, 1), (-2, 3, 2)]:     # centres at z < 20 A
            inside.append(_offsets(O, p, key, cell))
        for cell in [(0, 0, 5), (2, 2, 8)]:                  # z > 20 A
            outside.append(_offsets(O, p, key, cell))
    sd_in = np.std(np.concatenate(inside))
    sd_out = np.std(np.concatenate(outside))
    assert abs(sd_in / 0.5 - 1) < 0.08, sd_in
    assert abs(sd_out / 0.076 - 1) < 0.08, sd_out


def test_half_of_the_cells_at_ln2(O):
    # 8 atoms per cell, (10 / 5.431)^3 cells per voxel -> N atoms per voxel
    N = 8 * (VOX / 5.431) ** 3
    m = np.zeros((DN, DN, DN))
    vox = (4, 4, 1)
    m[vox] = np.log(2.0) * N                # e = ln 2 with e_crit = 1, dose_scale = 1
    p = O.set_feedback_map(O.params(_w()), np.append(m.ravel(), 0.0))
    cells = _cells_in_voxel(*vox)
    assert len(cells) >= 4
    amorph, total = 0, 0
    for key in range(300):
        for cell in cells:
            d = _offsets(O, p, key, cell)
            amorph += np.sqrt(np.mean(d ** 2)) > 0.25
            total += 1
    f = amorph / total
    assert abs(f - 0.5) < 4 * np.sqrt(0.25 / total), (f, total)
    # a neighbouring voxel with no damage: never amorphous
    other = _cells_in_voxel(4, 4, 3)
    for key in range(50):
        for cell in other:
            assert np.sqrt(np.mean(_offsets(O, p, key, cell) ** 2)) < 0.25


def test_amorphous_surface_layer_shortens_channelled_ranges(O):
    w = _w(tilt=0.0, rot=(0.0, 0.0), sigma=0.0, n_bins=100, bin_w=5.0, sigma_amorphous=0.4)
    p = O.params(w)
    n = 256
    plain = O.run(p, n, seed=3, records=True)["records"]
    m = np.zeros((DN, DN, DN))
    m[:, :, :4] = 1e9                       # amorphous down to 40 A
    amor = O.run(O.params(w), n, seed=3, records=True, damage_init=np.append(m.ravel(), 0.0))["records"]
    z0 = plain["z"][plain["status"] == 1]
    z1 = amor["z"][amor["status"] == 1]
    assert np.mean(z1) < 0.9 * np.mean(z0), (np.mean(z1), np.mean(z0))
