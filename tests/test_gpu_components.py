"""GPU parity of the stepper's components against the oracle, through the C ABI.

* Philox4x32-10 on the device: bit-exact (known answers and random blocks);
* cell creation: species and home cells bit-exact, positions within FP64
  rounding (FP64 path) or FP32 rounding (mixed path);
* window logic along a prescribed path: anchors and the set of cells in the
  final window bit-exact;
* forces of disordered configurations: ZBL ion-target and Tersoff target-
  target, 1e-5 relative in the mixed form, 1e-10 in the FP64 path.
"""
import numpy as np
import pytest

from paper_0810_4737_gb300.workloads import workload, SI, CE, O16

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_0810_4737_gb300 import build, reed
    build.build()
    return reed


def test_philox_bit_exact(R, O):
    import os
    from conftest import GOLDEN
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append(v)
    rows = np.array(rows, dtype=np.uint64).astype(np.uint32)
    out = R.reed_philox(rows[:, 0:4], rows[:, 4:6])
    assert np.array_equal(out, rows[:, 6:10])
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    gpu = R.reed_philox(ctr, key)
    for i in range(0, 4096, 97):
        assert np.array_equal(gpu[i], O.philox(ctr[i], key[i]))


@pytest.mark.parametrize("kind", ["diamond", "fluorite"])
def test_cell_atoms_match_oracle(R, O, kind):
    if kind == "diamond":
        w = workload("as10kev_si_300k_tersoff")
    else:
        w = workload("ar30kev_ceo2_300k_buck", tt="none")
    p = O.params(w)
    with R.Reed(w) as ctx:
        for key in (0, 1, 0xDEADBEEFCAFEF00D):
            for c in [(0, 0, 0), (3, -2, 7), (-5, 11, 0), (1, 1, -1), (100, -100, 1000)]:
                xg, sg = ctx.cell_atoms(key, *c)
                xo, so = O.cell_atoms(p, key, *c)
                assert xg.shape == xo.shape
                assert np.array_equal(sg, so)
                np.testing.assert_allclose(xg, xo, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,n", [("b1kev_si_0k_zbl", 3), ("as10kev_si_300k_tersoff", 5),
                                    ("ar30kev_ceo2_300k_buck", 4)])
@pytest.mark.parametrize("prec", [0, 1])
def test_window_replay_matches_oracle(R, O, name, n, prec):
    w = workload(name, tt="none", sigma=0.076)
    p = O.params(w)
    rng = np.random.default_rng(7 + n)
    steps = rng.normal(size=(4000, 3)) * 0.06
    steps[:, 2] += 0.02
    path = np.array([2.5, 1.5, -4.0]) + np.cumsum(steps, axis=0)
    key = 1234567
    with R.Reed(w) as ctx:
        ag, cg, bg, xg = ctx.window_replay(key, path, precision=prec)
    ao, co, bo, xo = O.window_replay(p, key, path)
    assert np.array_equal(ag, ao)
    kg = np.lexsort(np.c_[cg, bg].T)
    ko = np.lexsort(np.c_[co, bo].T)
    assert np.array_equal(cg[kg], co[ko]) and np.array_equal(bg[kg], bo[ko])
    tol = 1e-12 if prec == 1 else 4e-6
    np.testing.assert_allclose(xg[kg], xo[ko], rtol=0, atol=tol)


def _disordered(w, O, seed, ion_offset, n=None):
    """All atoms of an n^3-cell block around the ion with extra disorder."""
    p = O.params(w)
    rng = np.random.default_rng(seed)
    a, n = w["a"], (w["n"] if n is None else n)
    ion = np.array([1.3, 2.1, 7.7]) + ion_offset
    A = np.floor(ion / a + (0.5 if n % 2 == 0 else 0.0)).astype(int)
    xs, ss = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                c = A - n // 2 + np.array([i, j, k])
                x, s = O.cell_atoms(p, 99, *c)
                xs.append(x)
                ss.append(s)
    X = np.vstack(xs) + rng.normal(scale=0.12, size=(sum(len(x) for x in xs), 3))
    S = np.concatenate(ss)
    return ion, X, S


def _rel_err(fg, fo):
    scale = max(np.sqrt(np.mean(np.sum(fo ** 2, axis=1))), 1e-12)
    den = np.maximum(np.linalg.norm(fo, axis=1), 0.01 * scale)
    return np.max(np.linalg.norm(fg - fo, axis=1) / den)


@pytest.mark.parametrize("name", ["b1kev_si_0k_zbl", "as10kev_si_300k_tersoff"])
def test_forces_match_oracle(R, O, name):
    w = workload(name)
    p = O.params(w)
    for seed, off in [(1, 0.0), (2, 0.37), (3, np.array([2.2, -1.1, 0.6]))]:
        # every given atom is integrated and keeps a Tersoff force row in
        # shared memory: 4^3 cells (512 atoms) fit in the mixed form, 3^3 in FP64
        for prec, tol, n in ((1, 1e-10, 3), (0, 1e-5, 3), (0, 1e-5, 4)):
            ion, X, S = _disordered(w, O, seed, off, n=min(w["n"], n))
            # bring one atom close to the ion (hard collision)
            d = np.linalg.norm(X - ion, axis=1)
            X[np.argmin(d)] = ion + np.array([0.25, 0.1, -0.15])
            Eo, fio, fao, rho_o = O.forces(p, ion, X, S)
            with R.Reed(w) as ctx:
                Eg, fig, fag, rho_g = ctx.forces(ion, X, S, precision=prec)
                assert _rel_err(fag, fao) < tol, (prec, _rel_err(fag, fao))
                assert np.linalg.norm(fig - fio) <= tol * np.linalg.norm(fio)
                assert abs(Eg - Eo) <= tol * max(abs(Eo), 1.0) * 10


def test_forces_local_density_and_spline(R, O):
    w = workload("b1kev_si_0k_zbl", s_loc=0.5, spline_c=[0.05, -0.03, 0.02, 0.04, -0.05, 0.01])
    p = O.params(w)
    ion, X, S = _disordered(w, O, 4, 0.0)
    Eo, fio, fao, rho_o = O.forces(p, ion, X, S)
    with R.Reed(w) as ctx:
        for prec, tol in ((1, 1e-10), (0, 1e-5)):
            Eg, fig, fag, rho_g = ctx.forces(ion, X, S, precision=prec)
            assert _rel_err(fag, fao) < tol
            assert abs(rho_g - rho_o) <= tol * rho_o
