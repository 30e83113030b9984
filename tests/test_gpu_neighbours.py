"""Target neighbour lists are never truncated (the paper's Sec. 1: all the
relevant interactions every time step).

An atom's Tersoff list holds up to 12 neighbours in shared memory; a longer
list moves whole to an overflow row in global memory and the forces stay
exact.  Only a list longer than an overflow row, or more overflowing atoms
than a track has rows for, fails the call with REED_E_NEIGHBOR -- never a
silent truncation.  Configurations:

* a compressed diamond cluster (a = 4.3 A, 2^3 cells, 0.05 A disorder):
  second neighbours at a/sqrt(2) = 3.04 A fall inside the 3.2 A list
  radius, so atoms have 4 (one-thread unrolled path), 5-12 (one-warp path,
  shared row) and up to 16 (overflow row) list neighbours, and some of the
  second neighbours sit inside the Tersoff cutoff region; forces against
  the FP64 oracle's brute-force Tersoff at 1e-10 in the FP64 path and 1e-4
  in the mixed form.  (Each centre here sums up to 16 x 15 bond-angle terms,
  many in the steep part of the cutoff function, whose sizes exceed the net
  force by about two orders of magnitude; FP32 rounding of the terms then
  reaches ~2e-5 of the net force.  The workloads' disordered lattices are
  held to 1e-5 in test_gpu_components.)
* a 5^3 grid of 0.9 A spacing: every atom has more neighbours than a row
  holds -- refused.
"""
import numpy as np
import pytest

from paper_0810_4737_gb300.workloads import workload

pytestmark = pytest.mark.gpu

DIAMOND = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                    [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])


@pytest.fixture(scope="module")
def R():
    from paper_0810_4737_gb300 import build, reed
    build.build()
    return reed


def _rel_err(fg, fo):
    scale = max(np.sqrt(np.mean(np.sum(fo ** 2, axis=1))), 1e-12)
    den = np.maximum(np.linalg.norm(fo, axis=1), 0.01 * scale)
    return np.max(np.linalg.norm(fg - fo, axis=1) / den)


def _list_sizes(X, rl=3.2):
    d = np.linalg.norm(X[:, None] - X[None], axis=2)
    np.fill_diagonal(d, np.inf)
    return (d < rl).sum(axis=1)


def _cluster(a, seed, offset):
    X = np.array([(np.array([i, j, k]) + b) * a for i in range(2) for j in range(2) for k in range(2)
                  for b in DIAMOND]) + offset
    X = X + np.random.default_rng(seed).normal(scale=0.05, size=X.shape)
    return X, np.zeros(len(X), dtype=np.int32)


@pytest.mark.parametrize("seed", [5, 6])
def test_long_lists_give_exact_tersoff_forces(R, O, seed):
    w = workload("as10kev_si_300k_tersoff")
    p = O.params(w)
    X, S = _cluster(4.3, seed, np.array([0.4, -0.3, 0.2]))
    m = _list_sizes(X)
    # the three paths: unrolled (<= 4), general in shared memory (5-12), overflow rows (> 12)
    assert (m <= 4).any() and ((m > 4) & (m <= 12)).any() and 0 < (m > 12).sum() <= 32, np.bincount(m)
    ion = X.mean(axis=0) + np.array([6.0, 0.5, -0.5])   # within the ion-target cutoff of a few atoms
    Eo, fio, fao, _ = O.forces(p, ion, X, S)
    with R.Reed(w) as ctx:
        for prec, tol in ((1, 1e-10), (0, 1e-4)):
            Eg, fig, fag, _ = ctx.forces(ion, X, S, precision=prec)
            assert _rel_err(fag, fao) < tol, (prec, _rel_err(fag, fao))
            assert np.linalg.norm(fig - fio) <= tol * max(np.linalg.norm(fio), 1e-12)
            assert abs(Eg - Eo) <= 10 * tol * max(abs(Eo), 1.0), (prec, Eg, Eo)


def test_lists_beyond_the_overflow_rows_are_refused(R, O):
    w = workload("as10kev_si_300k_tersoff")
    g = np.arange(5) * 0.9
    X = np.array([[x, y, z] for x in g for y in g for z in g]) + 1.0
    S = np.zeros(len(X), dtype=np.int32)
    assert _list_sizes(X).max() > 64
    with R.Reed(w) as ctx:
        for prec in (0, 1):
            with pytest.raises(R.ReedError) as e:
                ctx.forces(np.array([30.0, 30.0, 30.0]), X, S, precision=prec)
            assert e.value.code == R.E_NEIGHBOR
        # the context stays usable
        Xc, Sc = _cluster(5.431, 1, np.zeros(3))
        ctx.forces(np.array([30.0, 30.0, 30.0]), Xc, Sc, precision=0)


@pytest.mark.parametrize("prec,n", [(0, 96), (1, 24)])
def test_refreshed_lists_stay_exact(R, prec, n):
    """Whole As 10 keV Tersoff tracks with the lists' self-check on: after
    every full build, each list equals a brute-force search of the window;
    after every partial refresh (only the lists of atoms that moved more
    than half the skin recomputed), every pair within the Tersoff cutoff is
    listed and no listed pair is farther than the list radius plus the skin.
    Rebuilds at window moves and refreshes between them both happen."""
    w = workload("as10kev_si_300k_tersoff")
    with R.Reed(w) as ctx:
        ctx.run(n_ions=n, seed=3, precision=prec, nl_check=True)
        st = ctx.stats()
    assert st["tracks"] == n and st["failed"] == 0
    assert st["rebuilds"] > 0 and st["list_refreshes"] > 0, st
    assert st["nl_check_errors"] == 0, st
    assert st["nb_overflow"] == 0 and st["bond_cap_overflow"] == 0
