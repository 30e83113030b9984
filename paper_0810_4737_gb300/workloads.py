"""Synthetic workload definitions shared by the tests, the benchmark and the
oracle binding.

This module holds input data only -- species, lattice, potential parameter
sets, beam geometry, counts and seeds -- and none of the method's
arithmetic.  Each side (the CUDA library and the CPU oracle) converts these
numbers into its own parameter layout and derives everything else itself.

The five workloads follow the synthetic cases of the REED-MD study:
  * ``b1kev_si_0k_zbl``      -- 32 B ions, 1 keV, perfect Si(100) at 0 K,
    3x3x3-cell window (216 atoms), ZBL ion-target only, fixed tilt 7 deg /
    rotation 22 deg (the small case);
  * ``as10kev_si_300k_tersoff`` -- 4096 As ions, 10 keV, Si at 300 K
    (sigma 0.076 A), Tersoff Si-Si with a ZBL blend, 5x5x5-cell window
    (1000 atoms, inner 27 cells integrated), rotation uniform in [0, 45) deg,
    100 depth bins of 1 nm (the throughput workload);
  * ``b50kev_si_300k_reed``  -- 65536 B ions, 50 keV, Si at 300 K, 12 cloning
    depths with weights 2^-k (geometric 20-600 nm as the initial guess of an
    adaptive run), 400 bins of 2 nm;
  * ``ar30kev_ceo2_300k_buck`` -- 16384 Ar ions, 30 keV, fluorite CeO2,
    4x4x4-cell window (768 atoms), Buckingham pairs with ZBL below 1 A,
    directions within 10 deg of [001], 64^3 damage voxels;
  * ``b10kev_si_300k_adjoint`` -- 16384 B ions, 10 keV, Si at 300 K, kernel-
    density depth profile (1 nm width, 200 bins) for the adjoint.

and the two actinide-oxide runs of the paper itself (Sec. 4.1, 4.2): ions
starting on a lattice site of bulk fluorite UO2 in a random direction, a
window of 27 cells of 12 atoms with the ion's cell in the centre, ZBL forces
only (Sec. 2 "First"), eight adaptive cloning distances, ranges measured from
the starting site:
  * ``u85kev_uo2_300k_recoil`` -- 5120 U-235 recoils of 85 keV (the recoil
    of a Pu-239 alpha decay), 200 bins of 5 A;
  * ``kr85mev_uo2_300k_recoil`` -- 1024 Kr fission fragments of 85 MeV,
    400 bins of 400 A (ranges of several micrometres), with the energy term
    of the time step at 100 eV: 0.05 A steps cannot resolve the closest
    approaches of an 85 MeV ion (~1e-3 A), and without the term a track can
    gain several times its energy.
The thermal displacement of the UO2 lattice comes from MD data the paper
cites but does not give; these workloads use the 0.076 A of the others.
"""
from __future__ import annotations

import copy

# Ion and target species: atomic number and mass (amu).
B11 = {"Z": 5.0, "M": 11.009305}
AS75 = {"Z": 33.0, "M": 74.921595}
AR40 = {"Z": 18.0, "M": 39.948}
SI = {"Z": 14.0, "M": 28.0855}
CE = {"Z": 58.0, "M": 140.116}
O16 = {"Z": 8.0, "M": 15.999}
U235 = {"Z": 92.0, "M": 235.043930}
U = {"Z": 92.0, "M": 238.02891}
KR = {"Z": 36.0, "M": 83.798}

# Tersoff Si(C) parameter set, Phys. Rev. B 38, 9902 (1988).
TERSOFF_SI_C = {
    "A": 1830.8, "B": 471.18, "lam1": 2.4799, "lam2": 1.7322,
    "beta": 1.1e-6, "n": 0.78734, "c": 100390.0, "d": 16.217, "h": -0.59825,
    "R": 2.85, "D": 0.15,
}

# Short-range Buckingham set for ceria: Ce4+-O2- from Gotte, Spangberg and
# Hakansson, Solid State Ionics 178 (2007) 1421; O2- - O2- from the Catlow
# oxide set.  Pair order: (cation-cation, cation-anion, anion-anion);
# A in eV, rho in A, C in eV A^6.  Cation-cation is ZBL only.
BUCKINGHAM_CEO2 = {
    "A": (0.0, 1986.83, 22764.3),
    "rho": (1.0, 0.35107, 0.149),
    "C": (0.0, 20.40, 27.89),
}

_BASE = {
    "lattice": "diamond",
    "target": "surface",    # "surface": z >= 0 with a (001) surface; "bulk": infinite, recoil beam
    "a": 5.431,
    "n": 3,
    "margin": 0,
    "sigma": 0.0,
    "species": [SI],
    "rc": 5.0,
    "rt": 4.5,
    "tt": "none",
    "tersoff": TERSOFF_SI_C,
    "blend": (1.0, 1.5),
    "buckingham": BUCKINGHAM_CEO2,
    "buck_cut": (4.5, 5.0),
    "buck_blend": (0.8, 1.0),
    "spline_c": [0.0] * 6,
    "s_e": 1.0,
    "s_loc": 0.0,
    "lam_loc": 0.5,
    "dt_max_fs": 0.1,
    "dx_max": 0.05,
    "de_max": 0.0,          # eV per step, energy term of the adaptive step (0 = off)
    "e_stop": 5.0,
    "step_cap": 2_000_000,
    "beam_mode": "fixed",
    "tilt": 7.0,
    "rot": (22.0, 22.0),
    "thresholds": [],
    "n_bins": 100,
    "bin_w": 2.0,
    "seed": 0,
    "damage_n": 0,          # cumulative damage map: voxels per edge (0 = off)
    "damage_voxel": 10.0,   # A
    "damage_min": 0.1,      # eV: atoms below this kinetic energy deposit nothing
}


def _geom(lo: float, hi: float, k: int) -> list:
    return [lo * (hi / lo) ** (i / (k - 1)) for i in range(k)]


WORKLOADS = {
    "b1kev_si_0k_zbl": dict(_BASE, ion=B11, energy=1000.0, n_ions=32, n_bins=100, bin_w=2.0),
    "as10kev_si_300k_tersoff": dict(
        _BASE, ion=AS75, energy=10000.0, n_ions=4096, n=5, margin=1, sigma=0.076,
        tt="tersoff", rot=(0.0, 45.0), n_bins=100, bin_w=10.0),
    "b50kev_si_300k_reed": dict(
        _BASE, ion=B11, energy=50000.0, n_ions=65536, sigma=0.076, rot=(0.0, 45.0),
        thresholds=_geom(200.0, 6000.0, 12), n_bins=400, bin_w=20.0),
    "ar30kev_ceo2_300k_buck": dict(
        _BASE, ion=AR40, energy=30000.0, n_ions=16384, lattice="fluorite", a=5.411, n=4,
        margin=0, sigma=0.076, species=[CE, O16], tt="buckingham", beam_mode="cone",
        tilt=10.0, rot=(0.0, 360.0), n_bins=200, bin_w=5.0, damage_n=64),
    "b10kev_si_300k_adjoint": dict(
        _BASE, ion=B11, energy=10000.0, n_ions=16384, sigma=0.076, rot=(0.0, 45.0),
        n_bins=200, bin_w=10.0),
    "u85kev_uo2_300k_recoil": dict(
        _BASE, ion=U235, energy=85000.0, n_ions=5120, lattice="fluorite", a=5.4704, n=3,
        sigma=0.076, species=[U, O16], target="bulk", beam_mode="recoil",
        thresholds=_geom(100.0, 800.0, 8), n_bins=200, bin_w=5.0),
    "kr85mev_uo2_300k_recoil": dict(
        _BASE, ion=KR, energy=85.0e6, n_ions=1024, lattice="fluorite", a=5.4704, n=3,
        sigma=0.076, species=[U, O16], target="bulk", beam_mode="recoil", step_cap=10_000_000,
        de_max=100.0, thresholds=_geom(20000.0, 100000.0, 8), n_bins=400, bin_w=400.0),
}


def workload(name: str, **overrides) -> dict:
    """A deep copy of a named workload with keyword overrides applied."""
    w = copy.deepcopy(WORKLOADS[name])
    w["name"] = name
    for k, v in overrides.items():
        w[k] = v
    return w
