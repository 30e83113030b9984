"""ctypes binding of the FP64 CPU oracle (``oracle/reed_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it; the product library never does.  It
imports nothing from the product package -- callers pass workload dicts in.

The shared library is compiled with gcc on first use (or by ``build()``)
into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reed_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

TAU_FS = 10.180505710  # sqrt(amu A^2 / eV) in fs

STOPPED, BACK, TRUNC = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: runs on x86-64 and Arm)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
               "-o", _OUT + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_OUT + ".tmp", _OUT)
    return _OUT


class Params(C.Structure):
    _fields_ = [
        ("Z1", C.c_double), ("M1", C.c_double),
        ("lattice", C.c_int), ("n", C.c_int), ("margin", C.c_int), ("nspec", C.c_int),
        ("target", C.c_int),
        ("a", C.c_double), ("sigma", C.c_double),
        ("Z2", C.c_double * 2), ("M2", C.c_double * 2),
        ("rc", C.c_double), ("rt", C.c_double),
        ("screening", C.c_int), ("tt", C.c_int),
        ("spline_c", C.c_double * 6),
        ("ters", C.c_double * 11),
        ("blend_lo", C.c_double), ("blend_hi", C.c_double),
        ("bk_A", C.c_double * 3), ("bk_rho", C.c_double * 3), ("bk_C", C.c_double * 3),
        ("bk_rc", C.c_double), ("bk_rt", C.c_double), ("bk_lo", C.c_double), ("bk_hi", C.c_double),
        ("s_e", C.c_double), ("s_loc", C.c_double), ("lam_loc", C.c_double),
        ("dt_max", C.c_double), ("dx_max", C.c_double), ("e_stop", C.c_double),
        ("step_cap", C.c_int64),
        ("E0", C.c_double), ("tilt", C.c_double), ("rot_lo", C.c_double), ("rot_hi", C.c_double),
        ("beam_mode", C.c_int),
        ("nthr", C.c_int), ("thr", C.c_double * 16),
        ("nbins", C.c_int), ("bin_w", C.c_double),
        ("dn", C.c_int), ("dvox", C.c_double), ("dmin", C.c_double),
        ("de_max", C.c_double),
        ("dose_scale", C.c_double), ("fb_ec", C.c_double), ("sigma_am", C.c_double),
        ("fb_map", C.c_void_p),
        ("dx_min", C.c_double),
    ]


class Record(C.Structure):
    _fields_ = [("id", C.c_uint64), ("primary", C.c_uint64), ("z", C.c_double), ("t", C.c_double),
                ("steps", C.c_int64), ("level", C.c_int32), ("status", C.c_int32)]


RECORD_DTYPE = np.dtype([("id", "<u8"), ("primary", "<u8"), ("z", "<f8"), ("t", "<f8"),
                         ("steps", "<i8"), ("level", "<i4"), ("status", "<i4")])

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U32 = C.POINTER(C.c_uint32)
_P = C.POINTER(Params)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            L.o_philox.argtypes = [_U32, _U32, _U32]
            L.o_track_key.argtypes = [C.c_uint64, C.c_uint64]
            L.o_track_key.restype = C.c_uint64
            L.o_child_id.argtypes = [C.c_uint64, C.c_int]
            L.o_child_id.restype = C.c_uint64
            L.o_gauss3.argtypes = [_U32, _D]
            L.o_cell_atoms.argtypes = [_P, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, _D, _I]
            L.o_cell_atoms.restype = C.c_int
            L.o_zbl.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, _D, _D]
            L.o_zbl_screen_length.argtypes = [C.c_double, C.c_double]
            L.o_zbl_screen_length.restype = C.c_double
            L.o_ion_pair_energy.argtypes = [_P, C.c_double, C.c_double, _D]
            L.o_ion_pair_energy.restype = C.c_double
            L.o_taper_export.argtypes = [C.c_double, C.c_double, C.c_double, _D]
            L.o_taper_export.restype = C.c_double
            L.o_forces.argtypes = [_P, _D, C.c_int, C.c_int, _D, _I, _D, _D, _D]
            L.o_forces.restype = C.c_double
            L.o_gamma_ls.argtypes = [_P]
            L.o_gamma_ls.restype = C.c_double
            L.o_rho0.argtypes = [_P]
            L.o_rho0.restype = C.c_double
            L.o_run.argtypes = [_P, C.c_int64, C.c_int64, C.c_uint64, C.c_int, _D,
                                C.POINTER(C.c_int64), _D, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]
            L.o_free.argtypes = [C.c_void_p]
            L.o_run_damage.argtypes = [_P, C.c_int64, C.c_int64, C.c_uint64, C.c_int, _D,
                                       C.POINTER(C.c_int64), _D, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), _D]
            L.o_track_energy.argtypes = [_P, C.c_uint64, C.c_uint64, _D]
            L.o_track_energy.restype = C.c_int
            L.o_trace.argtypes = [_P, C.c_uint64, C.c_uint64, C.c_int, _D, _I]
            L.o_trace.restype = C.c_int
            L.o_window_replay.argtypes = [_P, C.c_uint64, C.c_int, _D, _I, C.c_int, _I, _I, _D]
            L.o_window_replay.restype = C.c_int
            L.o_md_explicit.argtypes = [_P, _D, _D, C.c_int, _D, _D, _I, _I, C.c_int, C.c_double,
                                        C.c_double, _D]
            L.o_md_explicit.restype = C.c_int
            L.o_launch_state.argtypes = [_P, C.c_uint64, C.c_uint64, _D, _D]
            L.o_update_thresholds.argtypes = [_D, C.c_int, C.c_double, C.c_int, _D]
            L.o_update_thresholds.restype = C.c_int
            L.o_run_adaptive.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, C.c_int, _D,
                                         C.POINTER(C.c_int64), _D, _D, C.c_int]
            L.o_run_adaptive.restype = C.c_int
            L.o_pair_full.argtypes = [_P, C.c_double, C.c_double, _D, _D, _D, _D]
            L.o_segment_tangent.argtypes = [_P, C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_int64, _D]
            L.o_segment_tangent.restype = C.c_int
            L.o_segment_replay_theta.argtypes = [_P, C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_int64, C.c_int,
                                                 C.c_double, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.o_segment_replay_theta.restype = C.c_double
            L.o_bspline3_export.argtypes = [C.c_double, _D]
            L.o_bspline3_export.restype = C.c_double
            L.o_spline_corr_export.argtypes = [_D, C.c_double, _D]
            L.o_spline_corr_export.restype = C.c_double
            L.o_basis_count.argtypes = [C.c_int]
            L.o_basis_count.restype = C.c_int
            _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


_LATTICE = {"diamond": 0, "fluorite": 1, "explicit": -1}
_TT = {"none": 0, "tersoff": 1, "buckingham": 2}


def params(w: dict, screening: int = 1) -> Params:
    """Oracle parameters from a workload dict (see the workloads module)."""
    p = Params()
    p.Z1, p.M1 = w["ion"]["Z"], w["ion"]["M"]
    p.lattice = _LATTICE[w["lattice"]]
    p.n, p.margin = int(w["n"]), int(w["margin"])
    sp = w["species"]
    p.nspec = len(sp)
    p.a, p.sigma = w["a"], w["sigma"]
    for i, s in enumerate(sp):
        p.Z2[i], p.M2[i] = s["Z"], s["M"]
    p.rc, p.rt = w["rc"], w["rt"]
    p.screening = screening
    p.tt = _TT[w["tt"]]
    for i, c in enumerate(w["spline_c"]):
        p.spline_c[i] = c
    t = w["tersoff"]
    for i, k in enumerate(["A", "B", "lam1", "lam2", "beta", "n", "c", "d", "h", "R", "D"]):
        p.ters[i] = t[k]
    p.blend_lo, p.blend_hi = w["blend"]
    b = w["buckingham"]
    for i in range(3):
        p.bk_A[i], p.bk_rho[i], p.bk_C[i] = b["A"][i], b["rho"][i], b["C"][i]
    p.bk_rt, p.bk_rc = w["buck_cut"]
    p.bk_lo, p.bk_hi = w["buck_blend"]
    p.s_e, p.s_loc, p.lam_loc = w["s_e"], w["s_loc"], w["lam_loc"]
    p.dt_max = w["dt_max_fs"] / TAU_FS
    p.dx_max = w["dx_max"]
    p.e_stop = w["e_stop"]
    p.step_cap = int(w["step_cap"])
    p.E0 = w["energy"]
    p.tilt = w["tilt"]
    p.rot_lo, p.rot_hi = w["rot"]
    p.beam_mode = {"fixed": 0, "cone": 1, "recoil": 2}[w["beam_mode"]]
    p.target = {"surface": 0, "bulk": 1}[w.get("target", "surface")]
    thr = list(w["thresholds"])
    assert len(thr) <= 16
    p.nthr = len(thr)
    for i, d in enumerate(thr):
        p.thr[i] = d
    p.nbins, p.bin_w = int(w["n_bins"]), float(w["bin_w"])
    p.dn, p.dvox, p.dmin = int(w.get("damage_n", 0)), float(w.get("damage_voxel", 10.0)), float(w.get("damage_min", 0.1))
    p.de_max = float(w.get("de_max", 0.0))
    p.dose_scale = float(w.get("dose_scale", 0.0))
    p.fb_ec = float(w.get("e_crit", 0.0))
    p.sigma_am = float(w.get("sigma_amorphous", 0.0))
    p.fb_map = None
    p.dx_min = min(float(w.get("dx_min", 0.0)) or 1e-4, float(w["dx_max"]))
    return p


def set_feedback_map(p: Params, damage_map):
    """Damage map (dn^3 voxels + overflow, FP64) read by cell creation when
    damage feedback is on; the array is kept alive on the Params object."""
    a = np.ascontiguousarray(damage_map, dtype=np.float64).ravel()
    assert a.size == p.dn ** 3 + 1
    p._fb_keep = a
    p.fb_map = a.ctypes.data
    return p


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def track_key(seed: int, track_id: int) -> int:
    return int(lib().o_track_key(seed, track_id))


def child_id(parent: int, level: int) -> int:
    return int(lib().o_child_id(parent, level))


def gauss3(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    g = np.zeros(3)
    lib().o_gauss3(w.ctypes.data_as(_U32), _dp(g))
    return g


def cell_atoms(p: Params, key: int, ix: int, iy: int, iz: int):
    xyz = np.zeros((12, 3))
    sp = np.zeros(12, dtype=np.int32)
    m = lib().o_cell_atoms(C.byref(p), key, ix, iy, iz, _dp(xyz), _ip(sp))
    return xyz[:m].copy(), sp[:m].copy()


def zbl(Z1, Z2, r, screening=1):
    V, dV = C.c_double(), C.c_double()
    lib().o_zbl(Z1, Z2, screening, r, C.byref(V), C.byref(dV))
    return V.value, dV.value


def screen_length(Z1, Z2):
    return lib().o_zbl_screen_length(Z1, Z2)


def ion_pair(p: Params, Z2: float, r: float):
    dU = C.c_double()
    U = lib().o_ion_pair_energy(C.byref(p), Z2, r, C.byref(dU))
    return U, dU.value


def taper(r, rt, rc):
    dS = C.c_double()
    S = lib().o_taper_export(r, rt, rc, C.byref(dS))
    return S, dS.value


def forces(p: Params, ion_x, x, sp, with_ion=True):
    """(energy, f_ion[3], f_atoms[n,3], rho) for an explicit configuration."""
    xi = np.ascontiguousarray(ion_x, dtype=np.float64)
    xa = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(sp, dtype=np.int32)
    fi = np.zeros(3)
    fa = np.zeros_like(xa)
    rho = C.c_double()
    E = lib().o_forces(C.byref(p), _dp(xi), int(with_ion), xa.shape[0], _dp(xa), _ip(s), _dp(fi),
                       _dp(fa), C.byref(rho))
    return E, fi, fa, rho.value


def gamma_ls(p: Params) -> float:
    return lib().o_gamma_ls(C.byref(p))


def rho0(p: Params) -> float:
    return lib().o_rho0(C.byref(p))


def launch_state(p: Params, seed: int, track_id: int):
    x, v = np.zeros(3), np.zeros(3)
    lib().o_launch_state(C.byref(p), seed, track_id, _dp(x), _dp(v))
    return x, v


def run(p: Params, n_ions: int, seed: int, first_id: int = 0, threads: int | None = None,
        records: bool = True, damage_init=None):
    """Run primaries [first_id, first_id+n_ions); returns a dict with the
    histogram (nbins + under/over/back), counters and per-track records."""
    nb = p.nbins + 3
    hist = np.zeros(nb)
    cnt = np.zeros(4, dtype=np.int64)
    wt = np.zeros(1)
    if threads is None:
        threads = os.cpu_count() or 1
    ptr = C.c_void_p()
    nrec = C.c_int64(0)
    dmg = np.zeros(p.dn ** 3 + 1) if p.dn > 0 else None
    if dmg is not None and damage_init is not None:
        dmg[:] = np.asarray(damage_init, dtype=np.float64).ravel()   # cumulative map before this run
    lib().o_run_damage(C.byref(p), n_ions, first_id, seed, threads, _dp(hist),
                       cnt.ctypes.data_as(C.POINTER(C.c_int64)), _dp(wt),
                       C.byref(ptr) if records else None, C.byref(nrec), _dp(dmg) if dmg is not None else None)
    out = {"hist": hist[:p.nbins].copy(), "under": hist[p.nbins], "over": hist[p.nbins + 1],
           "back": hist[p.nbins + 2], "w_trunc": wt[0], "steps": int(cnt[0]),
           "tracks": int(cnt[1]), "clones": int(cnt[2]), "shifts": int(cnt[3])}
    if dmg is not None:
        out["damage"] = dmg[:-1].reshape(p.dn, p.dn, p.dn)
        out["damage_overflow"] = dmg[-1]
    if records:
        n = nrec.value
        buf = (C.c_char * (n * RECORD_DTYPE.itemsize)).from_address(ptr.value)
        out["records"] = np.frombuffer(bytes(buf), dtype=RECORD_DTYPE).copy()
        lib().o_free(ptr)
    return out


def trace(p: Params, seed: int, track_id: int, nsteps: int):
    """First nsteps steps of a primary: array (k, 8) of x y z t vx vy vz dt and
    the window anchors (k, 3)."""
    out = np.zeros((nsteps, 8))
    anc = np.zeros((nsteps, 3), dtype=np.int32)
    k = lib().o_trace(C.byref(p), seed, track_id, nsteps, _dp(out), _ip(anc))
    return out[:k].copy(), anc[:k].copy()


def window_replay(p: Params, key: int, path):
    path = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    n = path.shape[0]
    anc = np.zeros((n, 3), dtype=np.int32)
    cap = p.n ** 3 * 12 + 16
    cells = np.zeros((cap, 3), dtype=np.int32)
    bas = np.zeros(cap, dtype=np.int32)
    xyz = np.zeros((cap, 3))
    m = lib().o_window_replay(C.byref(p), key, n, _dp(path), _ip(anc), cap, _ip(cells), _ip(bas), _dp(xyz))
    return anc, cells[:m].copy(), bas[:m].copy(), xyz[:m].copy()


def md_explicit(p: Params, ion_x, ion_v, x, v, sp, act=None, nsteps=1000, dt_fixed=0.0,
                stop_sep=0.0, energies=False):
    """Explicit-atom MD with the oracle's integrator (no window, no lattice).
    Returns (ion_x, ion_v, x, v, steps, energies-or-None)."""
    xi = np.array(ion_x, dtype=np.float64)
    vi = np.array(ion_v, dtype=np.float64)
    xa = np.array(x, dtype=np.float64).reshape(-1, 3)
    va = np.array(v, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(sp, dtype=np.int32)
    a = np.ones(xa.shape[0], dtype=np.int32) if act is None else np.ascontiguousarray(act, dtype=np.int32)
    E = np.zeros(nsteps + 1) if energies else None
    k = lib().o_md_explicit(C.byref(p), _dp(xi), _dp(vi), xa.shape[0], _dp(xa), _dp(va), _ip(s), _ip(a),
                            nsteps, dt_fixed, stop_sep, _dp(E) if energies else None)
    return xi, vi, xa, va, k, (E[:k + 1] if energies else None)


def update_thresholds(hist_full, bin_w, nthr):
    """Cloning depths d_k = S^-1(2^-k) from a histogram of nbins + 3 entries."""
    h = np.ascontiguousarray(hist_full, dtype=np.float64)
    out = np.zeros(max(nthr, 1))
    rc = lib().o_update_thresholds(_dp(h), h.size - 3, bin_w, nthr, _dp(out))
    if rc != 0:
        raise ValueError("empty histogram")
    return out[:nthr].copy()


def run_adaptive(p: Params, n_ions: int, n_initial: int, epoch: int, seed: int, threads: int | None = None,
                 max_epochs: int = 256):
    """Adaptive-depth run (see o_run_adaptive); returns the histogram dict and
    the depths used by each enhanced epoch."""
    nb = p.nbins + 3
    hist = np.zeros(nb)
    cnt = np.zeros(4, dtype=np.int64)
    wt = np.zeros(1)
    th = np.zeros((max_epochs, 16))
    ne = lib().o_run_adaptive(C.byref(p), n_ions, n_initial, epoch, seed, threads or (os.cpu_count() or 1),
                              _dp(hist), cnt.ctypes.data_as(C.POINTER(C.c_int64)), _dp(wt), _dp(th), max_epochs)
    return {"hist": hist[:p.nbins].copy(), "under": hist[p.nbins], "over": hist[p.nbins + 1],
            "back": hist[p.nbins + 2], "w_trunc": wt[0], "steps": int(cnt[0]), "tracks": int(cnt[1]),
            "clones": int(cnt[2]), "thresholds": th[:min(ne, max_epochs), :p.nthr].copy(), "epochs": ne}


def track_energy(p: Params, seed: int, track_id: int) -> dict:
    """Energy bookkeeping of one primary (no cloning); needs p.dn > 0."""
    out = np.zeros(8)
    if lib().o_track_energy(C.byref(p), seed, track_id, _dp(out)) != 0:
        raise ValueError("needs a damage grid and <= 1024 bins")
    keys = ["E0", "ke_ion", "pe", "e_elec", "deposited", "below_threshold", "ke_window", "steps"]
    return dict(zip(keys, out.tolist()))


def pair_full(p: Params, Z2: float, r: float):
    """Ion-target pair: (U, dU/dr, d2U/dr2, d(dU/dr)/dc_k for k = 0..5)."""
    U, dU, d2U = C.c_double(), C.c_double(), C.c_double()
    dc = np.zeros(6)
    lib().o_pair_full(C.byref(p), Z2, r, C.byref(U), C.byref(dU), C.byref(d2U), _dp(dc))
    return U.value, dU.value, d2U.value, dc


def bspline3(u: float):
    """The oracle's centred cubic B-spline of unit knot spacing: (B(u), B'(u))."""
    du = C.c_double()
    b = lib().o_bspline3_export(u, C.byref(du))
    return b, du.value


def spline_corr(c, r: float):
    """The ZBL correction c(r) = sum_i c_i B_i(ln r) and dc/dr (oracle)."""
    cc = np.ascontiguousarray(c, dtype=np.float64)
    assert cc.size == 6
    d = C.c_double()
    v = lib().o_spline_corr_export(_dp(cc), r, C.byref(d))
    return v, d.value


def segment_tangent(p: Params, seed: int, track_id: int, seg: int = 200, every: int = 20, cap: int = 2_000_000):
    """Forward-mode dz_T/dtheta over the frozen last segment of a primary:
    dict(z, T, s0, grad[8]) with theta = (s_e, s_loc, c_1..c_6)."""
    out = np.zeros(11)
    if lib().o_segment_tangent(C.byref(p), seed, track_id, seg, every, cap, _dp(out)) != 0:
        raise ValueError("track did not stop")
    return {"z": out[0], "T": int(out[1]), "s0": int(out[2]), "grad": out[3:].copy()}


def segment_z(p: Params, seed: int, track_id: int, direction: int, delta: float, seg: int = 200, every: int = 20,
              cap: int = 2_000_000):
    """z_T of the frozen segment replayed with theta_direction += delta."""
    T, s0 = C.c_int64(), C.c_int64()
    z = lib().o_segment_replay_theta(C.byref(p), seed, track_id, seg, every, cap, direction, delta, C.byref(T),
                                     C.byref(s0))
    return z, T.value, s0.value
