"""Python binding of the C ABI in ``include/reed.h`` (ctypes).

Argument marshalling only: every step of the track computation runs in the
CUDA library.  Functions carry the C names; ``Reed`` wraps a context.  The
library must have been built (``paper_0810_4737_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
E_ARG, E_CUDA, E_TIMEOUT, E_QUEUE_FULL, E_NONFINITE, E_NOMEM, E_SMEM, E_STATE, E_NEIGHBOR = range(-1, -10, -1)
LATTICE = {"diamond": 0, "fluorite": 1}
TT = {"none": 0, "tersoff": 1, "buckingham": 2}
PREC_MIXED, PREC_FP64 = 0, 1
BEAM = {"fixed": 0, "cone": 1, "recoil": 2}
TARGET = {"surface": 0, "bulk": 1}
STOPPED, BACKSCATTERED, TRUNCATED, FAILED = 1, 2, 3, 4
TAU_FS = 10.180505710


class reed_lattice(C.Structure):
    _fields_ = [("kind", C.c_int32), ("window_n", C.c_int32), ("frozen_margin", C.c_int32),
                ("target", C.c_int32), ("a", C.c_double), ("sigma", C.c_double)]


class reed_species(C.Structure):
    _fields_ = [("Z", C.c_double), ("M", C.c_double)]


class reed_potentials(C.Structure):
    _fields_ = [("rc", C.c_double), ("r_taper", C.c_double), ("spline_c", C.c_double * 6),
                ("target_model", C.c_int32), ("reserved", C.c_int32), ("tersoff", C.c_double * 11),
                ("tersoff_blend", C.c_double * 2), ("buck_A", C.c_double * 3), ("buck_rho", C.c_double * 3),
                ("buck_C", C.c_double * 3), ("buck_cut", C.c_double * 2), ("buck_blend", C.c_double * 2),
                ("s_e", C.c_double), ("s_loc", C.c_double), ("lam_loc", C.c_double)]


class reed_run_opts(C.Structure):
    _fields_ = [("dt_max_fs", C.c_double), ("dx_max", C.c_double), ("e_stop", C.c_double),
                ("step_cap", C.c_int64), ("beam_mode", C.c_int32), ("precision", C.c_int32),
                ("n_thresholds", C.c_int32), ("n_bins", C.c_int32), ("thresholds", C.c_double * 16),
                ("bin_width", C.c_double), ("first_id", C.c_int64), ("threads_per_track", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("record_tracks", C.c_int32), ("trace_tracks", C.c_int32),
                ("trace_steps", C.c_int32), ("reserved", C.c_int32), ("record_capacity", C.c_int64),
                ("stream", C.c_void_p), ("adaptive", C.c_int32), ("device_thresholds", C.c_int32),
                ("epoch_size", C.c_int64), ("n_initial", C.c_int64), ("target_tracks", C.c_int64),
                ("damage_n", C.c_int32), ("reserved3", C.c_int32), ("damage_voxel", C.c_double),
                ("damage_min", C.c_double), ("adjoint", C.c_int32), ("adj_segment", C.c_int32),
                ("adj_every", C.c_int32), ("nl_check", C.c_int32),
                ("nl_skin", C.c_double), ("de_max", C.c_double), ("pool_poll_limit", C.c_int64),
                ("dx_min", C.c_double)]


class reed_track_record(C.Structure):
    _fields_ = [("id", C.c_uint64), ("primary", C.c_uint64), ("z", C.c_double), ("t", C.c_double),
                ("steps", C.c_int64), ("level", C.c_int32), ("status", C.c_int32)]


RECORD_DTYPE = np.dtype([("id", "<u8"), ("primary", "<u8"), ("z", "<f8"), ("t", "<f8"),
                         ("steps", "<i8"), ("level", "<i4"), ("status", "<i4")])


class reed_peaks_t(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("fp32_tflops", "fp64_tflops", "ex2_gops", "rsqrt_gops", "smem_tbs",
                                          "sm_mhz")] + [("sms", C.c_int32), ("reserved", C.c_int32)]


class reed_tune_entry(C.Structure):
    _fields_ = [("threads_per_track", C.c_int32), ("ctas_per_sm", C.c_int32), ("ion_steps_per_s", C.c_double)]


class reed_stats_t(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "primaries", "clones", "tracks", "steps", "pair_evals", "bond_evals", "shifts", "rebuilds",
        "stopped", "backscattered", "truncated", "failed", "dropped_clones", "nb_overflow", "bond_cap_overflow",
        "triplets", "atom_updates")] + [("phase_cycles", C.c_int64 * 6)] + \
        [("w_stopped", C.c_double), ("w_back", C.c_double), ("w_trunc", C.c_double), ("kernel_ms", C.c_double),
         ("threads_per_track", C.c_int32), ("ctas_per_sm", C.c_int32), ("grid", C.c_int32),
         ("smem_bytes", C.c_int32), ("splits", C.c_int64 * 16), ("pooled", C.c_int64),
         ("nb_spilled", C.c_int64), ("list_refreshes", C.c_int64), ("nl_check_errors", C.c_int64),
         ("centre_class", C.c_int64 * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_cycles"] = list(self.phase_cycles)
        d["centre_class"] = list(self.centre_class)
        d["splits"] = list(self.splits)
        return d


EXPORTED = ["reed_init", "reed_run", "reed_range_profile", "reed_stats", "reed_track_records", "reed_trace",
            "reed_reset", "reed_last_error", "reed_destroy", "reed_philox", "reed_cell_atoms", "reed_forces",
            "reed_window_replay", "reed_run_static", "reed_thresholds", "reed_damage_map", "reed_track_grads",
            "reed_kde_profile", "reed_grad", "reed_set_theta", "reed_update_thresholds", "reed_get_thresholds", "reed_peaks", "reed_autotune",
            "reed_set_damage_feedback", "reed_set_damage_map"]

_LIB = None
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_U32 = C.POINTER(C.c_uint32)


class ReedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("REED error %d: %s" % (code, msg))
        self.code = code


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libreed.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libreed.so is not built (%s); run paper_0810_4737_gb300.build.build()" % path)
        L = C.CDLL(path)
        vp = C.c_void_p
        L.reed_init.argtypes = [C.POINTER(vp), C.POINTER(reed_lattice), C.POINTER(reed_species), C.c_int,
                                C.POINTER(reed_potentials)]
        L.reed_run.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_int64, C.c_uint64, C.POINTER(reed_run_opts)]
        L.reed_range_profile.argtypes = [vp, vp, C.c_int, vp]
        L.reed_stats.argtypes = [vp, C.POINTER(reed_stats_t)]
        L.reed_track_records.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.reed_trace.argtypes = [vp, vp, vp, C.c_int, C.c_int]
        L.reed_reset.argtypes = [vp]
        L.reed_thresholds.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_int)]
        L.reed_damage_map.argtypes = [vp, vp, C.c_int, vp]
        L.reed_track_grads.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.reed_kde_profile.argtypes = [vp, C.c_double, C.c_int, C.c_double, vp]
        L.reed_grad.argtypes = [vp, C.c_double, C.c_int, C.c_double, vp, vp]
        L.reed_set_theta.argtypes = [vp, _D]
        L.reed_update_thresholds.argtypes = [vp, vp, C.c_int, C.c_double, C.c_int, _D]
        L.reed_get_thresholds.argtypes = [vp, vp]
        L.reed_peaks.argtypes = [C.POINTER(reed_peaks_t)]
        L.reed_set_damage_feedback.argtypes = [vp, C.c_double, C.c_double, C.c_double]
        L.reed_set_damage_map.argtypes = [vp, vp, C.c_int, C.c_double]
        L.reed_autotune.argtypes = [vp] + [C.c_double] * 6 + [C.c_int64, C.c_uint64, C.POINTER(reed_run_opts),
                                                              C.POINTER(reed_tune_entry), C.c_int, _I32]
        L.reed_last_error.argtypes = [vp]
        L.reed_last_error.restype = C.c_char_p
        L.reed_destroy.argtypes = [vp]
        L.reed_destroy.restype = None
        L.reed_philox.argtypes = [_U32, _U32, _U32, C.c_int64]
        L.reed_cell_atoms.argtypes = [vp, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, _D, _I32]
        L.reed_forces.argtypes = [vp, C.c_int, C.c_double, C.c_double, _D, C.c_int, _D, _I32, _D, _D, _D, _D]
        L.reed_window_replay.argtypes = [vp, C.c_int, C.c_uint64, _D, C.c_int, _I32, C.c_int, _I32, _I32, _D]
        L.reed_run_static.argtypes = [C.POINTER(reed_lattice), C.POINTER(reed_species), C.c_int,
                                      C.POINTER(reed_potentials), C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_int64, C.c_uint64, C.POINTER(reed_run_opts), vp,
                                      C.POINTER(reed_stats_t)]
        _LIB = L
    return _LIB


def _check(rc, ctx=None):
    if rc < 0:
        raise ReedError(rc, lib().reed_last_error(ctx).decode())
    return rc


# ---- marshalling of workload dicts into the C structs ----------------------

def lattice_struct(w) -> reed_lattice:
    return reed_lattice(kind=LATTICE[w["lattice"]], window_n=int(w["n"]), frozen_margin=int(w["margin"]),
                        target=TARGET[w.get("target", "surface")], a=float(w["a"]), sigma=float(w["sigma"]))


def species_array(w):
    sp = w["species"]
    arr = (reed_species * len(sp))()
    for i, s in enumerate(sp):
        arr[i].Z, arr[i].M = s["Z"], s["M"]
    return arr


def potentials_struct(w) -> reed_potentials:
    p = reed_potentials()
    p.rc, p.r_taper = w["rc"], w["rt"]
    for i, c in enumerate(w["spline_c"]):
        p.spline_c[i] = c
    p.target_model = TT[w["tt"]]
    t = w["tersoff"]
    for i, k in enumerate(["A", "B", "lam1", "lam2", "beta", "n", "c", "d", "h", "R", "D"]):
        p.tersoff[i] = t[k]
    p.tersoff_blend[0], p.tersoff_blend[1] = w["blend"]
    b = w["buckingham"]
    for i in range(3):
        p.buck_A[i], p.buck_rho[i], p.buck_C[i] = b["A"][i], b["rho"][i], b["C"][i]
    p.buck_cut[0], p.buck_cut[1] = w["buck_cut"]
    p.buck_blend[0], p.buck_blend[1] = w["buck_blend"]
    p.s_e, p.s_loc, p.lam_loc = w["s_e"], w["s_loc"], w["lam_loc"]
    return p


def run_opts(w, precision=PREC_MIXED, first_id=0, threads=0, ctas_per_sm=0, record=True, record_capacity=0,
             trace_tracks=0, trace_steps=0, stream=None, adaptive=False, epoch_size=4096, n_initial=50,
             target_tracks=0, damage=True, adjoint=False, adj_segment=200, adj_every=20, nl_skin=0.0, nl_check=False,
             device_thresholds=False, thresholds=None, pool_poll_limit=0) -> reed_run_opts:
    o = reed_run_opts()
    o.dt_max_fs, o.dx_max, o.e_stop = w["dt_max_fs"], w["dx_max"], w["e_stop"]
    o.step_cap = int(w["step_cap"])
    o.beam_mode = BEAM[w["beam_mode"]]
    o.precision = precision
    thr = list(w["thresholds"] if thresholds is None else thresholds)
    o.n_thresholds = len(thr)
    for i, d in enumerate(thr):
        o.thresholds[i] = d
    o.n_bins, o.bin_width = int(w["n_bins"]), float(w["bin_w"])
    o.first_id = first_id
    o.threads_per_track, o.ctas_per_sm = threads, ctas_per_sm
    o.record_tracks = 1 if record else 0
    o.record_capacity = record_capacity
    o.trace_tracks, o.trace_steps = trace_tracks, trace_steps
    o.stream = stream
    o.adaptive = 1 if adaptive else 0
    o.device_thresholds = 1 if device_thresholds else 0
    o.epoch_size, o.n_initial, o.target_tracks = epoch_size, n_initial, target_tracks
    o.damage_n = int(w.get("damage_n", 0)) if damage else 0
    o.damage_voxel, o.damage_min = float(w.get("damage_voxel", 10.0)), float(w.get("damage_min", 0.1))
    o.adjoint, o.adj_segment, o.adj_every = (1 if adjoint else 0), adj_segment, adj_every
    o.nl_skin = nl_skin
    o.nl_check = 1 if nl_check else 0
    o.de_max = float(w.get("de_max", 0.0))
    o.dx_min = float(w.get("dx_min", 0.0))
    o.pool_poll_limit = pool_poll_limit
    return o


# ---- the C entry points ----------------------------------------------------

def reed_init(lattice: reed_lattice, species, n_species: int, potentials: reed_potentials) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(lib().reed_init(C.byref(ctx), C.byref(lattice), species, n_species, C.byref(potentials)))
    return ctx


def reed_run(ctx, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, n_ions, seed, opts=None):
    return _check(lib().reed_run(ctx, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, n_ions, seed,
                                 C.byref(opts) if opts is not None else None), ctx)


def reed_range_profile(ctx, n_bins):
    bins = np.zeros(n_bins)
    extra = np.zeros(3)
    _check(lib().reed_range_profile(ctx, bins.ctypes.data, n_bins, extra.ctypes.data), ctx)
    return bins, extra


def reed_stats(ctx) -> dict:
    s = reed_stats_t()
    _check(lib().reed_stats(ctx, C.byref(s)), ctx)
    return s.as_dict()


def reed_track_records(ctx, cap=None) -> np.ndarray:
    n = C.c_int64(0)
    _check(lib().reed_track_records(ctx, None, 0, C.byref(n)), ctx)
    m = n.value if cap is None else min(cap, n.value)
    out = np.zeros(m, dtype=RECORD_DTYPE)
    if m:
        _check(lib().reed_track_records(ctx, out.ctypes.data, m, C.byref(n)), ctx)
    return out


def reed_trace(ctx, n_tracks, n_steps):
    traj = np.zeros((n_tracks, n_steps, 8))
    anc = np.zeros((n_tracks, n_steps, 3), dtype=np.int32)
    _check(lib().reed_trace(ctx, traj.ctypes.data, anc.ctypes.data, n_tracks, n_steps), ctx)
    return traj, anc


def reed_thresholds(ctx, max_epochs=1024):
    """Cloning depths of each enhanced epoch of the last adaptive run."""
    n = C.c_int(0)
    _check(lib().reed_thresholds(ctx, None, 0, C.byref(n)), ctx)
    h = np.zeros((min(n.value, max_epochs), 16))
    if h.shape[0]:
        _check(lib().reed_thresholds(ctx, h.ctypes.data, h.shape[0], C.byref(n)), ctx)
    return h


def reed_damage_map(ctx, n):
    """(n, n, n) damage map (eV) and the energy deposited outside it."""
    out = np.zeros((n, n, n))
    ov = np.zeros(1)
    _check(lib().reed_damage_map(ctx, out.ctypes.data, n, ov.ctypes.data), ctx)
    return out, float(ov[0])


def reed_track_grads(ctx):
    """(n_records, 8) per-track dz/dtheta of adjoint runs."""
    n = C.c_int64(0)
    _check(lib().reed_track_grads(ctx, None, 0, C.byref(n)), ctx)
    out = np.zeros((n.value, 8))
    if n.value:
        _check(lib().reed_track_grads(ctx, out.ctypes.data, n.value, C.byref(n)), ctx)
    return out


def reed_kde_profile(ctx, sigma, n_bins, bin_width, out=None):
    """Kernel-density range profile (A^-1); out may be a device pointer."""
    if out is None:
        p = np.zeros(n_bins)
        _check(lib().reed_kde_profile(ctx, sigma, n_bins, bin_width, p.ctypes.data), ctx)
        return p
    _check(lib().reed_kde_profile(ctx, sigma, n_bins, bin_width, out), ctx)
    return None


def reed_grad(ctx, sigma, n_bins, bin_width, dL_dp_ptr):
    """dL/dtheta (8) for a profile cotangent at dL_dp_ptr (host or device)."""
    g = np.zeros(8)
    _check(lib().reed_grad(ctx, sigma, n_bins, bin_width, dL_dp_ptr, g.ctypes.data), ctx)
    return g


def reed_set_theta(ctx, theta):
    t = np.ascontiguousarray(theta, dtype=np.float64)
    assert t.size == 8
    _check(lib().reed_set_theta(ctx, t.ctypes.data_as(_D)), ctx)


def reed_update_thresholds(ctx, n_thresholds, hist_ptr=None, n_bins=0, bin_width=0.0, thresholds=None):
    """Set the device cloning depths: re-estimated from a range profile at
    hist_ptr (host or device address), or copied from `thresholds`."""
    t = None
    if thresholds is not None:
        t = np.ascontiguousarray(thresholds, dtype=np.float64)
    _check(lib().reed_update_thresholds(ctx, hist_ptr, n_bins, bin_width, n_thresholds,
                                        t.ctypes.data_as(_D) if t is not None else None), ctx)


def reed_get_thresholds(ctx):
    out = np.zeros(16)
    _check(lib().reed_get_thresholds(ctx, out.ctypes.data), ctx)
    return out


def reed_set_damage_feedback(ctx, dose_scale, e_crit, sigma_amorphous):
    _check(lib().reed_set_damage_feedback(ctx, dose_scale, e_crit, sigma_amorphous), ctx)


def reed_set_damage_map(ctx, damage_map, voxel):
    """damage_map: n^3 voxels + overflow (as reed_damage_map returns them),
    a flat array, an (n, n, n) array plus an overflow, or a device address."""
    if isinstance(damage_map, int):
        raise ValueError("give the voxel count with a device address: use lib().reed_set_damage_map")
    a = np.ascontiguousarray(damage_map, dtype=np.float64).ravel()
    n = int(round((a.size - 1) ** (1.0 / 3.0)))
    assert n ** 3 + 1 == a.size, "expected n^3 voxels and the overflow"
    _check(lib().reed_set_damage_map(ctx, a.ctypes.data, n, voxel), ctx)


def reed_peaks() -> dict:
    """Measured FP32/FP64/SFU/shared-memory throughput of the current GPU."""
    p = reed_peaks_t()
    _check(lib().reed_peaks(C.byref(p)), None)
    return {n: getattr(p, n) for n, _ in reed_peaks_t._fields_ if n != "reserved"}


def reed_reset(ctx):
    _check(lib().reed_reset(ctx), ctx)


def reed_last_error(ctx=None) -> str:
    return lib().reed_last_error(ctx).decode()


def reed_destroy(ctx):
    lib().reed_destroy(ctx)


def reed_philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(c)
    _check(lib().reed_philox(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32), c.shape[0]))
    return out


def reed_cell_atoms(ctx, key, ix, iy, iz):
    xyz = np.zeros((12, 3))
    sp = np.zeros(12, dtype=np.int32)
    n = _check(lib().reed_cell_atoms(ctx, key, ix, iy, iz, xyz.ctypes.data_as(_D), sp.ctypes.data_as(_I32)), ctx)
    return xyz[:n].copy(), sp[:n].copy()


def reed_forces(ctx, precision, ion_Z, ion_M, ion_x, xyz, sp):
    xi = np.ascontiguousarray(ion_x, dtype=np.float64)
    xa = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(sp, dtype=np.int32)
    fi = np.zeros(3)
    fa = np.zeros_like(xa)
    E, rho = C.c_double(), C.c_double()
    _check(lib().reed_forces(ctx, precision, ion_Z, ion_M, xi.ctypes.data_as(_D), xa.shape[0], xa.ctypes.data_as(_D),
                             s.ctypes.data_as(_I32), fi.ctypes.data_as(_D), fa.ctypes.data_as(_D), C.byref(E),
                             C.byref(rho)), ctx)
    return E.value, fi, fa, rho.value


def reed_window_replay(ctx, precision, key, path, cap=2000):
    p = np.ascontiguousarray(path, dtype=np.float64).reshape(-1, 3)
    anc = np.zeros((p.shape[0], 3), dtype=np.int32)
    cells = np.zeros((cap, 3), dtype=np.int32)
    bas = np.zeros(cap, dtype=np.int32)
    xyz = np.zeros((cap, 3))
    n = _check(lib().reed_window_replay(ctx, precision, key, p.ctypes.data_as(_D), p.shape[0],
                                        anc.ctypes.data_as(_I32), cap, cells.ctypes.data_as(_I32),
                                        bas.ctypes.data_as(_I32), xyz.ctypes.data_as(_D)), ctx)
    m = min(n, cap)
    return anc, cells[:m].copy(), bas[:m].copy(), xyz[:m].copy()


def reed_run_static(w, n_ions, seed, hist_out_ptr, precision=PREC_MIXED, stream=None, **kw):
    """Run without any device allocation (see include/reed.h): the workload
    dict describes target and run; hist_out_ptr is a device buffer of
    n_bins + 3 doubles owned by the caller.  Returns the stats dict."""
    sp = species_array(w)
    o = run_opts(w, precision=precision, record=False, stream=stream, damage=False, **kw)
    st = reed_stats_t()
    ion = w["ion"]
    _check(lib().reed_run_static(C.byref(lattice_struct(w)), sp, len(w["species"]), C.byref(potentials_struct(w)),
                                 ion["Z"], ion["M"], w["energy"], w["tilt"], w["rot"][0], w["rot"][1], n_ions, seed,
                                 C.byref(o), hist_out_ptr, C.byref(st)))
    return st.as_dict()


class Reed:
    """A context for one target workload (lattice, species, potentials)."""

    def __init__(self, w: dict):
        self.w = w
        self._sp = species_array(w)
        self.ctx = reed_init(lattice_struct(w), self._sp, len(w["species"]), potentials_struct(w))
        if float(w.get("e_crit", 0.0)) > 0.0:
            reed_set_damage_feedback(self.ctx, float(w.get("dose_scale", 0.0)), float(w["e_crit"]),
                                     float(w.get("sigma_amorphous", 0.0)))

    def run(self, n_ions=None, seed=None, precision=PREC_MIXED, tolerate=(), **kw):
        """Run primaries; error codes listed in `tolerate` (e.g. E_QUEUE_FULL)
        are returned instead of raised (the run completed, see stats())."""
        w = dict(self.w, step_cap=kw.pop("step_cap", self.w["step_cap"]))
        o = run_opts(w, precision=precision, **kw)
        ion = w["ion"]
        rc = lib().reed_run(self.ctx, ion["Z"], ion["M"], w["energy"], w["tilt"], w["rot"][0], w["rot"][1],
                            w["n_ions"] if n_ions is None else n_ions, w["seed"] if seed is None else seed,
                            C.byref(o))
        if rc < 0 and rc not in tolerate:
            _check(rc, self.ctx)
        return rc

    def profile(self):
        return reed_range_profile(self.ctx, int(self.w["n_bins"]))

    def stats(self):
        return reed_stats(self.ctx)

    def records(self):
        return reed_track_records(self.ctx)

    def trace(self, n_tracks, n_steps):
        return reed_trace(self.ctx, n_tracks, n_steps)

    def reset(self):
        reed_reset(self.ctx)

    def autotune(self, n_trial, seed=None, precision=PREC_MIXED, **kw):
        """Time the launch configurations on n_trial primaries and keep the
        fastest for later runs; returns [(threads, ctas_per_sm, ion-steps/s)]."""
        w = dict(self.w, step_cap=kw.pop("step_cap", self.w["step_cap"]))
        o = run_opts(w, precision=precision, **kw)
        ion = w["ion"]
        tab = (reed_tune_entry * 16)()
        n = C.c_int32(0)
        _check(lib().reed_autotune(self.ctx, ion["Z"], ion["M"], w["energy"], w["tilt"], w["rot"][0], w["rot"][1],
                                   n_trial, w["seed"] if seed is None else seed, C.byref(o), tab, 16, C.byref(n)),
               self.ctx)
        return [(tab[i].threads_per_track, tab[i].ctas_per_sm, tab[i].ion_steps_per_s) for i in range(n.value)]

    def thresholds(self):
        return reed_thresholds(self.ctx)

    def damage_map(self):
        return reed_damage_map(self.ctx, int(self.w["damage_n"]))

    def set_damage_map(self, damage_map, voxel=None):
        reed_set_damage_map(self.ctx, damage_map, float(self.w.get("damage_voxel", 10.0)) if voxel is None else voxel)

    def track_grads(self):
        return reed_track_grads(self.ctx)

    def set_theta(self, theta):
        reed_set_theta(self.ctx, theta)

    def forces(self, ion_x, xyz, sp, precision=PREC_MIXED):
        ion = self.w["ion"]
        return reed_forces(self.ctx, precision, ion["Z"], ion["M"], ion_x, xyz, sp)

    def cell_atoms(self, key, ix, iy, iz):
        return reed_cell_atoms(self.ctx, key, ix, iy, iz)

    def window_replay(self, key, path, precision=PREC_MIXED, cap=2000):
        return reed_window_replay(self.ctx, precision, key, path, cap)

    def close(self):
        if self.ctx:
            reed_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProfileFunction:
    """Differentiable kernel-density range profile, p(theta), theta = (s_e,
    s_loc, c_1..c_6) as a torch.autograd.Function: forward runs the tracks
    with the truncated-segment adjoint on and returns the profile (a float64
    CUDA tensor of n_bins); backward returns dL/dtheta from the per-track
    sensitivities (include/reed.h: reed_grad)."""

    @staticmethod
    def make(w, n_ions, seed, sigma, n_bins, bin_width, precision=PREC_MIXED):
        import torch

        ctx_holder = {}

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(fctx, theta):
                if "r" not in ctx_holder:
                    ctx_holder["r"] = Reed(w)
                r = ctx_holder["r"]
                fctx.theta_device = theta.device
                r.reset()
                r.set_theta(theta.detach().double().cpu().numpy())
                stream = torch.cuda.current_stream().cuda_stream or None
                r.run(n_ions=n_ions, seed=seed, precision=precision, adjoint=True, stream=stream)
                p = torch.empty(n_bins, dtype=torch.float64, device="cuda")
                reed_kde_profile(r.ctx, sigma, n_bins, bin_width, p.data_ptr())
                return p

            @staticmethod
            def backward(fctx, gp):
                r = ctx_holder["r"]
                gp = gp.detach().double().contiguous()
                g = reed_grad(r.ctx, sigma, n_bins, bin_width, gp.data_ptr())
                return torch.as_tensor(g, dtype=torch.float64, device=fctx.theta_device)

        return _Fn.apply, ctx_holder
