/*
 * reed.h -- C ABI of the GB300 REED-MD track stepper.
 *
 * REED-MD (Rare-Event-Enhanced Domain-following Molecular Dynamics) follows
 * many independent ion tracks through a crystal (Jeon & Gronbech-Jensen,
 * "Efficient Parallel Algorithm for Statistical Ion Track Simulations in
 * Crystalline Materials", Sec. 2).  Each track is a small molecular-dynamics
 * system: the ion plus an n^3-cell window of target atoms that moves with the
 * ion (cells behind it are dropped, statistically realised cells are created
 * ahead, Fig. "moving cell"); ion-target forces use the universal ZBL
 * screening; target-target forces are Tersoff (Si) or short-range pairs; the
 * ion feels electronic stopping; the integrator is velocity Verlet with an
 * adaptive step (Sec. 2, Fig. "dt_E").  Tracks are split at cloning depths
 * and carry weights 2^-k (Sec. 2, Fig. "split"); cloning depths are frozen
 * while a track runs (Sec. 3).  The paper's MPI host-client feedback (Sec.
 * 3) is replaced by device-resident tallies updated with atomics.
 *
 * Conventions (all entry points):
 *   - return an int status: REED_OK (0) or a negative REED_E_* code; the
 *     message of the last failure is available from reed_last_error();
 *   - pointers marked "host" must point to host memory; "host or device"
 *     accepts either (copies use cudaMemcpyDefault); output buffers are always
 *     owned by the caller and are written, never retained;
 *   - a reed_ctx owns all device memory it uses and is not thread-safe: use
 *     one context per host thread (and per stream);
 *   - units: Angstrom, eV, amu, femtoseconds where stated; angles in degrees.
 *
 * Nothing here allocates on the caller's behalf except reed_init (the
 * context) and reed_run (grows the context's buffers on first use).
 */
#ifndef REED_H
#define REED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define REED_OK 0
#define REED_E_ARG -1        /* an argument is out of range or inconsistent */
#define REED_E_CUDA -2       /* a CUDA runtime call failed */
#define REED_E_TIMEOUT -3    /* a bounded device-side wait expired */
#define REED_E_QUEUE_FULL -4 /* clone stack capacity exceeded (clones dropped) */
#define REED_E_NONFINITE -5  /* an ion state became NaN/Inf (track abandoned) */
#define REED_E_NOMEM -6      /* device memory allocation failed */
#define REED_E_SMEM -7       /* the window does not fit in shared memory */
#define REED_E_STATE -8      /* call made in the wrong state (e.g. no run yet) */
#define REED_E_NEIGHBOR -9   /* the run completed but some target forces were incomplete: an
                                atom had more list neighbours than its overflow row holds
                                (64 Tersoff, 192 pair), a track needed more than 32 overflow
                                rows at once, or a needed atom found no list row
                                (reed_stats: nb_overflow, bond_cap_overflow).  Every force of
                                the paper's model is evaluated otherwise (Sec. 1: all the
                                relevant interactions every time step). */

/* ---- enumerations ------------------------------------------------------ */
#define REED_LATTICE_DIAMOND 0   /* 8-atom cubic cell, one species (Si) */
#define REED_LATTICE_FLUORITE 1  /* 12-atom cubic cell: cation fcc + 8 anions (Sec. 2: UO2) */

#define REED_TT_NONE 0        /* target atoms feel only the ion */
#define REED_TT_TERSOFF 1     /* Tersoff bond order + ZBL blend (species 0) */
#define REED_TT_BUCKINGHAM 2  /* Buckingham pairs splined to ZBL */

#define REED_PREC_MIXED 0  /* FP32 forces/atoms, FP64 ion position, time, tallies */
#define REED_PREC_FP64 1   /* everything FP64 (plain path) */

#define REED_BEAM_FIXED 0  /* fixed tilt, rotation uniform in [rot_lo, rot_hi) */
#define REED_BEAM_CONE 1   /* direction uniform in solid angle within tilt of [001] */
#define REED_BEAM_RECOIL 2 /* bulk targets only: start on the lattice site at the
                              origin, direction uniform over the sphere (Sec. 4.1) */

#define REED_TARGET_SURFACE 0 /* target occupies z >= 0 with a (001) surface */
#define REED_TARGET_BULK 1    /* infinite crystal; the site of basis atom 0 of cell
                                 (0,0,0) is vacant (the recoil atom's own site) */

#define REED_TRACK_STOPPED 1        /* E < e_stop: tallied at its depth */
#define REED_TRACK_BACKSCATTERED 2  /* left through the surface (z < -rc, vz < 0) */
#define REED_TRACK_TRUNCATED 3      /* hit step_cap */
#define REED_TRACK_FAILED 4         /* non-finite state */

/* ---- configuration structs (plain data, copied by the library) -------- */

/* Target lattice and window (Sec. 2 "Second"; Fig. "moving cell").  A
 * SURFACE target occupies z >= 0 with a (001) surface; a BULK target fills
 * space and is run with REED_BEAM_RECOIL, the on-lattice recoils of the
 * paper's UO2 runs (Sec. 4.1, 4.2).  The window holds window_n^3 cells around
 * the ion's cell (odd n) or its nearest cell corner (even n).  With
 * target-target forces, frozen_margin outer cell layers are kept fixed (they
 * provide the environment of the integrated inner cells). */
typedef struct {
    int32_t kind;          /* REED_LATTICE_* */
    int32_t window_n;      /* cells per window edge, 2..6 */
    int32_t frozen_margin; /* 0 or 1 */
    int32_t target;        /* REED_TARGET_* */
    double a;              /* lattice constant, A (> 2 rc / (window_n - 1) advised) */
    double sigma;          /* thermal displacement RMS per Cartesian coordinate, A (Sec. 4.1) */
} reed_lattice;

/* A target species: diamond uses species 0; fluorite 0 = cation, 1 = anion. */
typedef struct {
    double Z;  /* atomic number */
    double M;  /* mass, amu */
} reed_species;

/* Interaction parameters.  Ion-target: ZBL universal potential (Sec. 2
 * "First") times exp(sum_i spline_c[i] B_i(ln r)) (cubic B-splines centred on
 * ln r = ln{0.2,0.35,0.6,1.0,1.7,3.0} A; all zero = pure ZBL), tapered to
 * zero between r_taper and rc with a C2 quintic.  Electronic stopping (Sec. 2
 * "Third"): drag F = -gamma (1 + s_loc (rho/rho0 - 1)) v inside the target,
 * gamma = s_e * Lindhard-Scharff, rho = sum over atoms of S(r) exp(-r/lam_loc). */
typedef struct {
    double rc, r_taper;          /* A */
    double spline_c[6];
    int32_t target_model;        /* REED_TT_* */
    int32_t reserved;
    double tersoff[11];          /* A B lam1 lam2 beta n c d h R D (PRB 38, 9902) */
    double tersoff_blend[2];     /* ZBL below [0], Tersoff above [1], A */
    double buck_A[3], buck_rho[3], buck_C[3];  /* pairs (0,0), (0,1), (1,1) */
    double buck_cut[2];          /* taper start, cutoff, A */
    double buck_blend[2];        /* ZBL below [0], Buckingham above [1], A */
    double s_e, s_loc, lam_loc;  /* stopping scale, local-density weight, density length (A) */
} reed_potentials;

/* Options of one reed_run call. */
typedef struct {
    double dt_max_fs;        /* upper bound of the step, fs (0.1) */
    double dx_max;           /* max step length of the fastest particle, A (0.05) */
    double e_stop;           /* a track stops when the ion's energy drops below, eV (5) */
    int64_t step_cap;        /* steps per track before truncation (2e6) */
    int32_t beam_mode;       /* REED_BEAM_* */
    int32_t precision;       /* REED_PREC_* */
    int32_t n_thresholds;    /* cloning depths in use, 0..16 (0 = no rare-event enhancement) */
    int32_t n_bins;          /* range histogram bins (fixed by the first run after init/reset) */
    double thresholds[16];   /* ascending cloning depths d_1..d_k, A */
    double bin_width;        /* A (fixed by the first run after init/reset) */
    int64_t first_id;        /* id of the first primary of this run (ids are the RNG streams) */
    int32_t threads_per_track; /* 0 = tuned or default, else 32/64/128/256 (512: pair-list model) */
    int32_t ctas_per_sm;       /* 0 = autotune / maximum occupancy */
    int32_t record_tracks;     /* 1: keep one reed_track_record per finished track */
    int32_t trace_tracks;      /* record the first trace_steps steps of primaries */
    int32_t trace_steps;       /*   first_id .. first_id + trace_tracks - 1 */
    int32_t reserved;
    int64_t record_capacity;   /* records kept (further tracks are counted only); fixed by the
                                  first run that keeps records after init/reset (0 = n_ions x
                                  (1 + 4 n_thresholds) + 1024 of that run) */
    void* stream;              /* cudaStream_t to run on; NULL = default stream */
    /* Adaptive cloning depths (Sec. 2; re-estimated from finished ions, Sec. 3):
     * with adaptive = 1 the first n_initial primaries run without enhancement,
     * then the run proceeds in epochs of epoch_size primaries; before each
     * epoch the n_thresholds depths are re-estimated on the device as
     * d_k = S^-1(2^-k), S(d) = weighted fraction of finished tracks stopped at
     * depth >= d (linear interpolation in the range histogram; +inf when the
     * target lies beyond it).  With n_initial = 0 the first epoch uses
     * thresholds[] as the initial guess.  A track never sees its depths change. */
    int32_t adaptive;
    /* 1: a non-adaptive run takes its n_thresholds cloning depths from the
     * context's device copy set by reed_update_thresholds (thresholds[] is
     * ignored); the multi-process form of the epoch update. */
    int32_t device_thresholds;
    int64_t epoch_size;        /* primaries per epoch (adaptive) */
    int64_t n_initial;         /* unenhanced primaries before the first epoch (adaptive) */
    /* Stop handing out primaries once this many tracks (clones included) have
     * finished; tracks already running are completed (the paper's kill
     * signal, Sec. 3).  0 = run all n_ions. */
    int64_t target_tracks;
    /* Cumulative damage (the paper's shared damage information, Sec. 1, 3):
     * an atom leaving the simulation -- its cell dropped behind the ion, or the
     * track finished -- deposits weight x kinetic energy, when above
     * damage_min, into a damage_n^3 grid of damage_voxel cubes with origin
     * (-damage_n damage_voxel / 2, same, 0).  damage_n = 0: no map. */
    int32_t damage_n;
    int32_t reserved3;
    double damage_voxel;       /* A */
    double damage_min;         /* eV */
    /* Truncated-segment sensitivities (target model NONE, frozen_margin 0,
     * no cloning, records on): for every stopped track, dz_T/dtheta for theta = (s_e, s_loc,
     * spline_c[0..5]) through its last adj_segment steps (the state
     * adj_segment..adj_segment+adj_every-1 steps before the end held fixed),
     * with dt, window moves and the drag's on/off frozen; checkpoints every
     * adj_every steps (defaults 200 and 20). */
    int32_t adjoint;
    int32_t adj_segment;
    int32_t adj_every;
    /* Self-check of the target neighbour lists (slow; for tests): after
     * every build and refresh each list is compared with a brute-force
     * search over the window; differences are counted in nl_check_errors. */
    int32_t nl_check;
    /* Target neighbour lists (Tersoff, Buckingham): list radius = cutoff +
     * nl_skin; the lists are rebuilt after a window move and when the two
     * longest atom paths since their last list add up to more than nl_skin
     * (Tersoff: then only the lists of atoms whose path exceeds nl_skin / 4
     * are recomputed, and the entries of the others that involve them).
     * 0 = 0.3 A for Tersoff and for the pair lists. */
    double nl_skin;
    /* Energy term of the adaptive step (the paper's step rule in terms of the
     * kinetic and collisional energy, Sec. 2): when > 0, also
     * dt <= de_max / P with P the largest |F . v| over the ion and the
     * integrated atoms at the start of the step (conservative forces), i.e. no
     * particle's kinetic energy changes by much more than de_max (eV) in one
     * step -- but never so that the fastest particle moves less than dx_min
     * in the step.  0 = off. */
    double de_max;
    /* Polls of the shared clone pool by a CTA that ran out of work before it
     * gives up and the run returns REED_E_TIMEOUT (each poll sleeps about
     * 0.5-4 us); 0 = 2^26, about five minutes. */
    int64_t pool_poll_limit;
    /* Shortest step of the fastest particle that the energy term may impose,
     * A: below a few ulp of a single-precision window coordinate (~1e-6 A) a
     * step moves nothing and a collision stalls.  0 = 1e-4 A. */
    double dx_min;
} reed_run_opts;

/* Per-track result: the depth and weight of one finished track (Sec. 3, result messages). */
typedef struct {
    uint64_t id;        /* track id (primaries: first_id + i; clones: hashed) */
    uint64_t primary;   /* id of the primary whose lineage it belongs to */
    double z;           /* depth at the end of the track, A (BULK: distance from the start) */
    double t;           /* simulated time, tau (1 tau = 10.1805 fs) */
    int64_t steps;      /* integration steps of the track's history (a clone counts its
                           parent's steps before the split; step_cap applies to this) */
    int32_t level;      /* cloning levels passed: weight = 2^-level */
    int32_t status;     /* REED_TRACK_* */
} reed_track_record;

typedef struct {
    int64_t primaries, clones, tracks, steps;  /* tracks = finished tracks (primaries + clones) */
    int64_t pair_evals;      /* ion-target pairs inside rc */
    int64_t bond_evals;      /* target-target pair or bond terms evaluated */
    int64_t shifts;          /* window moves */
    int64_t rebuilds;        /* neighbour-list builds */
    int64_t stopped, backscattered, truncated, failed;
    int64_t dropped_clones;  /* clones lost to a full stack */
    int64_t nb_overflow;     /* neighbour-list entries that found no room (REED_E_NEIGHBOR) */
    int64_t bond_cap_overflow; /* needed atoms left without a list row (REED_E_NEIGHBOR) */
    int64_t triplets;        /* Tersoff bond-angle (zeta) terms evaluated */
    int64_t atom_updates;    /* integrated target-atom updates (atoms x steps) */
    int64_t phase_cycles[6]; /* SM clock cycles per step phase, summed over CTAs: ion update,
                                atom move, neighbour build, Tersoff pass 1, forces, track admin */
    double w_stopped, w_back, w_trunc;   /* weights */
    double kernel_ms;        /* device time of the last reed_run */
    int32_t threads_per_track, ctas_per_sm, grid, smem_bytes;  /* last launch */
    int64_t splits[16];      /* clones made on first passing cloning depth k+1 (the
                                paper's per-depth split statistics, Sec. 3) */
    int64_t pooled;          /* clones run by another CTA than the one that made them
                                (taken from the shared clone pool) */
    int64_t nb_spilled;      /* lists that outgrew their shared-memory row and moved whole
                                to an overflow row in global memory (exact, only slower) */
    int64_t list_refreshes;  /* Tersoff partial list refreshes (only the lists of atoms that
                                moved more than a quarter of the skin recomputed) */
    int64_t nl_check_errors; /* with opt->nl_check: list entries that differ from a
                                brute-force search (0 when the lists are exact) */
    int64_t centre_class[4]; /* Tersoff centre evaluations per step, summed over steps, by
                                list length: at most 4 neighbours (one thread per centre),
                                5-8, 9-16 and more (8, 16 or 32 lanes per centre) */
} reed_stats_t;

typedef struct reed_ctx reed_ctx;

/* Create a context for one target (lattice, species, potentials) -- the
 * crystal, its statistically realised cells and the interactions of Sec. 2
 * ("First": ion-target ZBL; "Second": the moving window of unit cells;
 * "Third": electronic stopping) and the target-target forces of Sec. 1.
 * *out receives the context; free it with reed_destroy.  n_species must be
 * 1 for DIAMOND and 2 for FLUORITE.  Selects the current CUDA device.
 * Errors: REED_E_ARG (invalid parameters), REED_E_CUDA, REED_E_NOMEM. */
int reed_init(reed_ctx** out, const reed_lattice* lat, const reed_species* sp, int n_species,
              const reed_potentials* pot);

/* Run n_ions primary tracks (ids opt->first_id ...) of an ion (Z, M amu) at
 * energy_eV launched at z = -rc with lateral position uniform in the (0,0)
 * surface cell and direction from tilt_deg and rotation U[rot_deg_lo,
 * rot_deg_hi) (or a cone of half-angle tilt_deg), Sec. 2 -- or, on a BULK
 * target with REED_BEAM_RECOIL, from the lattice site at the origin in a
 * direction uniform over the sphere (the angles are then ignored), its depth
 * being the distance from that site.  Every primary is
 * followed, with all its clones, until it stops, leaves through the surface
 * or reaches step_cap; results accumulate into the context's tallies until
 * reed_reset.  seed selects the random streams (Philox4x32-10 keyed by seed
 * and track id).  Blocks until the run is finished.  opt may be NULL (all
 * defaults: 0.1 fs, 0.05 A, 5 eV, 2e6 steps, mixed precision, no cloning,
 * 100 bins of 10 A).  With record_tracks and record_capacity 0 the record
 * buffer holds n_ions * (1 + 4 n_thresholds) + 1024 records.
 * Clones are run depth first by the CTA that made them, or, while some CTA
 * is out of work, donated to a shared pool that idle CTAs take from (the
 * paper's host handing returned clones to free clients, Sec. 3).
 * Returns REED_OK or an error:
 * REED_E_NEIGHBOR (completed, but some target forces were incomplete), REED_E_ARG (also a RECOIL beam on a SURFACE target or the reverse, or the
 * adjoint on a BULK target), REED_E_SMEM, REED_E_CUDA, REED_E_NOMEM; REED_E_QUEUE_FULL and
 * REED_E_NONFINITE mean the run completed but clones or tracks were lost
 * (counted in reed_stats); REED_E_TIMEOUT means a CTA out of work stopped
 * polling the clone pool after opt->pool_poll_limit polls (donated clones may
 * be missing). */
int reed_run(reed_ctx* ctx, double ion_Z, double ion_M, double energy_eV, double tilt_deg,
             double rot_deg_lo, double rot_deg_hi, int64_t n_ions, uint64_t seed,
             const reed_run_opts* opt);

/* Weighted range profile (Sec. 2): bins_out[n_bins] (host or device, FP64)
 * receives sum of weights 2^-level of stopped tracks per depth bin
 * [b*w, (b+1)*w) (depth = z, or on a BULK target the distance from the
 * start; cloning depths use the same coordinate); extra3 (host or device, may be NULL) receives
 * {stopped above the surface, stopped beyond the last bin, backscattered}.
 * n_bins must equal the tally's bin count.  Errors: REED_E_STATE (no run),
 * REED_E_ARG. */
int reed_range_profile(reed_ctx* ctx, double* bins_out, int n_bins, double* extra3);

/* Truncated-segment sensitivities of the range profile for fitting model
 * parameters to measured profiles (the paper notes REED-MD profiles match
 * measurements with minimal empirical fitting of model parameters, Sec. 1;
 * it computes no sensitivities itself).  theta = (s_e, s_loc,
 * spline_c[0..5]) as in reed_potentials.
 *
 * Per-track dz_T/dtheta (8 doubles per record, in record order; zero for
 * tracks that did not stop) of adjoint runs (opt->adjoint): out (host or
 * device, may be NULL to query the count) receives up to cap rows; *n_out
 * (host) the number of rows kept.  REED_E_STATE if no adjoint run since
 * init/reset, REED_E_ARG on a null n_out or a negative cap. */
int reed_track_grads(reed_ctx* ctx, double* out, int64_t cap, int64_t* n_out);

/* Kernel-density range profile of the stopped tracks recorded since
 * init/reset: p[b] = sum_i w_i N(z_b; z_i, sigma) / sum_i w_i at bin centres
 * z_b = (b + 1/2) bin_width (A^-1, w_i = 2^-level); p_out host or device,
 * n_bins doubles.  Needs records (opt->record_tracks): REED_E_STATE without,
 * REED_E_ARG for sigma or bin_width <= 0 or n_bins < 1.  Sums in record
 * order, so two runs agree to rounding, not bit for bit. */
int reed_kde_profile(reed_ctx* ctx, double sigma, int n_bins, double bin_width, double* p_out);

/* Gradient of a loss of that profile: dL_dtheta[8] (host or device) =
 * sum_i (sum_b dL_dp[b] dp_b/dz_i) dz_i/dtheta, from the per-track
 * sensitivities of an adjoint run (the weights and sum_i w_i do not depend
 * on theta); dL_dp host or device, n_bins doubles.  REED_E_STATE if no
 * adjoint run since init/reset, REED_E_ARG as for reed_kde_profile. */
int reed_grad(reed_ctx* ctx, double sigma, int n_bins, double bin_width, const double* dL_dp, double* dL_dtheta);

/* Set theta = (s_e, s_loc, spline_c[0..5]) of the context's potentials for
 * later runs (host, 8 doubles).  REED_E_ARG on a null pointer. */
int reed_set_theta(reed_ctx* ctx, const double* theta8);

/* Cumulative damage map of all runs since init/reset -- the shared damage
 * information the paper's tracks feed back (Sec. 1, Sec. 3: the host keeps
 * the accumulated damage and hands it to new tracks; here a device-resident
 * FP64 map updated with atomics): out (host or device)
 * receives n^3 doubles (eV, index (ix n + iy) n + iz; voxel (0,0,0) starts
 * at (-n v / 2, -n v / 2, 0), on a BULK target at (-n v / 2) in all three),
 * overflow (may be NULL) the energy deposited outside the grid.  n must
 * equal damage_n. */
int reed_damage_map(reed_ctx* ctx, double* out, int n, double* overflow);

/* Counters of all runs since init/reset (host pointer): tracks, steps, the
 * per-depth split statistics of Sec. 3 (splits[]), and the work and phase
 * clocks that stand in for the computation and communication loads the
 * paper measures per client in Sec. 4 (Tables 3-4). */
int reed_stats(reed_ctx* ctx, reed_stats_t* out);

/* Copy up to cap per-track records (host or device) of all runs since
 * init/reset; *n_out (host) receives the number of records kept. */
int reed_track_records(reed_ctx* ctx, reed_track_record* out, int64_t cap, int64_t* n_out);

/* Copy the trajectory trace of the last run (opt->trace_tracks x
 * opt->trace_steps): traj (host or device) gets 8 doubles per step
 * (x y z t vx vy vz dt; steps after a track ended are zero), anchors (host or
 * device, may be NULL) 3 int32 window anchor indices per step. */
int reed_trace(reed_ctx* ctx, double* traj, int32_t* anchors, int n_tracks, int n_steps);

/* Cloning depths used by the enhanced epochs of the last adaptive run (the
 * evolution of cloning points, Sec. 4.1): history (host or device) receives up
 * to max_epochs rows of 16 doubles (first n_thresholds valid, +inf = no
 * depth); *n_epochs (host) the number of enhanced epochs run. */
int reed_thresholds(reed_ctx* ctx, double* history, int max_epochs, int* n_epochs);

/* Set the context's device copy of the cloning depths, read by runs with
 * opt->device_thresholds = 1.  With hist != NULL (host or device, n_bins + 3
 * FP64 in the reed_range_profile layout, e.g. the sum of several processes'
 * range profiles) the first n_thresholds depths are re-estimated from it on
 * the device exactly as an adaptive run does between epochs (d_k = S^-1(2^-k),
 * Sec. 2 and the feedback of Sec. 3; an empty histogram leaves them as they
 * are); else they are copied from thresholds (host, n_thresholds values).
 * n_bins must be the context's bin count; 1 <= n_thresholds <= 16.  Returns
 * REED_E_ARG on a bad size, REED_E_CUDA on a device error.  Synchronous. */
int reed_update_thresholds(reed_ctx* ctx, const double* hist, int n_bins, double bin_width, int n_thresholds,
                           const double* thresholds);

/* The current device copy of the cloning depths (host or device out, 16
 * doubles). */
int reed_get_thresholds(reed_ctx* ctx, double* out16);

/* Launch-configuration autotuner (the batching form's tuning): runs
 * n_trial primaries of the given beam (ids from 2^40 up, so no primary of a
 * real run is repeated) once per candidate -- threads_per_track in {32, 64,
 * 128, 256, and 512 where the model allows it} and, for each, CTAs per SM
 * at the occupancy maximum, three quarters and half of it -- and keeps the
 * fastest (ion-steps per second of
 * kernel time) for later runs of this context whose opt->threads_per_track
 * and opt->ctas_per_sm are 0 and whose precision and adjoint flag match opt.
 * The trials run in a private context, so this context's tallies are not
 * touched; records, traces, damage and cloning are off in them, and
 * opt->step_cap bounds each trial track.  table (host, may be NULL) receives up
 * to cap timed candidates, *n_out (host, may be NULL) their number. */
typedef struct {
    int32_t threads_per_track, ctas_per_sm;
    double ion_steps_per_s;
} reed_tune_entry;

int reed_autotune(reed_ctx* ctx, double ion_Z, double ion_M, double energy_eV, double tilt_deg, double rot_deg_lo,
                  double rot_deg_hi, int64_t n_trial, uint64_t seed, const reed_run_opts* opt, reed_tune_entry* table,
                  int cap, int* n_out);

/* Damage feedback (a reading of the paper's cumulative damage information
 * fed back to the tracks, Sec. 1 and 3; the mechanism is not given there):
 * while e_crit > 0 and the context holds a damage map, a newly created cell
 * is amorphous with probability 1 - exp(-e / e_crit), where e = dose_scale *
 * D / N is the energy deposited per target atom in the map voxel D that
 * holds the cell's centre (N = lattice atoms per voxel, dose_scale = physical
 * ions each simulated primary stands for); an amorphous cell's atoms get
 * Gaussian offsets of sigma_amorphous (A) instead of the lattice's sigma.
 * The decision uses its own Philox block of the cell (tag 3).  Each launch
 * reads the map as it stood when the launch started (epochs of an adaptive
 * run see the damage of the epochs before them), so results do not depend on
 * timing.  e_crit = 0 turns it off.  REED_E_ARG on negative values. */
int reed_set_damage_feedback(reed_ctx* ctx, double dose_scale, double e_crit, double sigma_amorphous);

/* Replace the context's cumulative damage map: map (host or device) holds
 * n^3 voxels of voxel A ([ix][iy][iz], x and y centred on the entry cell, z
 * from the surface; on a BULK target all three centred on the start) and the overflow, as reed_damage_map returns it, e.g. the
 * sum of several processes' maps.  Later runs must use the same n and voxel.
 * REED_E_ARG for n outside 1..512 or voxel <= 0. */
int reed_set_damage_map(reed_ctx* ctx, const double* map, int n, double voxel);

/* Measured throughput of the units that bound the track stepper, on the
 * current device (microbenchmarks of independent instruction streams, a few
 * tenths of a second in all): FP32 and FP64 FMA, the SFU's ex2 and rsqrt,
 * 128-bit shared-memory loads, and the SM clock seen while they ran.  The
 * denominators of the stepper's roofline (no paper counterpart). */
typedef struct {
    double fp32_tflops, fp64_tflops;   /* FMA = 2 FLOP */
    double ex2_gops, rsqrt_gops;       /* SFU results per second (1e9) */
    double smem_tbs;                   /* shared-memory load bandwidth, TB/s */
    double sm_mhz;                     /* clock64 cycles per second during the run */
    int32_t sms, reserved;
} reed_peaks_t;

int reed_peaks(reed_peaks_t* out);

/* Zero all tallies, records and counters; drop the damage map and the
 * sensitivities (cloning depths, damage-feedback settings and autotuned
 * launch shapes are kept). */
int reed_reset(reed_ctx* ctx);

/* Message of the last failure of this context (ctx == NULL: of the last
 * failed reed_init or reed_run_static on this thread).  Never NULL.  The
 * paper has no counterpart (error reporting of this interface). */
const char* reed_last_error(reed_ctx* ctx);

/* Free the context and every device buffer it owns (NULL is ignored).  The
 * paper has no counterpart (resource management of this interface). */
void reed_destroy(reed_ctx* ctx);

/* ---- diagnostics: the stepper's own device functions on given inputs --- */

/* Philox4x32-10 (Salmon et al., SC'11) on the device: n blocks; ctr 4n,
 * key 2n, out 4n uint32 (host pointers). */
int reed_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);

/* Atoms of absolute cell (ix,iy,iz) as the stepper creates them for a track
 * with Philox key `key` (Sec. 2, Sec. 4.1): xyz_out (host, 3*12 doubles,
 * absolute coordinates), species_out (host, 12 int32).  Returns the atom count
 * (0 above the surface; on a BULK target cell (0,0,0) lacks basis atom 0) or
 * a negative status. */
int reed_cell_atoms(reed_ctx* ctx, uint64_t key, int32_t ix, int32_t iy, int32_t iz,
                    double* xyz_out, int32_t* species_out);

/* Conservative forces of one configuration computed by the stepper's force
 * pass in `precision` (REED_PREC_*): ion at ion_x (host, 3 doubles, ion
 * (Z, M) as given), n atoms at xyz (host, 3n, absolute) with species sp
 * (host, n).  Outputs (host): f_ion[3], f_atoms[3n], energy[1] (potential
 * energy; may be NULL), rho[1] (local density at the ion; may be NULL).
 * n <= the window size of the context's lattice. */
int reed_forces(reed_ctx* ctx, int precision, double ion_Z, double ion_M, const double* ion_x, int n,
                const double* xyz, const int32_t* sp, double* f_ion, double* f_atoms, double* energy,
                double* rho);

/* Drive the window logic along a prescribed ion path (host, 3*npts doubles):
 * anchors_out (host, 3*npts int32) gets the window anchor after each point;
 * at the end the window's atoms are written (host; cells_out 3*cap int32
 * absolute home cells, basis_out cap int32, xyz_out 3*cap doubles absolute).
 * Returns the number of atoms in the final window or a negative status. */
int reed_window_replay(reed_ctx* ctx, int precision, uint64_t key, const double* path, int npts,
                       int32_t* anchors_out, int cap, int32_t* cells_out, int32_t* basis_out,
                       double* xyz_out);

/* ---- a run that allocates no device memory ---------------------------- */

/* reed_run_static: the same track run as reed_run, for callers that cannot
 * allocate device memory -- for example a host that hands all GPU memory to
 * its own pool allocator and treats any other cudaMalloc as an error, or a
 * latency-critical loop that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; it
 * is an interface convenience.
 *
 * No context is needed: the target is described by lat, sp, n_species, pot
 * (as for reed_init) and the run by the remaining arguments (as for
 * reed_run).  The launch's scratch (counters, primary queue, status word,
 * clone stacks, neighbour-list overflow rows) lives in one file-scope device
 * array of 64 MiB that every GPU loading the library holds until the process
 * exits.  The array's device address belongs to a CUDA context: the first
 * call in each context of a device looks it up (cudaGetSymbolAddress) and
 * caches it under the context's unique id.  Configurations whose scratch
 * does not fit (SMs x (n_thresholds x window record + overflow rows)) are
 * rejected with REED_E_ARG; the launch uses fewer CTAs per SM when that
 * makes it fit.  No
 * per-track records or traces (record_tracks, trace_tracks, trace_steps
 * must be 0).
 *
 * hist_out (device, n_bins + 3 doubles) is overwritten with the weighted
 * range profile followed by {above the surface, beyond the last bin,
 * backscattered}; stats_out (host, may be NULL) receives the counters.
 * Every call shares the one scratch array and clears it first, so calls
 * whose work overlaps on the GPU (from several host threads or streams)
 * race.  Blocks until the run is finished: it synchronises opt->stream and
 * reads the counters back before returning.  Returns as reed_run;
 * reed_last_error(NULL) has the message. */
int reed_run_static(const reed_lattice* lat, const reed_species* sp, int n_species, const reed_potentials* pot,
                    double ion_Z, double ion_M, double energy_eV, double tilt_deg, double rot_deg_lo,
                    double rot_deg_hi, int64_t n_ions, uint64_t seed, const reed_run_opts* opt, double* hist_out,
                    reed_stats_t* stats_out);

#ifdef __cplusplus
}
#endif

#endif /* REED_H */
