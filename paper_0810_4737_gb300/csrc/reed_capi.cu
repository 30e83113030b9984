// reed_capi.cu -- host implementation of the C ABI declared in include/reed.h.
//
// A context holds the target description and all device buffers (tallies,
// records, clone stacks).  reed_run turns the user's description into the
// device parameter block (every derived constant is computed here in FP64),
// sizes the persistent launch to the GPU (CTAs per SM from the occupancy of
// the window in shared memory, grid = SMs x CTAs/SM) and runs it on the
// caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <math_constants.h>

#include "reed.h"
#include "reed_internal.h"

namespace {

thread_local std::string g_init_error = "no error";

// Lattice bases in units of a (diamond cubic; fluorite = cation fcc + the 8
// tetrahedral anion sites).
const double kDiamond[8][3] = {{0, 0, 0}, {0, .5, .5}, {.5, 0, .5}, {.5, .5, 0},
                               {.25, .25, .25}, {.25, .75, .75}, {.75, .25, .75}, {.75, .75, .25}};
// Fluorite: cations on the fcc sites, anions on the eight (1/4,1/4,1/4)-type
// sites.  The basis index keys the thermal-displacement stream, so this
// order is part of the stream definition.
const double kFluorite[12][3] = {{0, 0, 0},       {0, .5, .5},     {.5, 0, .5},     {.5, .5, 0},
                                 {.25, .25, .25}, {.75, .25, .25}, {.25, .75, .25}, {.25, .25, .75},
                                 {.75, .75, .25}, {.75, .25, .75}, {.25, .75, .75}, {.75, .75, .75}};

// ZBL-correction knot radii (A); B-splines are centred on ln r of each.
const double kKnots[6] = {0.2, 0.35, 0.6, 1.0, 1.7, 3.0};

// default neighbour-list skins, A (measured on the As 10 keV Tersoff batch
// with partial refreshes: 0.2 / 0.25 / 0.3 A give 15.7 / 16.3 / 16.3 M
// ion-steps/s; the CeO2 pair lists are best at 0.3)
const double kSkinTersoff = 0.3;
const double kSkinPairs = 0.3;
#define REED_NTHETA_HOST 8
#define REED_STEP_RING_HOST 256

double screen_inv(double Z1, double Z2) { return (std::pow(Z1, 0.23) + std::pow(Z2, 0.23)) / (0.8854 * REED_BOHR); }

}  // namespace

struct reed_ctx {
    int device = 0, sms = 0;
    size_t smem_optin = 0;
    reed_lattice lat{};
    reed_species sp[2]{};
    int nspec = 0;
    reed_potentials pot{};
    // tallies
    int nbins = 0;
    double bin_w = 0.0;
    double* d_hist = nullptr;
    unsigned long long* d_counters = nullptr;
    unsigned long long* d_splits = nullptr;   // clones per cloning level
    double* d_wsum = nullptr;
    unsigned long long* d_next = nullptr;
    int* d_status = nullptr;
    // records
    reed_track_record* d_records = nullptr;
    unsigned long long* d_rec_count = nullptr;
    long long rec_cap = 0;
    // trace
    double* d_trace = nullptr;
    int* d_trace_anchor = nullptr;
    int trace_tracks = 0, trace_steps = 0;
    // clone stacks
    unsigned char* d_stacks = nullptr;
    size_t stacks_bytes = 0;
    // neighbour-list overflow rows (per CTA)
    unsigned char* d_spill = nullptr;
    size_t spill_bytes = 0;
    // shared clone pool: records, slot states and its two counters
    unsigned char* d_pool = nullptr;
    size_t pool_bytes = 0;
    unsigned* d_pool_state = nullptr;   // pool slots + 3 control words
    int pool_state_cap = 0;
    // scratch for diagnostics
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // truncated-segment sensitivities
    double* d_grads = nullptr;
    long long grads_cap = 0;
    unsigned char* d_adj = nullptr;
    size_t adj_bytes = 0;
    double* d_kde = nullptr;       // scratch for the profile / gradient kernels
    size_t kde_bytes = 0;
    // cumulative damage map (fixed by the first run that asks for it)
    double* d_damage = nullptr;
    int dn = 0;
    double dvox = 0.0;
    // adaptive cloning depths: current set and per-epoch history
    double* d_thr = nullptr;
    double* d_thr_hist = nullptr;
    int thr_hist_cap = 0, thr_epochs = 0;
    unsigned long long* d_finished = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    // damage feedback settings (e_crit <= 0: off) and the per-launch snapshot
    double fb_dose = 0.0, fb_ec = 0.0, fb_sam = 0.0;
    double* d_dsnap = nullptr;
    size_t dsnap_bytes = 0;
    // autotuned launch configuration per [precision][adjoint] (0 = none)
    int tuned_threads[2][2] = {{0, 0}, {0, 0}};
    int tuned_ctas[2][2] = {{0, 0}, {0, 0}};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;
    LaunchCfg last_cfg{};
    std::string err = "no error";
};

namespace {

int fail(reed_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_init_error = buf;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? REED_E_NOMEM : REED_E_CUDA,         \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);      \
    } while (0)

double lindhard_gamma_unit(const reed_ctx* ctx, double Z1, double M1);

template <typename T> void fill_hot(HotParams<T>& h, const DevParams& P, const reed_ctx* ctx, double skin)
{
    const reed_potentials& q = ctx->pot;
    h.a = (T)P.a;
    for (int s = 0; s < 2; ++s) {
        h.invM2[s] = (T)P.invM2[s];
        h.zk[s] = (T)P.zk[s];
        h.zia[s] = (T)P.zia[s];
    }
    h.rc2 = (T)(P.rc * P.rc);
    h.rt = (T)P.rt;
    h.inv_tw = (T)P.inv_tw;
    h.lam_inv = (T)P.lam_inv;
    for (int i = 0; i < 6; ++i) {
        h.spline_c[i] = (T)P.spline_c[i];
        h.spline_ctr[i] = (T)P.spline_ctr[i];
    }
    h.spline_invh = (T)P.spline_invh;
    // Tersoff
    const double* t = q.tersoff;
    const double A = t[0], B = t[1], l1 = t[2], l2 = t[3], beta = t[4], n = t[5], c = t[6], d = t[7], hh = t[8],
                 R = t[9], D = t[10];
    h.tA = (T)A;
    h.tB = (T)B;
    h.tl1 = (T)l1;
    h.tl2 = (T)l2;
    h.tbn = (T)(n > 0 ? std::pow(beta, n) : 0.0);
    h.tn = (T)n;
    h.tmhn = (T)(n > 0 ? -0.5 / n : 0.0);
    h.tc2 = (T)(c * c);
    h.td2 = (T)(d * d);
    h.th = (T)hh;
    h.tR = (T)R;
    h.tRmD = (T)(R - D);
    h.tcut = (T)(R + D);
    h.tq = (T)(D > 0 ? 0.5 * REED_PI / D : 0.0);
    h.tdq = (T)(D > 0 ? -0.25 * REED_PI / D : 0.0);
    h.tc2d2 = (T)(d != 0 ? c * c / (d * d) : 0.0);
    h.t_blo = (T)q.tersoff_blend[0];
    h.t_binvw = (T)(1.0 / std::max(1e-12, q.tersoff_blend[1] - q.tersoff_blend[0]));
    h.t_zk = (T)(P.Z2[0] * P.Z2[0] * REED_E2);
    h.t_zia = (T)screen_inv(P.Z2[0], P.Z2[0]);
    double cut = P.tt == REED_TT_BUCKINGHAM ? q.buck_cut[1] : R + D;
    h.rlist2 = (T)((cut + skin) * (cut + skin));
    h.skin = (T)skin;
    h.de_max = (T)P.de_max;
    h.dx_min = (T)P.dx_min;
    h.g_lo = (T)(-P.half_n * P.a);
    h.g_inv = (T)(P.g_nb / (P.n * P.a));
    // Buckingham
    for (int p = 0; p < 3; ++p) {
        h.bA[p] = (T)q.buck_A[p];
        h.brho_inv[p] = (T)(q.buck_rho[p] > 0 ? 1.0 / q.buck_rho[p] : 0.0);
        h.bC[p] = (T)q.buck_C[p];
        int si = p == 2 ? 1 : 0, sj = p == 0 ? 0 : 1;
        if (ctx->nspec < 2) si = sj = 0;
        h.b_zk[p] = (T)(ctx->sp[si].Z * ctx->sp[sj].Z * REED_E2);
        h.b_zia[p] = (T)screen_inv(ctx->sp[si].Z, ctx->sp[sj].Z);
    }
    h.b_lo = (T)q.buck_blend[0];
    h.b_binvw = (T)(1.0 / std::max(1e-12, q.buck_blend[1] - q.buck_blend[0]));
    h.b_rt = (T)q.buck_cut[0];
    h.b_rinvw = (T)(1.0 / std::max(1e-12, q.buck_cut[1] - q.buck_cut[0]));
    h.b_rc2 = (T)(q.buck_cut[1] * q.buck_cut[1]);
    h.dt_max = (T)P.dt_max;
    h.dx_max = (T)P.dx_max;
    h.e_stop = (T)P.e_stop;
    h.M1 = (T)P.M1;
    h.invM1 = (T)P.invM1;
    h.gamma = (T)P.gamma;
    h.gamma0 = (T)lindhard_gamma_unit(ctx, P.Z1, P.M1);
    h.s_loc = (T)P.s_loc;
    h.rho0_inv = (T)P.rho0_inv;
    h.anchor_lo = (T)(-P.anchor_shift * P.a);
    h.anchor_hi = (T)((1.0 - P.anchor_shift) * P.a);
}

int basis_count(int kind) { return kind == REED_LATTICE_FLUORITE ? 12 : 8; }

// Lindhard-Scharff electronic stopping: S = k sqrt(E), k = 1.212 Z1^(7/6) Z2 /
// ((Z1^(2/3) + Z2^(2/3))^(3/2) sqrt(M1)) eV^(1/2) A^2; as a drag on the
// velocity, gamma = N k sqrt(M1/2) summed over target species.
double lindhard_gamma_unit(const reed_ctx* ctx, double Z1, double M1);

double lindhard_gamma(const reed_ctx* ctx, double Z1, double M1)
{
    return ctx->pot.s_e * lindhard_gamma_unit(ctx, Z1, M1);
}

// the same without the stopping scale s_e
double lindhard_gamma_unit(const reed_ctx* ctx, double Z1, double M1)
{
    const double vol = ctx->lat.a * ctx->lat.a * ctx->lat.a;
    double g = 0.0;
    for (int s = 0; s < ctx->nspec; ++s) {
        int count = ctx->lat.kind == REED_LATTICE_FLUORITE ? (s == 0 ? 4 : 8) : 8;
        double Z2 = ctx->sp[s].Z;
        double den = std::pow(std::pow(Z1, 2.0 / 3.0) + std::pow(Z2, 2.0 / 3.0), 1.5);
        double k = 1.212 * std::pow(Z1, 7.0 / 6.0) * Z2 / (den * std::sqrt(M1));
        g += count / vol * k;
    }
    return g * std::sqrt(M1 / 2.0);
}

// Rows of Tersoff bond storage: atoms of a perfect bulk window that are
// integrated or within the list radius of an integrated atom, plus 25 %
// head-room for disorder and cascades (capped at the window size).
int bond_capacity(const DevParams& P, double skin)
{
    if (P.tt == REED_TT_NONE) return 0;
    if (P.margin == 0) return P.na;
    if (P.tt == REED_TT_BUCKINGHAM) {   // lists of the integrated atoms only
        const int k = P.n - 2 * P.margin;
        return k * k * k * P.nb;
    }
    const double rl = P.hd.tcut + skin;
    std::vector<double> x;
    std::vector<char> act;
    for (int i = 0; i < P.n; ++i)
        for (int j = 0; j < P.n; ++j)
            for (int k = 0; k < P.n; ++k) {
                int o[3] = {i, j, k};
                bool a = true;
                for (int d = 0; d < 3; ++d)
                    if (o[d] < P.margin || o[d] > P.n - 1 - P.margin) a = false;
                for (int b = 0; b < P.nb; ++b) {
                    for (int d = 0; d < 3; ++d) x.push_back((o[d] + P.bas[b][d]) * P.a);
                    act.push_back(a);
                }
            }
    const size_t m = act.size();
    int count = 0;
    for (size_t i = 0; i < m; ++i) {
        bool need = act[i];
        for (size_t j = 0; j < m && !need; ++j) {
            if (!act[j]) continue;
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz < rl * rl) need = true;
        }
        count += need;
    }
    return std::min(P.na, (int)std::ceil(1.25 * count) + 32);
}

int make_params(reed_ctx* ctx, DevParams& P, double Z1, double M1, double E, double tilt, double rlo, double rhi,
                const reed_run_opts& o)
{
    std::memset(&P, 0, sizeof(P));
    const reed_lattice& L = ctx->lat;
    P.kind = L.kind;
    P.n = L.window_n;
    P.margin = L.frozen_margin;
    P.bulk = L.target == REED_TARGET_BULK;
    P.nb = basis_count(L.kind);
    P.na = P.n * P.n * P.n * P.nb;
    P.nspec = ctx->nspec;
    P.half_n = P.n / 2;
    P.a = L.a;
    P.inv_a = 1.0 / L.a;
    P.sigma = L.sigma;
    P.anchor_shift = (P.n % 2 == 0) ? 0.5 : 0.0;
    for (int b = 0; b < P.nb; ++b) {
        for (int d = 0; d < 3; ++d)
            P.bas[b][d] = L.kind == REED_LATTICE_FLUORITE ? kFluorite[b][d] : kDiamond[b][d];
        P.bspec[b] = (L.kind == REED_LATTICE_FLUORITE && b >= 4) ? 1 : 0;
    }
    for (int s = 0; s < 2; ++s) {
        const reed_species& q = ctx->sp[s < ctx->nspec ? s : 0];
        P.Z2[s] = q.Z;
        P.M2[s] = q.M;
        P.invM2[s] = 1.0 / q.M;
        P.zk[s] = Z1 * q.Z * REED_E2;
        P.zia[s] = screen_inv(Z1, q.Z);
    }
    P.Z1 = Z1;
    P.M1 = M1;
    P.invM1 = 1.0 / M1;
    const reed_potentials& q = ctx->pot;
    P.rc = q.rc;
    P.rt = q.r_taper;
    P.rc2 = q.rc * q.rc;
    P.inv_tw = 1.0 / (q.rc - q.r_taper);
    P.spline_on = 0;
    for (int i = 0; i < 6; ++i) {
        P.spline_c[i] = q.spline_c[i];
        P.spline_ctr[i] = std::log(kKnots[i]);
        if (q.spline_c[i] != 0.0) P.spline_on = 1;
    }
    P.spline_invh = 5.0 / (std::log(kKnots[5]) - std::log(kKnots[0]));
    P.tt = q.target_model;
    P.gamma = lindhard_gamma(ctx, Z1, M1);
    P.s_loc = q.s_loc;
    P.lam_inv = 1.0 / q.lam_loc;
    P.rho0_inv = 1.0 / (P.nb / (L.a * L.a * L.a) * 8.0 * REED_PI * q.lam_loc * q.lam_loc * q.lam_loc);
    P.rho_on = q.s_loc != 0.0;
    P.dt_max = o.dt_max_fs / REED_TAU_FS;
    P.dx_max = o.dx_max;
    P.e_stop = o.e_stop;
    P.step_cap = o.step_cap;
    P.v0 = std::sqrt(2.0 * E / M1);
    P.tilt = tilt * REED_PI / 180.0;
    P.rot_lo = rlo * REED_PI / 180.0;
    P.rot_span = (rhi - rlo) * REED_PI / 180.0;
    P.cos_tmax = std::cos(P.tilt);
    P.beam_mode = o.beam_mode;
    P.nthr = o.n_thresholds;
    for (int i = 0; i < o.n_thresholds; ++i) P.thr[i] = o.thresholds[i];
    P.nbins = ctx->nbins;
    P.bin_w = ctx->bin_w;
    P.first_id = o.first_id;
    P.dn = o.damage_n;
    P.dvox = o.damage_voxel > 0 ? o.damage_voxel : 10.0;
    P.dhalf = 0.5 * P.dn * P.dvox;
    P.dzhalf = P.bulk ? P.dhalf : 0.0;
    P.dmin = o.damage_min;
    P.de_max = o.de_max > 0.0 ? o.de_max : 0.0;
    P.dx_min = o.dx_min > 0.0 ? std::min(o.dx_min, o.dx_max) : std::min(1e-4, o.dx_max);
    P.pool_polls = o.pool_poll_limit > 0 ? o.pool_poll_limit : (1ll << 26);
    P.nl_check = o.nl_check ? 1 : 0;
    const double skin = o.nl_skin > 0.0 ? o.nl_skin : (P.tt == REED_TT_TERSOFF ? kSkinTersoff : kSkinPairs);
    // neighbour-search grid over the window: bins no narrower than the list
    // radius (with a margin for rounding) -- for Tersoff, whose lists are
    // refreshed between builds on the bins of the last build, than the list
    // radius plus half the skin -- at most 10 per axis
    {
        const double rl = (P.tt == REED_TT_BUCKINGHAM ? ctx->pot.buck_cut[1]
                                                     : ctx->pot.tersoff[9] + ctx->pot.tersoff[10] + 0.5 * skin) + skin;
        P.g_nb = std::max(1, std::min(10, (int)std::floor(P.n * P.a / (rl * 1.001))));
        P.g_nbins = P.g_nb * P.g_nb * P.g_nb;
    }
    fill_hot<float>(P.hf, P, ctx, skin);
    fill_hot<double>(P.hd, P, ctx, skin);
    P.bond_cap = bond_capacity(P, skin);
    {
        const int k = P.n - 2 * P.margin;
        P.act_cap = k * k * k * P.nb;
    }
    return REED_OK;
}

// Damage feedback fields of the parameters: on when the context has
// settings and a map; map = the cumulative map the created cells read.
void set_feedback(const reed_ctx* ctx, DevParams& P, const double* map)
{
    P.fb_map = nullptr;
    if (!(ctx->fb_ec > 0.0) || !ctx->d_damage || !map) return;
    P.fb_map = map;
    P.fb_n = ctx->dn;
    P.fb_vox = ctx->dvox;
    P.fb_half = 0.5 * ctx->dn * ctx->dvox;
    P.fb_zhalf = ctx->lat.target == REED_TARGET_BULK ? P.fb_half : 0.0;
    P.fb_dose = ctx->fb_dose;
    P.fb_atoms = basis_count(ctx->lat.kind) * std::pow(ctx->dvox / ctx->lat.a, 3.0);
    P.fb_ec = ctx->fb_ec;
    P.sigma_am = ctx->fb_sam;
}

// Beam and target geometry must agree: recoils start inside a bulk target,
// the other beams enter through the surface.  The adjoint's loss is on the
// depth below a surface.
const char* beam_error(const reed_lattice& L, const reed_run_opts& o)
{
    if (o.beam_mode != REED_BEAM_FIXED && o.beam_mode != REED_BEAM_CONE && o.beam_mode != REED_BEAM_RECOIL)
        return "beam_mode";
    if ((o.beam_mode == REED_BEAM_RECOIL) != (L.target == REED_TARGET_BULK))
        return "REED_BEAM_RECOIL goes with a BULK target and the other beams with a SURFACE target";
    if (o.adjoint && L.target == REED_TARGET_BULK) return "the adjoint needs a SURFACE target";
    return nullptr;
}

reed_run_opts default_opts()
{
    reed_run_opts o;
    std::memset(&o, 0, sizeof(o));
    o.dt_max_fs = 0.1;
    o.dx_max = 0.05;
    o.e_stop = 5.0;
    o.step_cap = 2000000;
    o.n_bins = 100;
    o.bin_width = 10.0;
    return o;
}

template <typename T> int dev_alloc(reed_ctx* ctx, T** p, size_t bytes)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    CK(cudaMalloc((void**)p, bytes));
    return REED_OK;
}

int ensure_tallies(reed_ctx* ctx, int nbins, double bin_w)
{
    if (ctx->d_hist) {
        if (nbins != ctx->nbins || bin_w != ctx->bin_w)
            return fail(ctx, REED_E_ARG, "histogram is %d x %g A since the last reset; got %d x %g", ctx->nbins,
                        ctx->bin_w, nbins, bin_w);
        return REED_OK;
    }
    ctx->nbins = nbins;
    ctx->bin_w = bin_w;
    int rc;
    if ((rc = dev_alloc(ctx, &ctx->d_hist, sizeof(double) * (nbins + 3)))) return rc;
    CK(cudaMemset(ctx->d_hist, 0, sizeof(double) * (nbins + 3)));
    return REED_OK;
}

bool valid_threads(int t) { return t == 32 || t == 64 || t == 128 || t == 256 || t == 512; }

}  // namespace

// ---------------------------------------------------------------------------
// Cloning-depth update at an epoch boundary (one thread): d_k = S^-1(2^-k)
// with S(d) the weighted fraction of finished tracks that stopped at depth
// >= d, read off the range histogram (nbins + under, over, back) with linear
// interpolation inside a bin; +inf when the target weight lies beyond the
// histogram.  An empty histogram leaves the depths unchanged.  The new set
// is also appended to the history row.
// ---------------------------------------------------------------------------
static __global__ void update_thresholds_kernel(const double* __restrict__ hist, int nbins, double bin_w, int nthr,
                                         double* __restrict__ thr, double* __restrict__ history_row)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double total = 0.0;
    for (int b = 0; b < nbins + 3; ++b) total += hist[b];
    if (total > 0.0) {
        const double beyond = hist[nbins + 1];
        for (int k = 1; k <= nthr; ++k) {
            const double target = ldexp(total, -k);
            double d = CUDART_INF;
            if (beyond < target) {
                double tail = beyond;
                d = 0.0;
                for (int b = nbins - 1; b >= 0; --b) {
                    const double wb = hist[b];
                    if (tail + wb >= target) {
                        d = ((double)b + 1.0 - (target - tail) / wb) * bin_w;
                        break;
                    }
                    tail += wb;
                }
            }
            thr[k - 1] = d;
        }
    }
    if (history_row)
        for (int k = 0; k < REED_MAX_THR; ++k) history_row[k] = k < nthr ? thr[k] : 0.0;
}


// ---------------------------------------------------------------------------
// Kernel-density profile of the recorded stopped tracks and its gradient
// (the adjoint workload's loss interface).  Deterministic: fixed summation
// orders, no atomics.
// ---------------------------------------------------------------------------
static __global__ void kde_weight_kernel(const reed_track_record* __restrict__ rec, long long n, double* __restrict__ wsum)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (long long i = 0; i < n; ++i)
        if (rec[i].status == REED_TRACK_STOPPED) s += ldexp(1.0, -rec[i].level);
    *wsum = s;
}

static __global__ void kde_profile_kernel(const reed_track_record* __restrict__ rec, long long n, const double* wsum,
                                          double sigma, int nb, double bw, double* __restrict__ p)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double zb = (b + 0.5) * bw, c = 1.0 / (sqrt(2.0 * REED_PI) * sigma), i2s = 0.5 / (sigma * sigma);
    double acc = 0.0;
    for (long long i = 0; i < n; ++i) {
        if (rec[i].status != REED_TRACK_STOPPED) continue;
        const double d = zb - rec[i].z;
        acc += ldexp(1.0, -rec[i].level) * exp(-d * d * i2s);
    }
    p[b] = *wsum > 0.0 ? acc * c / *wsum : 0.0;
}

// per-record contributions dL/dz_i * dz_i/dtheta, reduced per block in order
static __global__ void kde_grad_kernel(const reed_track_record* __restrict__ rec, const double* __restrict__ grads,
                                       long long n, const double* wsum, double sigma, int nb, double bw,
                                       const double* __restrict__ dLdp, double* __restrict__ part)
{
    __shared__ double red[256][REED_NTHETA_HOST];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double g[REED_NTHETA_HOST] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < n && rec[i].status == REED_TRACK_STOPPED && *wsum > 0.0) {
        const double c = 1.0 / (sqrt(2.0 * REED_PI) * sigma), is2 = 1.0 / (sigma * sigma);
        const double w = ldexp(1.0, -rec[i].level) / *wsum, z = rec[i].z;
        double dz = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double d = (b + 0.5) * bw - z;
            dz += dLdp[b] * w * c * exp(-0.5 * d * d * is2) * d * is2;
        }
        for (int k = 0; k < REED_NTHETA_HOST; ++k) g[k] = dz * grads[(size_t)i * REED_NTHETA_HOST + k];
    }
    for (int k = 0; k < REED_NTHETA_HOST; ++k) red[threadIdx.x][k] = g[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < REED_NTHETA_HOST; ++k) red[threadIdx.x][k] += red[threadIdx.x + o][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < REED_NTHETA_HOST; ++k) part[(size_t)blockIdx.x * REED_NTHETA_HOST + k] = red[0][k];
}

static __global__ void sum_parts_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out)
{
    if (threadIdx.x >= REED_NTHETA_HOST || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * REED_NTHETA_HOST + threadIdx.x];
    out[threadIdx.x] = s;
}

extern "C" {

int reed_init(reed_ctx** out, const reed_lattice* lat, const reed_species* sp, int n_species,
              const reed_potentials* pot)
{
    reed_ctx* ctx = nullptr;
    if (!out || !lat || !sp || !pot) return fail(nullptr, REED_E_ARG, "reed_init: null argument");
    *out = nullptr;
    if (lat->kind != REED_LATTICE_DIAMOND && lat->kind != REED_LATTICE_FLUORITE)
        return fail(nullptr, REED_E_ARG, "unknown lattice kind %d", lat->kind);
    if (lat->window_n < 2 || lat->window_n > 6) return fail(nullptr, REED_E_ARG, "window_n must be 2..6");
    if (lat->frozen_margin < 0 || 2 * lat->frozen_margin >= lat->window_n)
        return fail(nullptr, REED_E_ARG, "frozen_margin must be 0 or 1 and leave an integrated core");
    if (lat->target != REED_TARGET_SURFACE && lat->target != REED_TARGET_BULK)
        return fail(nullptr, REED_E_ARG, "unknown target geometry %d", lat->target);
    if (!(lat->a > 0.5) || !(lat->sigma >= 0.0)) return fail(nullptr, REED_E_ARG, "invalid lattice constant or sigma");
    int need = lat->kind == REED_LATTICE_FLUORITE ? 2 : 1;
    if (n_species != need) return fail(nullptr, REED_E_ARG, "lattice needs %d species, got %d", need, n_species);
    for (int s = 0; s < n_species; ++s)
        if (!(sp[s].Z > 0) || !(sp[s].M > 0)) return fail(nullptr, REED_E_ARG, "species %d: Z and M must be > 0", s);
    if (!(pot->rc > 0) || !(pot->r_taper >= 0) || !(pot->r_taper < pot->rc))
        return fail(nullptr, REED_E_ARG, "need 0 <= r_taper < rc");
    if (pot->target_model != REED_TT_NONE && pot->target_model != REED_TT_TERSOFF &&
        pot->target_model != REED_TT_BUCKINGHAM)
        return fail(nullptr, REED_E_ARG, "unknown target model %d", pot->target_model);
    if (pot->target_model == REED_TT_BUCKINGHAM && !(pot->buck_cut[1] > pot->buck_cut[0] && pot->buck_cut[0] >= 0))
        return fail(nullptr, REED_E_ARG, "Buckingham needs 0 <= taper start < cutoff");
    if (pot->target_model == REED_TT_TERSOFF && lat->kind != REED_LATTICE_DIAMOND)
        return fail(nullptr, REED_E_ARG, "Tersoff needs the one-species diamond lattice");
    if (!(pot->lam_loc > 0)) return fail(nullptr, REED_E_ARG, "lam_loc must be > 0");
    int na = lat->window_n * lat->window_n * lat->window_n * basis_count(lat->kind);
    if (na > 65535) return fail(nullptr, REED_E_ARG, "window too large");

    ctx = new reed_ctx();
    ctx->lat = *lat;
    ctx->nspec = n_species;
    for (int s = 0; s < n_species; ++s) ctx->sp[s] = sp[s];
    ctx->pot = *pot;
    cudaError_t e;
    if ((e = cudaGetDevice(&ctx->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess) {
        delete ctx;
        return fail(nullptr, REED_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    ctx->smem_optin = (size_t)optin;
    if (cudaMalloc((void**)&ctx->d_counters, sizeof(unsigned long long) * REED_NCOUNT) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_splits, sizeof(unsigned long long) * (REED_MAX_THR + 1)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_wsum, sizeof(double) * 4) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_next, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_rec_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_thr, sizeof(double) * REED_MAX_THR) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_finished, sizeof(unsigned long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        reed_destroy(ctx);
        return fail(nullptr, REED_E_NOMEM, "device allocation failed");
    }
    cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * REED_NCOUNT);
    cudaMemset(ctx->d_splits, 0, sizeof(unsigned long long) * (REED_MAX_THR + 1));
    cudaMemset(ctx->d_wsum, 0, sizeof(double) * 4);
    cudaMemset(ctx->d_rec_count, 0, sizeof(unsigned long long));
    {   // no cloning depth until one is set
        double inf[REED_MAX_THR];
        for (int k = 0; k < REED_MAX_THR; ++k) inf[k] = HUGE_VAL;
        cudaMemcpy(ctx->d_thr, inf, sizeof(inf), cudaMemcpyHostToDevice);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        reed_destroy(ctx);
        return fail(nullptr, REED_E_CUDA, "%s", cudaGetErrorString(e));
    }
    *out = ctx;
    return REED_OK;
}

int reed_run(reed_ctx* ctx, double ion_Z, double ion_M, double energy_eV, double tilt_deg, double rot_deg_lo,
             double rot_deg_hi, int64_t n_ions, uint64_t seed, const reed_run_opts* opt)
{
    if (!ctx) return REED_E_ARG;
    const reed_run_opts o = opt ? *opt : default_opts();
    if (!(ion_Z > 0) || !(ion_M > 0) || !(energy_eV > 0)) return fail(ctx, REED_E_ARG, "ion Z, M, energy must be > 0");
    if (n_ions < 0) return fail(ctx, REED_E_ARG, "n_ions < 0");
    if (!(o.dt_max_fs > 0) || !(o.dx_max > 0) || !(o.e_stop >= 0) || o.step_cap < 1)
        return fail(ctx, REED_E_ARG, "invalid integrator options");
    if (o.n_thresholds < 0 || o.n_thresholds > REED_MAX_THR) return fail(ctx, REED_E_ARG, "n_thresholds must be 0..16");
    for (int i = 1; i < o.n_thresholds; ++i)
        if (!(o.thresholds[i] > o.thresholds[i - 1])) return fail(ctx, REED_E_ARG, "thresholds must ascend");
    if (o.n_bins < 1 || !(o.bin_width > 0)) return fail(ctx, REED_E_ARG, "invalid histogram");
    if (const char* m = beam_error(ctx->lat, o)) return fail(ctx, REED_E_ARG, "%s", m);
    if (o.precision != REED_PREC_MIXED && o.precision != REED_PREC_FP64) return fail(ctx, REED_E_ARG, "precision");
    if (o.threads_per_track && !valid_threads(o.threads_per_track))
        return fail(ctx, REED_E_ARG, "threads_per_track must be 0, 32, 64, 128, 256 or 512");
    if (o.ctas_per_sm < 0 || o.trace_tracks < 0 || o.trace_steps < 0 || o.record_capacity < 0)
        return fail(ctx, REED_E_ARG, "negative option");
    int rc;
    if ((rc = ensure_tallies(ctx, o.n_bins, o.bin_width))) return rc;
    cudaStream_t st = (cudaStream_t)o.stream;

    DevParams P;
    make_params(ctx, P, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, o);
    P.seed = seed;
    P.n_primaries = n_ions;
    P.trace_tracks = o.trace_tracks;
    P.trace_steps = o.trace_steps;
    P.record = o.record_tracks ? 1 : 0;

    // records (kept across runs until reset; capacity fixed by the first run)
    if (P.record) {
        if (!ctx->d_records) {
            ctx->rec_cap = o.record_capacity > 0 ? o.record_capacity
                                                 : n_ions * (1 + 4 * (int64_t)o.n_thresholds) + 1024;
            if ((rc = dev_alloc(ctx, &ctx->d_records, sizeof(reed_track_record) * ctx->rec_cap))) return rc;
        }
        P.record_cap = ctx->rec_cap;
    }
    // damage map (kept across runs until reset; geometry fixed by the first run)
    if (o.damage_n < 0 || o.damage_n > 512) return fail(ctx, REED_E_ARG, "damage_n must be 0..512");
    if (o.damage_n > 0) {
        if (!ctx->d_damage) {
            const size_t nd = (size_t)o.damage_n * o.damage_n * o.damage_n + 1;
            if ((rc = dev_alloc(ctx, &ctx->d_damage, sizeof(double) * nd))) return rc;
            CK(cudaMemset(ctx->d_damage, 0, sizeof(double) * nd));
            ctx->dn = o.damage_n;
            ctx->dvox = P.dvox;
        } else if (ctx->dn != o.damage_n || ctx->dvox != P.dvox) {
            return fail(ctx, REED_E_ARG, "damage map is %d^3 x %g A since the last reset", ctx->dn, ctx->dvox);
        }
    }
    // trace buffers (per run)
    ctx->trace_tracks = o.trace_tracks;
    ctx->trace_steps = o.trace_steps;
    if (o.trace_tracks > 0 && o.trace_steps > 0) {
        size_t m = (size_t)o.trace_tracks * o.trace_steps;
        if ((rc = dev_alloc(ctx, &ctx->d_trace, sizeof(double) * 8 * m))) return rc;
        if ((rc = dev_alloc(ctx, &ctx->d_trace_anchor, sizeof(int) * 3 * m))) return rc;
        CK(cudaMemsetAsync(ctx->d_trace, 0, sizeof(double) * 8 * m, st));
        CK(cudaMemsetAsync(ctx->d_trace_anchor, 0, sizeof(int) * 3 * m, st));
    }

    // launch shape
    const int tt = P.tt;
    const bool f64 = o.precision == REED_PREC_FP64;
    // truncated-segment sensitivities
    if (o.adjoint) {
        if (tt != REED_TT_NONE || P.nthr > 0 || o.adaptive || !o.record_tracks)
            return fail(ctx, REED_E_ARG, "adjoint runs need target model NONE, no cloning and record_tracks");
        // (the reverse pass treats every atom of the window as integrated)
        if (P.margin != 0) return fail(ctx, REED_E_ARG, "adjoint runs need frozen_margin 0");
        const int seg = o.adj_segment > 0 ? o.adj_segment : 200, every = o.adj_every > 0 ? o.adj_every : 20;
        if (seg % every != 0 || seg + every > REED_STEP_RING_HOST)
            return fail(ctx, REED_E_ARG, "adj_segment must be a multiple of adj_every and adj_segment + adj_every <= %d",
                        REED_STEP_RING_HOST);
        P.adjoint = 1;
        P.rho_on = 1;   // d/ds_loc needs the local density even at s_loc = 0
        P.adj_seg = seg;
        P.adj_every = every;
        P.adj_nck = seg / every + 1;
    }
    const size_t smem = f64 ? reed_f64::smem_bytes(tt, P.na, P.bond_cap, P.adjoint, P.g_nbins, P.act_cap)
                            : reed_f32::smem_bytes(tt, P.na, P.bond_cap, P.adjoint, P.g_nbins, P.act_cap);
    if (smem > ctx->smem_optin)
        return fail(ctx, REED_E_SMEM, "window of %d atoms needs %zu B of shared memory (max %zu)", P.na, smem,
                    ctx->smem_optin);
    LaunchCfg L;
    const int pi = f64 ? 1 : 0, ai = P.adjoint ? 1 : 0;
    const bool tuned = !o.threads_per_track && !o.ctas_per_sm && ctx->tuned_threads[pi][ai] > 0;
    L.threads = o.threads_per_track ? o.threads_per_track
                                    : (tuned ? ctx->tuned_threads[pi][ai] : (tt == REED_TT_NONE ? 64 : 256));
    L.smem = smem;
    int occ = 0;
    CK(f64 ? reed_f64::occupancy(tt, L.threads, smem, &occ, P.adjoint)
           : reed_f32::occupancy(tt, L.threads, smem, &occ, P.adjoint));
    if (occ < 1) return fail(ctx, REED_E_SMEM, "kernel does not fit on an SM (%zu B shared, %d threads)", smem, L.threads);
    L.ctas_per_sm = o.ctas_per_sm ? std::min(o.ctas_per_sm, occ) : (tuned ? std::min(ctx->tuned_ctas[pi][ai], occ) : occ);
    L.grid = ctx->sms * L.ctas_per_sm;

    // clone stacks: one record per cloning level per CTA
    DevBuf B;
    std::memset(&B, 0, sizeof(B));
    B.entry_bytes = f64 ? reed_f64::entry_bytes(tt, P.na) : reed_f32::entry_bytes(tt, P.na);
    B.stack_depth = P.nthr;
    B.stack_stride = B.entry_bytes * (size_t)std::max(P.nthr, 1);
    if (P.nthr > 0) {
        size_t need = B.stack_stride * (size_t)L.grid;
        if (need > ctx->stacks_bytes) {
            if ((rc = dev_alloc(ctx, &ctx->d_stacks, need))) return rc;
            ctx->stacks_bytes = need;
        }
        B.stacks = ctx->d_stacks;
        // the shared pool: one record per CTA, taken by CTAs that run out of work
        const size_t pool_need = B.entry_bytes * (size_t)L.grid;
        if (pool_need > ctx->pool_bytes) {
            if ((rc = dev_alloc(ctx, &ctx->d_pool, pool_need))) return rc;
            ctx->pool_bytes = pool_need;
        }
        if (L.grid + 3 > ctx->pool_state_cap) {
            if ((rc = dev_alloc(ctx, &ctx->d_pool_state, sizeof(unsigned) * (size_t)(L.grid + 3)))) return rc;
            ctx->pool_state_cap = L.grid + 3;
        }
        B.pool = ctx->d_pool;
        B.pool_state = ctx->d_pool_state;
        B.pool_ctl = ctx->d_pool_state + L.grid;
        B.pool_slots = L.grid;
    }
    // neighbour-list overflow rows: one block per CTA
    B.spill_stride = f64 ? reed_f64::spill_bytes(tt) : reed_f32::spill_bytes(tt);
    if (B.spill_stride) {
        const size_t need = B.spill_stride * (size_t)L.grid;
        if (need > ctx->spill_bytes) {
            if ((rc = dev_alloc(ctx, &ctx->d_spill, need))) return rc;
            ctx->spill_bytes = need;
        }
        B.spill = ctx->d_spill;
    }
    B.hist = ctx->d_hist;
    B.counters = ctx->d_counters;
    B.splits = ctx->d_splits;
    B.wsum = ctx->d_wsum;
    B.next = ctx->d_next;
    B.records = ctx->d_records;
    B.record_count = ctx->d_rec_count;
    B.trace = ctx->d_trace;
    B.trace_anchor = ctx->d_trace_anchor;
    B.status = ctx->d_status;

    B.thr = ctx->d_thr;
    B.finished = ctx->d_finished;
    B.damage = o.damage_n > 0 ? ctx->d_damage : nullptr;
    if (P.adjoint) {
        if (!ctx->d_grads || ctx->grads_cap < ctx->rec_cap) {
            if ((rc = dev_alloc(ctx, &ctx->d_grads, sizeof(double) * REED_NTHETA_HOST * (size_t)ctx->rec_cap))) return rc;
            CK(cudaMemset(ctx->d_grads, 0, sizeof(double) * REED_NTHETA_HOST * (size_t)ctx->rec_cap));
            ctx->grads_cap = ctx->rec_cap;
        }
        const size_t per = f64 ? reed_f64::adj_scratch_bytes(P, B.entry_bytes) : reed_f32::adj_scratch_bytes(P, B.entry_bytes);
        const size_t need = per * (size_t)L.grid;
        if (need > ctx->adj_bytes) {
            if ((rc = dev_alloc(ctx, &ctx->d_adj, need))) return rc;
            ctx->adj_bytes = need;
        }
        B.adj = ctx->d_adj;
        B.adj_stride = per;
        B.grads = ctx->d_grads;
    }
    P.stop_after = o.target_tracks;

    // epochs: one launch, or (adaptive) unenhanced primaries followed by
    // epochs whose cloning depths are re-estimated on the device first
    struct Epoch {
        int64_t first, count;
        int nthr, update, guess;
    };
    std::vector<Epoch> ep;
    if (!o.adaptive) {
        ep.push_back({o.first_id, n_ions, P.nthr, 0, 0});
    } else {
        if (o.epoch_size < 1 || o.n_initial < 0 || P.nthr < 1)
            return fail(ctx, REED_E_ARG, "adaptive runs need epoch_size >= 1, n_initial >= 0, n_thresholds >= 1");
        const int64_t ninit = std::min<int64_t>(o.n_initial, n_ions);
        int64_t done = 0;
        if (ninit > 0) {
            ep.push_back({o.first_id, ninit, 0, 0, 0});
            done = ninit;
        }
        bool first_enh = true;
        while (done < n_ions) {
            const int64_t m = std::min<int64_t>(o.epoch_size, n_ions - done);
            const int guess = (first_enh && ninit == 0) ? 1 : 0;
            ep.push_back({o.first_id + done, m, P.nthr, guess ? 0 : 1, guess});
            done += m;
            first_enh = false;
        }
        int nenh = 0;
        for (const Epoch& e : ep) nenh += e.nthr > 0;
        if (nenh > ctx->thr_hist_cap) {
            if ((rc = dev_alloc(ctx, &ctx->d_thr_hist, sizeof(double) * REED_MAX_THR * (size_t)nenh))) return rc;
            ctx->thr_hist_cap = nenh;
        }
        ctx->thr_epochs = nenh;
        CK(cudaMemcpy(ctx->d_thr, o.thresholds, sizeof(double) * REED_MAX_THR, cudaMemcpyHostToDevice));
    }
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
    CK(cudaMemsetAsync(ctx->d_finished, 0, sizeof(unsigned long long), st));
    // damage feedback: every launch reads a snapshot of the cumulative map
    // taken as it starts, so a launch's tracks do not depend on timing
    size_t snap_bytes = 0;
    if (ctx->fb_ec > 0.0 && ctx->d_damage) {
        snap_bytes = sizeof(double) * ((size_t)ctx->dn * ctx->dn * ctx->dn + 1);
        if (snap_bytes > ctx->dsnap_bytes) {
            if ((rc = dev_alloc(ctx, &ctx->d_dsnap, snap_bytes))) return rc;
            ctx->dsnap_bytes = snap_bytes;
        }
        set_feedback(ctx, P, ctx->d_dsnap);
    }

    // the device work of the run, on stream s
    auto enqueue = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        int row = 0;
        for (const Epoch& x : ep) {
            if (x.count <= 0) continue;
            DevParams Pe = P;
            Pe.first_id = x.first;
            Pe.n_primaries = x.count;
            Pe.nthr = x.nthr;
            Pe.thr_from_device = ((o.adaptive || o.device_thresholds) && x.nthr > 0) ? 1 : 0;
            if ((e = cudaMemsetAsync(ctx->d_next, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
            if (snap_bytes &&
                (e = cudaMemcpyAsync(ctx->d_dsnap, ctx->d_damage, snap_bytes, cudaMemcpyDeviceToDevice, s)) !=
                    cudaSuccess)
                return e;
            if (B.pool &&
                (e = cudaMemsetAsync(B.pool_state, 0, sizeof(unsigned) * (size_t)(B.pool_slots + 3), s)) != cudaSuccess)
                return e;
            if (o.adaptive && x.nthr > 0) {
                double* hrow = ctx->d_thr_hist + (size_t)REED_MAX_THR * row++;
                if (x.update) {
                    update_thresholds_kernel<<<1, 1, 0, s>>>(ctx->d_hist, ctx->nbins, ctx->bin_w, x.nthr, ctx->d_thr,
                                                             hrow);
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                } else if ((e = cudaMemcpyAsync(hrow, ctx->d_thr, sizeof(double) * REED_MAX_THR,
                                                cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
                    return e;
                }
            }
            e = f64 ? reed_f64::launch_track(tt, Pe, B, L, s) : reed_f32::launch_track(tt, Pe, B, L, s);
            if (e != cudaSuccess) return e;
        }
        return e;
    };
    CK(cudaEventRecord(ctx->ev0, st));
    if (ep.size() > 1) {
        // several dependent launches: capture them once into a CUDA graph
        cudaEvent_t ready = ctx->ev1;
        CK(cudaEventRecord(ready, st));
        CK(cudaStreamWaitEvent(ctx->cap_stream, ready, 0));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = enqueue(ctx->cap_stream);
        cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
        CK(ce);
        CK(ee);
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        cudaError_t le = cudaGraphLaunch(exec, st);
        cudaError_t se = cudaStreamSynchronize(st);
        cudaGraphExecDestroy(exec);
        CK(le);
        CK(se);
    } else {
        CK(enqueue(st));
    }
    CK(cudaEventRecord(ctx->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    ctx->last_ms = ms;
    ctx->last_cfg = L;
    int status = 0;
    CK(cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & ERR_TIMEOUT)
        return fail(ctx, REED_E_TIMEOUT, "an idle CTA stopped waiting for the shared clone pool: tracks may be missing");
    if (status & ERR_NONFINITE) return fail(ctx, REED_E_NONFINITE, "a track became non-finite (see reed_stats)");
    if (status & ERR_QUEUE) return fail(ctx, REED_E_QUEUE_FULL, "clone stack overflow: clones dropped");
    if (status & ERR_NEIGHBOR)
        return fail(ctx, REED_E_NEIGHBOR,
                    "a neighbour list outgrew its overflow row or the overflow rows ran out (see nb_overflow, "
                    "bond_cap_overflow in reed_stats): forces were incomplete");
    return REED_OK;
}

int reed_range_profile(reed_ctx* ctx, double* bins_out, int n_bins, double* extra3)
{
    if (!ctx) return REED_E_ARG;
    if (!ctx->d_hist) return fail(ctx, REED_E_STATE, "no run since init/reset");
    if (n_bins != ctx->nbins || !bins_out) return fail(ctx, REED_E_ARG, "expected %d bins", ctx->nbins);
    CK(cudaMemcpy(bins_out, ctx->d_hist, sizeof(double) * n_bins, cudaMemcpyDefault));
    if (extra3) CK(cudaMemcpy(extra3, ctx->d_hist + n_bins, sizeof(double) * 3, cudaMemcpyDefault));
    return REED_OK;
}

int reed_stats(reed_ctx* ctx, reed_stats_t* out)
{
    if (!ctx || !out) return REED_E_ARG;
    unsigned long long c[REED_NCOUNT], sp[REED_MAX_THR + 1];
    double w[4];
    CK(cudaMemcpy(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(sp, ctx->d_splits, sizeof(sp), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w, ctx->d_wsum, sizeof(w), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->primaries = (int64_t)c[C_PRIMARIES];
    out->clones = (int64_t)c[C_CLONES];
    out->tracks = (int64_t)c[C_TRACKS];
    out->steps = (int64_t)c[C_STEPS];
    out->pair_evals = (int64_t)c[C_PAIRS];
    out->bond_evals = (int64_t)c[C_BONDS];
    out->shifts = (int64_t)c[C_SHIFTS];
    out->rebuilds = (int64_t)c[C_REBUILDS];
    out->dropped_clones = (int64_t)c[C_DROPPED];
    out->nb_overflow = (int64_t)c[C_NBOVF];
    out->bond_cap_overflow = (int64_t)c[C_CAPOVF];
    out->nb_spilled = (int64_t)c[C_SPILLED];
    out->list_refreshes = (int64_t)c[C_REFRESH];
    out->nl_check_errors = (int64_t)c[C_NLCHECK];
    out->triplets = (int64_t)c[C_TRIPLETS];
    out->atom_updates = (int64_t)c[C_MOVED];
    for (int k = 0; k < REED_NPHASE; ++k) out->phase_cycles[k] = (int64_t)c[C_PHASE0 + k];
    for (int k = 0; k < 4; ++k) out->centre_class[k] = (int64_t)c[C_CLS0 + k];
    for (int k = 0; k < REED_MAX_THR; ++k) out->splits[k] = (int64_t)sp[k];
    out->pooled = (int64_t)sp[REED_MAX_THR];
    out->failed = (int64_t)c[C_FAILED];
    out->stopped = (int64_t)c[C_STOP];
    out->backscattered = (int64_t)c[C_BACK];
    out->truncated = (int64_t)c[C_TRUNC];
    out->w_stopped = w[W_STOPPED];
    out->w_back = w[W_BACK];
    out->w_trunc = w[W_TRUNC];
    out->kernel_ms = ctx->last_ms;
    out->threads_per_track = ctx->last_cfg.threads;
    out->ctas_per_sm = ctx->last_cfg.ctas_per_sm;
    out->grid = ctx->last_cfg.grid;
    out->smem_bytes = (int32_t)ctx->last_cfg.smem;
    return REED_OK;
}

int reed_track_records(reed_ctx* ctx, reed_track_record* out, int64_t cap, int64_t* n_out)
{
    if (!ctx || !n_out || cap < 0) return REED_E_ARG;
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, ctx->d_rec_count, sizeof(n), cudaMemcpyDeviceToHost));
    int64_t kept = std::min<int64_t>((int64_t)n, ctx->rec_cap);
    int64_t m = std::min<int64_t>(kept, cap);
    if (m > 0 && out) CK(cudaMemcpy(out, ctx->d_records, sizeof(reed_track_record) * m, cudaMemcpyDefault));
    *n_out = kept;
    return REED_OK;
}

int reed_trace(reed_ctx* ctx, double* traj, int32_t* anchors, int n_tracks, int n_steps)
{
    if (!ctx) return REED_E_ARG;
    if (n_tracks != ctx->trace_tracks || n_steps != ctx->trace_steps || !ctx->d_trace)
        return fail(ctx, REED_E_STATE, "last run traced %d x %d", ctx->trace_tracks, ctx->trace_steps);
    size_t m = (size_t)n_tracks * n_steps;
    if (traj) CK(cudaMemcpy(traj, ctx->d_trace, sizeof(double) * 8 * m, cudaMemcpyDefault));
    if (anchors) CK(cudaMemcpy(anchors, ctx->d_trace_anchor, sizeof(int) * 3 * m, cudaMemcpyDefault));
    return REED_OK;
}

int reed_track_grads(reed_ctx* ctx, double* out, int64_t cap, int64_t* n_out)
{
    if (!ctx || !n_out || cap < 0) return REED_E_ARG;
    if (!ctx->d_grads) return fail(ctx, REED_E_STATE, "no adjoint run since init/reset");
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, ctx->d_rec_count, sizeof(n), cudaMemcpyDeviceToHost));
    const int64_t kept = std::min<int64_t>((int64_t)n, ctx->rec_cap);
    const int64_t m = std::min<int64_t>(kept, cap);
    if (m > 0 && out) CK(cudaMemcpy(out, ctx->d_grads, sizeof(double) * REED_NTHETA_HOST * m, cudaMemcpyDefault));
    *n_out = kept;
    return REED_OK;
}

namespace {
int kde_prepare(reed_ctx* ctx, int n_bins, long long* nrec, double** wsum, double** part, int* nblk)
{
    if (!ctx->d_records) return fail(ctx, REED_E_STATE, "no recorded tracks since init/reset");
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, ctx->d_rec_count, sizeof(n), cudaMemcpyDeviceToHost));
    *nrec = std::min<long long>((long long)n, ctx->rec_cap);
    *nblk = (int)((*nrec + 255) / 256);
    const size_t need = sizeof(double) * (8 + 2 * (size_t)n_bins + REED_NTHETA_HOST * (size_t)std::max(*nblk, 1) + 8);
    if (need > ctx->kde_bytes) {
        if (ctx->d_kde) cudaFree(ctx->d_kde);
        ctx->d_kde = nullptr;
        ctx->kde_bytes = 0;
        CK(cudaMalloc((void**)&ctx->d_kde, need));
        ctx->kde_bytes = need;
    }
    *wsum = ctx->d_kde;
    *part = ctx->d_kde + 8 + 2 * (size_t)n_bins;
    return REED_OK;
}
}  // namespace

int reed_kde_profile(reed_ctx* ctx, double sigma, int n_bins, double bin_width, double* p_out)
{
    if (!ctx || !p_out || n_bins < 1 || !(sigma > 0) || !(bin_width > 0)) return REED_E_ARG;
    long long n;
    double *wsum, *part;
    int nblk, rc;
    if ((rc = kde_prepare(ctx, n_bins, &n, &wsum, &part, &nblk))) return rc;
    double* dp = ctx->d_kde + 8;
    kde_weight_kernel<<<1, 1>>>(ctx->d_records, n, wsum);
    kde_profile_kernel<<<(n_bins + 127) / 128, 128>>>(ctx->d_records, n, wsum, sigma, n_bins, bin_width, dp);
    CK(cudaGetLastError());
    CK(cudaMemcpy(p_out, dp, sizeof(double) * n_bins, cudaMemcpyDefault));
    return REED_OK;
}

int reed_grad(reed_ctx* ctx, double sigma, int n_bins, double bin_width, const double* dL_dp, double* dL_dtheta)
{
    if (!ctx || !dL_dp || !dL_dtheta || n_bins < 1 || !(sigma > 0) || !(bin_width > 0)) return REED_E_ARG;
    if (!ctx->d_grads) return fail(ctx, REED_E_STATE, "no adjoint run since init/reset");
    long long n;
    double *wsum, *part;
    int nblk, rc;
    if ((rc = kde_prepare(ctx, n_bins, &n, &wsum, &part, &nblk))) return rc;
    double* dl = ctx->d_kde + 8 + n_bins;
    CK(cudaMemcpy(dl, dL_dp, sizeof(double) * n_bins, cudaMemcpyDefault));
    kde_weight_kernel<<<1, 1>>>(ctx->d_records, n, wsum);
    if (nblk > 0)
        kde_grad_kernel<<<nblk, 256>>>(ctx->d_records, ctx->d_grads, n, wsum, sigma, n_bins, bin_width, dl, part);
    double* out = part + (size_t)REED_NTHETA_HOST * std::max(nblk, 1);
    if (nblk > 0) sum_parts_kernel<<<1, 32>>>(part, nblk, out);
    else CK(cudaMemset(out, 0, sizeof(double) * REED_NTHETA_HOST));
    CK(cudaGetLastError());
    CK(cudaMemcpy(dL_dtheta, out, sizeof(double) * REED_NTHETA_HOST, cudaMemcpyDefault));
    return REED_OK;
}

int reed_set_theta(reed_ctx* ctx, const double* theta8)
{
    if (!ctx || !theta8) return REED_E_ARG;
    ctx->pot.s_e = theta8[0];
    ctx->pot.s_loc = theta8[1];
    for (int i = 0; i < 6; ++i) ctx->pot.spline_c[i] = theta8[2 + i];
    return REED_OK;
}

int reed_damage_map(reed_ctx* ctx, double* out, int n, double* overflow)
{
    if (!ctx || !out) return REED_E_ARG;
    if (!ctx->d_damage) return fail(ctx, REED_E_STATE, "no damage map since init/reset");
    if (n != ctx->dn) return fail(ctx, REED_E_ARG, "damage map has %d voxels per edge", ctx->dn);
    const size_t v = (size_t)n * n * n;
    CK(cudaMemcpy(out, ctx->d_damage, sizeof(double) * v, cudaMemcpyDefault));
    if (overflow) CK(cudaMemcpy(overflow, ctx->d_damage + v, sizeof(double), cudaMemcpyDefault));
    return REED_OK;
}

int reed_thresholds(reed_ctx* ctx, double* history, int max_epochs, int* n_epochs)
{
    if (!ctx || !n_epochs || max_epochs < 0) return REED_E_ARG;
    *n_epochs = ctx->thr_epochs;
    const int m = std::min(max_epochs, ctx->thr_epochs);
    if (m > 0 && history)
        CK(cudaMemcpy(history, ctx->d_thr_hist, sizeof(double) * REED_MAX_THR * m, cudaMemcpyDefault));
    return REED_OK;
}

int reed_set_damage_feedback(reed_ctx* ctx, double dose_scale, double e_crit, double sigma_amorphous)
{
    if (!ctx || !(dose_scale >= 0.0) || !(e_crit >= 0.0) || !(sigma_amorphous >= 0.0)) return REED_E_ARG;
    ctx->fb_dose = dose_scale;
    ctx->fb_ec = e_crit;
    ctx->fb_sam = sigma_amorphous;
    return REED_OK;
}

int reed_set_damage_map(reed_ctx* ctx, const double* map, int n, double voxel)
{
    if (!ctx || !map || n < 1 || n > 512 || !(voxel > 0.0)) return REED_E_ARG;
    const size_t nd = (size_t)n * n * n + 1;
    int rc;
    if (!ctx->d_damage || ctx->dn != n) {
        if ((rc = dev_alloc(ctx, &ctx->d_damage, sizeof(double) * nd))) return rc;
    }
    ctx->dn = n;
    ctx->dvox = voxel;
    CK(cudaMemcpy(ctx->d_damage, map, sizeof(double) * nd, cudaMemcpyDefault));
    return REED_OK;
}

int reed_update_thresholds(reed_ctx* ctx, const double* hist, int n_bins, double bin_width, int n_thresholds,
                           const double* thresholds)
{
    if (!ctx || n_thresholds < 1 || n_thresholds > REED_MAX_THR) return REED_E_ARG;
    if (hist) {
        if (n_bins < 1 || !(bin_width > 0)) return fail(ctx, REED_E_ARG, "need n_bins >= 1 and bin_width > 0");
        const size_t need = sizeof(double) * ((size_t)n_bins + 3);
        if (need > ctx->kde_bytes) {
            if (ctx->d_kde) cudaFree(ctx->d_kde);
            ctx->d_kde = nullptr;
            ctx->kde_bytes = 0;
            CK(cudaMalloc((void**)&ctx->d_kde, need));
            ctx->kde_bytes = need;
        }
        CK(cudaMemcpy(ctx->d_kde, hist, need, cudaMemcpyDefault));
        update_thresholds_kernel<<<1, 1>>>(ctx->d_kde, n_bins, bin_width, n_thresholds, ctx->d_thr, nullptr);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
    } else {
        if (!thresholds) return REED_E_ARG;
        CK(cudaMemcpy(ctx->d_thr, thresholds, sizeof(double) * n_thresholds, cudaMemcpyHostToDevice));
    }
    return REED_OK;
}

int reed_get_thresholds(reed_ctx* ctx, double* out16)
{
    if (!ctx || !out16) return REED_E_ARG;
    CK(cudaMemcpy(out16, ctx->d_thr, sizeof(double) * REED_MAX_THR, cudaMemcpyDefault));
    return REED_OK;
}

int reed_reset(reed_ctx* ctx)
{
    if (!ctx) return REED_E_ARG;
    if (ctx->d_hist) cudaFree(ctx->d_hist);
    ctx->d_hist = nullptr;
    if (ctx->d_records) cudaFree(ctx->d_records);
    ctx->d_records = nullptr;
    ctx->rec_cap = 0;
    if (ctx->d_damage) cudaFree(ctx->d_damage);
    ctx->d_damage = nullptr;
    ctx->dn = 0;
    if (ctx->d_grads) cudaFree(ctx->d_grads);
    ctx->d_grads = nullptr;
    ctx->grads_cap = 0;
    CK(cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * REED_NCOUNT));
    CK(cudaMemset(ctx->d_splits, 0, sizeof(unsigned long long) * (REED_MAX_THR + 1)));
    CK(cudaMemset(ctx->d_wsum, 0, sizeof(double) * 4));
    CK(cudaMemset(ctx->d_rec_count, 0, sizeof(unsigned long long)));
    return REED_OK;
}

const char* reed_last_error(reed_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

void reed_destroy(reed_ctx* ctx)
{
    if (!ctx) return;
    void* ptrs[] = {ctx->d_dsnap, ctx->d_pool, ctx->d_pool_state, ctx->d_hist, ctx->d_counters, ctx->d_splits, ctx->d_wsum, ctx->d_next, ctx->d_status, ctx->d_records,
                    ctx->d_rec_count, ctx->d_trace, ctx->d_trace_anchor, ctx->d_stacks, ctx->d_scratch,
                    ctx->d_thr, ctx->d_thr_hist, ctx->d_finished, ctx->d_damage, ctx->d_grads,
                    ctx->d_adj, ctx->d_kde, ctx->d_spill};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

int reed_autotune(reed_ctx* ctx, double ion_Z, double ion_M, double energy_eV, double tilt_deg, double rot_deg_lo,
                  double rot_deg_hi, int64_t n_trial, uint64_t seed, const reed_run_opts* opt, reed_tune_entry* table,
                  int cap, int* n_out)
{
    if (!ctx || !opt || n_trial < 1 || cap < 0) return REED_E_ARG;
    if (n_out) *n_out = 0;
    reed_ctx* t = nullptr;
    int rc = reed_init(&t, &ctx->lat, ctx->sp, ctx->nspec, &ctx->pot);
    if (rc) return fail(ctx, rc, "autotune: %s", g_init_error.c_str());
    reed_run_opts o = *opt;
    o.record_tracks = 0;
    o.trace_tracks = 0;
    o.trace_steps = 0;
    o.adaptive = 0;
    o.device_thresholds = 0;
    o.n_thresholds = 0;
    o.damage_n = 0;
    o.target_tracks = 0;
    o.first_id = (int64_t)1 << 40;
    const int pi = opt->precision == REED_PREC_FP64 ? 1 : 0, ai = opt->adjoint ? 1 : 0;
    if (ai) o.record_tracks = 1;
    int best_t = 0, best_c = 0, n = 0;
    double best = -1.0;
    static const int kThreads[5] = {32, 64, 128, 256, 512};
    for (int ti = 0; ti < 5; ++ti) {
        // the occupancy maximum for this thread count: a run with ctas_per_sm
        // far above it is clamped to it
        reed_run_opts probe = o;
        probe.threads_per_track = kThreads[ti];
        probe.ctas_per_sm = 1 << 20;
        probe.step_cap = 1;
        reed_reset(t);
        rc = reed_run(t, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, 1, seed, &probe);
        if (rc < 0) continue;   // does not fit (shared memory / threads)
        o.threads_per_track = kThreads[ti];
        const int occ = t->last_cfg.ctas_per_sm;
        int cands[3] = {occ, (3 * occ + 3) / 4, (occ + 1) / 2};
        for (int ci = 0; ci < 3; ++ci) {
            const int c = cands[ci];
            bool dup = false;
            for (int k = 0; k < ci; ++k) dup |= cands[k] == c;
            if (dup || c < 1) continue;
            o.ctas_per_sm = c;
            reed_reset(t);
            rc = reed_run(t, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, n_trial, seed, &o);
            if (rc < 0) {
                reed_destroy(t);
                return fail(ctx, rc, "autotune trial (%d threads, %d CTAs/SM) failed", kThreads[ti], c);
            }
            reed_stats_t st;
            reed_stats(t, &st);
            const double v = st.kernel_ms > 0 ? (double)st.steps / (st.kernel_ms * 1e-3) : 0.0;
            if (table && n < cap) table[n] = {kThreads[ti], c, v};
            ++n;
            if (v > best) {
                best = v;
                best_t = kThreads[ti];
                best_c = c;
            }
        }
    }
    reed_destroy(t);
    if (n_out) *n_out = n;
    if (best_t == 0) return fail(ctx, REED_E_SMEM, "autotune: no launch configuration fits");
    ctx->tuned_threads[pi][ai] = best_t;
    ctx->tuned_ctas[pi][ai] = best_c;
    return REED_OK;
}

// ---- diagnostics -------------------------------------------------------

static __global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                                     uint32_t* __restrict__ out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    philox10(c, key[2 * i], key[2 * i + 1]);
    for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
}

int reed_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n)
{
    reed_ctx* ctx = nullptr;
    if (!ctr || !key || !out || n < 0) return fail(nullptr, REED_E_ARG, "reed_philox: bad argument");
    if (n == 0) return REED_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    CK(cudaMalloc((void**)&dc, 16 * n));
    CK(cudaMalloc((void**)&dk, 8 * n));
    CK(cudaMalloc((void**)&dout, 16 * n));
    CK(cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice));
    philox_kernel<<<(unsigned)((n + 127) / 128), 128>>>(dc, dk, dout, n);
    CK(cudaGetLastError());
    CK(cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost));
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return REED_OK;
}

namespace {
size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

int scratch(reed_ctx* ctx, size_t bytes, void** p)
{
    if (bytes > ctx->scratch_bytes) {
        if (ctx->d_scratch) cudaFree(ctx->d_scratch);
        ctx->d_scratch = nullptr;
        ctx->scratch_bytes = 0;
        CK(cudaMalloc(&ctx->d_scratch, bytes));
        ctx->scratch_bytes = bytes;
    }
    *p = ctx->d_scratch;
    return REED_OK;
}

reed_run_opts diag_opts()
{
    reed_run_opts o = default_opts();
    return o;
}
}  // namespace

int reed_cell_atoms(reed_ctx* ctx, uint64_t key, int32_t ix, int32_t iy, int32_t iz, double* xyz_out,
                    int32_t* species_out)
{
    if (!ctx || !xyz_out || !species_out) return REED_E_ARG;
    DevParams P;
    reed_run_opts o = diag_opts();
    make_params(ctx, P, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, o);
    set_feedback(ctx, P, ctx->d_damage);
    void* s = nullptr;
    int rc;
    if ((rc = scratch(ctx, 512, &s))) return rc;
    double* dx = (double*)s;
    int* dsp = (int*)((char*)s + 36 * sizeof(double));
    int* dn = dsp + 12;
    CK(reed_f64::launch_cell_atoms(P, key, ix, iy, iz, dx, dsp, dn, 0));
    int n = 0;
    CK(cudaMemcpy(&n, dn, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(xyz_out, dx, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(species_out, dsp, sizeof(int) * n, cudaMemcpyDeviceToHost));
    return n;
}

int reed_forces(reed_ctx* ctx, int precision, double ion_Z, double ion_M, const double* ion_x, int n,
                const double* xyz, const int32_t* sp, double* f_ion, double* f_atoms, double* energy, double* rho)
{
    if (!ctx || !ion_x || (n > 0 && (!xyz || !sp || !f_atoms)) || !f_ion || n < 0) return REED_E_ARG;
    DevParams P;
    reed_run_opts o = diag_opts();
    make_params(ctx, P, ion_Z, ion_M, 1.0, 0.0, 0.0, 0.0, o);
    if (n > P.na) return fail(ctx, REED_E_ARG, "at most %d atoms", P.na);
    for (int i = 0; i < n; ++i)
        if (sp[i] < 0 || sp[i] >= ctx->nspec) return fail(ctx, REED_E_ARG, "species %d out of range", sp[i]);
    const bool f64 = precision == REED_PREC_FP64;
    // every given atom is integrated
    if (P.tt == REED_TT_TERSOFF) P.bond_cap = std::max(n, 1);
    P.act_cap = std::max(n, 1);
    size_t smem = f64 ? reed_f64::smem_bytes(P.tt, P.na, P.bond_cap, 0, P.g_nbins, P.act_cap)
                      : reed_f32::smem_bytes(P.tt, P.na, P.bond_cap, 0, P.g_nbins, P.act_cap);
    if (smem > ctx->smem_optin) return fail(ctx, REED_E_SMEM, "window needs %zu B shared memory", smem);
    size_t bx = up16(sizeof(double) * 3 * (size_t)std::max(n, 1)), bs = up16(sizeof(int) * (size_t)std::max(n, 1));
    size_t bi = up16(sizeof(double) * 3), bo = up16(sizeof(double) * (6 + 3 * (size_t)std::max(n, 1)));
    size_t bsp = up16(f64 ? reed_f64::spill_bytes(P.tt) : reed_f32::spill_bytes(P.tt));
    void* s = nullptr;
    int rc;
    if ((rc = scratch(ctx, bx + bs + bi + bo + bsp, &s))) return rc;
    double* dx = (double*)s;
    int* dsp = (int*)((char*)s + bx);
    double* dion = (double*)((char*)s + bx + bs);
    double* dout = (double*)((char*)s + bx + bs + bi);
    unsigned char* dspill = bsp ? (unsigned char*)s + bx + bs + bi + bo : nullptr;
    if (n > 0) {
        CK(cudaMemcpy(dx, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dsp, sp, sizeof(int) * n, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(dion, ion_x, sizeof(double) * 3, cudaMemcpyHostToDevice));
    CK(f64 ? reed_f64::launch_forces(P.tt, P, n, dx, dsp, dion, dout, dspill, smem, 0)
           : reed_f32::launch_forces(P.tt, P, n, dx, dsp, dion, dout, dspill, smem, 0));
    std::vector<double> h(6 + 3 * (size_t)n);
    CK(cudaMemcpy(h.data(), dout, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    for (int d = 0; d < 3; ++d) f_ion[d] = h[d];
    if (energy) *energy = h[3];
    if (rho) *rho = h[4];
    for (int i = 0; i < 3 * n; ++i) f_atoms[i] = h[5 + i];
    if (h[5 + 3 * (size_t)n] != 0.0)
        return fail(ctx, REED_E_NEIGHBOR, "%.0f neighbour-list entries did not fit: forces incomplete",
                    h[5 + 3 * (size_t)n]);
    return REED_OK;
}

int reed_window_replay(reed_ctx* ctx, int precision, uint64_t key, const double* path, int npts,
                       int32_t* anchors_out, int cap, int32_t* cells_out, int32_t* basis_out, double* xyz_out)
{
    if (!ctx || !path || npts < 1 || !anchors_out || cap < 0) return REED_E_ARG;
    DevParams P;
    reed_run_opts o = diag_opts();
    make_params(ctx, P, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, o);
    set_feedback(ctx, P, ctx->d_damage);
    const bool f64 = precision == REED_PREC_FP64;
    size_t smem = f64 ? reed_f64::smem_bytes(REED_TT_NONE, P.na, 0) : reed_f32::smem_bytes(REED_TT_NONE, P.na, 0);
    size_t bp = sizeof(double) * 3 * npts, ba = sizeof(int) * 3 * npts;
    size_t c = (size_t)std::max(cap, 1);
    size_t bc = sizeof(int) * 3 * c, bb = sizeof(int) * c, bx = sizeof(double) * 3 * c;
    void* s = nullptr;
    int rc;
    if ((rc = scratch(ctx, bp + ba + bc + bb + bx + 64, &s))) return rc;
    char* q = (char*)s;
    double* dpath = (double*)q;
    double* dxyz = (double*)(q + bp);
    int* danc = (int*)(q + bp + bx);
    int* dcells = danc + 3 * npts;
    int* dbas = dcells + 3 * c;
    int* dn = dbas + c;
    CK(cudaMemcpy(dpath, path, bp, cudaMemcpyHostToDevice));
    CK(f64 ? reed_f64::launch_window_replay(P, key, dpath, npts, danc, cap, dcells, dbas, dxyz, dn, smem, 0)
           : reed_f32::launch_window_replay(P, key, dpath, npts, danc, cap, dcells, dbas, dxyz, dn, smem, 0));
    int n = 0;
    CK(cudaMemcpy(&n, dn, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(anchors_out, danc, ba, cudaMemcpyDeviceToHost));
    int m = std::min(n, cap);
    if (m > 0) {
        CK(cudaMemcpy(cells_out, dcells, sizeof(int) * 3 * m, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(basis_out, dbas, sizeof(int) * m, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(xyz_out, dxyz, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost));
    }
    return n;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// reed_run_static: a run that allocates no device memory.
//
// The scratch of the stepper launch -- work counters, the primary queue head,
// the status word, the per-CTA clone stacks and neighbour-list overflow rows
// -- lives in the file-scope array below instead of context buffers.  It is
// part of this module's image: every GPU that loads the library holds it
// until the process exits.  Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in for the device copy); its device
// address belongs to one CUDA context, so it is looked up with
// cudaGetSymbolAddress once per device and context (set-up on the first call
// there) and cached under the context's unique id.
// ---------------------------------------------------------------------------
#include <mutex>

#define REED_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
#define REED_STATIC_HEADER 4096
#define REED_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_reed_static_scratch[REED_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mutex;
struct StaticSlot {
    unsigned long long ctx_id;   // unique id of the context the address belongs to (0: none yet)
    void* addr;
};
StaticSlot g_static[REED_STATIC_MAX_DEVICES] = {};

// driver entry points, resolved through the runtime (no link against the driver library)
typedef int (*CtxGetCurrentFn)(void** ctx);                          // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);         // cuCtxGetId
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
std::once_flag g_ctx_once;

// Unique id of the calling thread's current context (0 if none is current).
int current_context_id(unsigned long long* id)
{
    reed_ctx* ctx = nullptr;
    std::call_once(g_ctx_once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = (CtxGetIdFn)f;
    });
    if (!g_ctx_current || !g_ctx_id) return fail(ctx, REED_E_CUDA, "reed_run_static: driver context queries unavailable");
    void* c = nullptr;
    if (g_ctx_current(&c) != 0) return fail(ctx, REED_E_CUDA, "reed_run_static: cuCtxGetCurrent failed");
    *id = 0;
    if (c && g_ctx_id(c, id) != 0) return fail(ctx, REED_E_CUDA, "reed_run_static: cuCtxGetId failed");
    return REED_OK;
}

// Device address of the scratch array in the current device's current
// context: looked up on the first call in that context, then cached.
int static_scratch(void** out)
{
    reed_ctx* ctx = nullptr;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= REED_STATIC_MAX_DEVICES)
        return fail(nullptr, REED_E_ARG, "reed_run_static: device %d out of range", dev);
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticSlot& slot = g_static[dev];
    if (id == 0 || slot.ctx_id != id || !slot.addr) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_reed_static_scratch));   // makes the runtime's context current if none was
        if (id == 0 && (rc = current_context_id(&id))) return rc;
        slot.addr = p;
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return REED_OK;
}
}  // namespace

extern "C" int reed_run_static(const reed_lattice* lat, const reed_species* sp, int n_species,
                               const reed_potentials* pot, double ion_Z, double ion_M, double energy_eV,
                               double tilt_deg, double rot_deg_lo, double rot_deg_hi, int64_t n_ions, uint64_t seed,
                               const reed_run_opts* opt, double* hist_out, reed_stats_t* stats_out)
{
    reed_ctx* ctx = nullptr;   // errors go to the thread's init-error message
    if (!lat || !sp || !pot || !opt || !hist_out) return fail(nullptr, REED_E_ARG, "reed_run_static: null argument");
    const reed_run_opts& o = *opt;
    // the same checks as reed_init and reed_run
    if (lat->kind != REED_LATTICE_DIAMOND && lat->kind != REED_LATTICE_FLUORITE)
        return fail(nullptr, REED_E_ARG, "unknown lattice kind %d", lat->kind);
    if (lat->window_n < 2 || lat->window_n > 6) return fail(nullptr, REED_E_ARG, "window_n must be 2..6");
    if (lat->frozen_margin < 0 || 2 * lat->frozen_margin >= lat->window_n)
        return fail(nullptr, REED_E_ARG, "frozen_margin must be 0 or 1 and leave an integrated core");
    if (lat->target != REED_TARGET_SURFACE && lat->target != REED_TARGET_BULK)
        return fail(nullptr, REED_E_ARG, "unknown target geometry %d", lat->target);
    if (!(lat->a > 0.5) || !(lat->sigma >= 0.0)) return fail(nullptr, REED_E_ARG, "invalid lattice constant or sigma");
    if (n_species != (lat->kind == REED_LATTICE_FLUORITE ? 2 : 1))
        return fail(nullptr, REED_E_ARG, "wrong number of species");
    for (int s = 0; s < n_species; ++s)
        if (!(sp[s].Z > 0) || !(sp[s].M > 0)) return fail(nullptr, REED_E_ARG, "species %d: Z and M must be > 0", s);
    if (!(pot->rc > 0) || !(pot->r_taper >= 0) || !(pot->r_taper < pot->rc) || !(pot->lam_loc > 0))
        return fail(nullptr, REED_E_ARG, "invalid ion-target cutoff or density length");
    if (pot->target_model != REED_TT_NONE && pot->target_model != REED_TT_TERSOFF &&
        pot->target_model != REED_TT_BUCKINGHAM)
        return fail(nullptr, REED_E_ARG, "unknown target model %d", pot->target_model);
    if (pot->target_model == REED_TT_BUCKINGHAM && !(pot->buck_cut[1] > pot->buck_cut[0] && pot->buck_cut[0] >= 0))
        return fail(nullptr, REED_E_ARG, "Buckingham needs 0 <= taper start < cutoff");
    if (pot->target_model == REED_TT_TERSOFF && lat->kind != REED_LATTICE_DIAMOND)
        return fail(nullptr, REED_E_ARG, "Tersoff needs the one-species diamond lattice");
    if (!(ion_Z > 0) || !(ion_M > 0) || !(energy_eV > 0) || n_ions < 0)
        return fail(nullptr, REED_E_ARG, "ion Z, M, energy must be > 0 and n_ions >= 0");
    if (!(o.dt_max_fs > 0) || !(o.dx_max > 0) || !(o.e_stop >= 0) || o.step_cap < 1)
        return fail(nullptr, REED_E_ARG, "invalid integrator options");
    if (o.n_thresholds < 0 || o.n_thresholds > REED_MAX_THR) return fail(nullptr, REED_E_ARG, "n_thresholds must be 0..16");
    for (int i = 1; i < o.n_thresholds; ++i)
        if (!(o.thresholds[i] > o.thresholds[i - 1])) return fail(nullptr, REED_E_ARG, "thresholds must ascend");
    if (o.n_bins < 1 || !(o.bin_width > 0)) return fail(nullptr, REED_E_ARG, "invalid histogram");
    if (const char* m = beam_error(*lat, o)) return fail(nullptr, REED_E_ARG, "%s", m);
    if (o.precision != REED_PREC_MIXED && o.precision != REED_PREC_FP64) return fail(nullptr, REED_E_ARG, "precision");
    if (o.threads_per_track && !valid_threads(o.threads_per_track))
        return fail(nullptr, REED_E_ARG, "threads_per_track must be 0, 32, 64, 128, 256 or 512");
    if (o.ctas_per_sm < 0) return fail(nullptr, REED_E_ARG, "negative ctas_per_sm");
    if (o.record_tracks || o.trace_tracks || o.trace_steps)
        return fail(nullptr, REED_E_ARG, "reed_run_static keeps no per-track records or traces");
    if (o.adaptive || o.device_thresholds)
        return fail(nullptr, REED_E_ARG, "reed_run_static runs fixed cloning depths only");
    if (o.damage_n) return fail(nullptr, REED_E_ARG, "reed_run_static keeps no damage map");
    if (o.adjoint) return fail(nullptr, REED_E_ARG, "reed_run_static computes no sensitivities");

    // device parameters from a host-only description of the target
    reed_ctx desc;
    desc.lat = *lat;
    desc.nspec = n_species;
    for (int s = 0; s < n_species; ++s) desc.sp[s] = sp[s];
    desc.pot = *pot;
    desc.nbins = o.n_bins;
    desc.bin_w = o.bin_width;
    CK(cudaGetDevice(&desc.device));
    CK(cudaDeviceGetAttribute(&desc.sms, cudaDevAttrMultiProcessorCount, desc.device));
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, desc.device));
    DevParams P;
    make_params(&desc, P, ion_Z, ion_M, energy_eV, tilt_deg, rot_deg_lo, rot_deg_hi, o);
    P.seed = seed;
    P.n_primaries = n_ions;
    P.record = 0;
    P.trace_tracks = 0;
    P.trace_steps = 0;

    const int tt = P.tt;
    const bool f64 = o.precision == REED_PREC_FP64;
    const size_t smem = f64 ? reed_f64::smem_bytes(tt, P.na, P.bond_cap, 0, P.g_nbins, P.act_cap)
                            : reed_f32::smem_bytes(tt, P.na, P.bond_cap, 0, P.g_nbins, P.act_cap);
    if (smem > (size_t)optin)
        return fail(nullptr, REED_E_SMEM, "window of %d atoms needs %zu B of shared memory (max %d)", P.na, smem, optin);
    LaunchCfg L;
    L.threads = o.threads_per_track ? o.threads_per_track : (tt == REED_TT_NONE ? 64 : 256);
    L.smem = smem;
    int occ = 0;
    CK(f64 ? reed_f64::occupancy(tt, L.threads, smem, &occ, P.adjoint)
           : reed_f32::occupancy(tt, L.threads, smem, &occ, P.adjoint));
    if (occ < 1) return fail(nullptr, REED_E_SMEM, "kernel does not fit on an SM");
    L.ctas_per_sm = o.ctas_per_sm ? std::min(o.ctas_per_sm, occ) : occ;

    // clone stacks and overflow rows must fit in the static scratch: fewer
    // CTAs per SM if needed
    DevBuf B;
    std::memset(&B, 0, sizeof(B));
    B.entry_bytes = f64 ? reed_f64::entry_bytes(tt, P.na) : reed_f32::entry_bytes(tt, P.na);
    B.stack_depth = P.nthr;
    B.stack_stride = P.nthr > 0 ? B.entry_bytes * (size_t)P.nthr : 0;
    B.spill_stride = f64 ? reed_f64::spill_bytes(tt) : reed_f32::spill_bytes(tt);
    const size_t room = REED_STATIC_SCRATCH_BYTES - REED_STATIC_HEADER;
    const size_t per_cta = B.stack_stride + B.spill_stride;
    while (L.ctas_per_sm > 1 && per_cta * (size_t)desc.sms * L.ctas_per_sm > room) --L.ctas_per_sm;
    if (per_cta * (size_t)desc.sms * L.ctas_per_sm > room)
        return fail(nullptr, REED_E_ARG,
                    "clone stacks and list overflow rows need %zu B (%d SMs x (%d levels x %zu B + %zu B)), more "
                    "than the %zu B static scratch",
                    per_cta * (size_t)desc.sms, desc.sms, P.nthr, B.entry_bytes, B.spill_stride, room);
    L.grid = desc.sms * L.ctas_per_sm;

    unsigned char* base = nullptr;
    int rc = static_scratch((void**)&base);
    if (rc) return rc;
    B.counters = reinterpret_cast<unsigned long long*>(base);
    B.wsum = reinterpret_cast<double*>(base + 256);
    B.next = reinterpret_cast<unsigned long long*>(base + 512);
    B.status = reinterpret_cast<int*>(base + 768);
    B.record_count = reinterpret_cast<unsigned long long*>(base + 1024);
    B.finished = reinterpret_cast<unsigned long long*>(base + 1280);
    B.splits = reinterpret_cast<unsigned long long*>(base + 1536);
    B.thr = nullptr;
    B.damage = nullptr;
    P.stop_after = o.target_tracks;
    B.stacks = P.nthr > 0 ? base + REED_STATIC_HEADER : nullptr;
    B.spill = B.spill_stride ? base + REED_STATIC_HEADER + B.stack_stride * (size_t)L.grid : nullptr;
    B.hist = hist_out;
    B.records = nullptr;
    B.trace = nullptr;
    B.trace_anchor = nullptr;

    cudaStream_t st = (cudaStream_t)o.stream;
    // the array keeps the previous call's contents: clear what must start at zero
    CK(cudaMemsetAsync(base, 0, REED_STATIC_HEADER, st));
    CK(cudaMemsetAsync(hist_out, 0, sizeof(double) * (o.n_bins + 3), st));
    if (n_ions > 0) CK(f64 ? reed_f64::launch_track(tt, P, B, L, st) : reed_f32::launch_track(tt, P, B, L, st));
    CK(cudaStreamSynchronize(st));
    unsigned long long c[REED_NCOUNT];
    double w[4];
    int status = 0;
    CK(cudaMemcpy(c, B.counters, sizeof(c), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w, B.wsum, sizeof(w), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&status, B.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (stats_out) {
        std::memset(stats_out, 0, sizeof(*stats_out));
        stats_out->primaries = (int64_t)c[C_PRIMARIES];
        stats_out->clones = (int64_t)c[C_CLONES];
        stats_out->tracks = (int64_t)c[C_TRACKS];
        stats_out->steps = (int64_t)c[C_STEPS];
        stats_out->pair_evals = (int64_t)c[C_PAIRS];
        stats_out->bond_evals = (int64_t)c[C_BONDS];
        stats_out->shifts = (int64_t)c[C_SHIFTS];
        stats_out->rebuilds = (int64_t)c[C_REBUILDS];
        stats_out->dropped_clones = (int64_t)c[C_DROPPED];
        stats_out->nb_overflow = (int64_t)c[C_NBOVF];
        stats_out->bond_cap_overflow = (int64_t)c[C_CAPOVF];
        stats_out->nb_spilled = (int64_t)c[C_SPILLED];
        stats_out->list_refreshes = (int64_t)c[C_REFRESH];
        stats_out->nl_check_errors = (int64_t)c[C_NLCHECK];
        stats_out->failed = (int64_t)c[C_FAILED];
        stats_out->stopped = (int64_t)c[C_STOP];
        stats_out->backscattered = (int64_t)c[C_BACK];
        stats_out->truncated = (int64_t)c[C_TRUNC];
        stats_out->triplets = (int64_t)c[C_TRIPLETS];
        stats_out->atom_updates = (int64_t)c[C_MOVED];
        for (int k = 0; k < REED_NPHASE; ++k) stats_out->phase_cycles[k] = (int64_t)c[C_PHASE0 + k];
        for (int k = 0; k < 4; ++k) stats_out->centre_class[k] = (int64_t)c[C_CLS0 + k];
        unsigned long long sp[REED_MAX_THR + 1];
        CK(cudaMemcpy(sp, B.splits, sizeof(sp), cudaMemcpyDeviceToHost));
        for (int k = 0; k < REED_MAX_THR; ++k) stats_out->splits[k] = (int64_t)sp[k];
        stats_out->pooled = (int64_t)sp[REED_MAX_THR];
        stats_out->w_stopped = w[W_STOPPED];
        stats_out->w_back = w[W_BACK];
        stats_out->w_trunc = w[W_TRUNC];
        stats_out->threads_per_track = L.threads;
        stats_out->ctas_per_sm = L.ctas_per_sm;
        stats_out->grid = L.grid;
        stats_out->smem_bytes = (int32_t)L.smem;
    }
    if (status & ERR_NONFINITE) return fail(nullptr, REED_E_NONFINITE, "a track became non-finite");
    if (status & ERR_QUEUE) return fail(nullptr, REED_E_QUEUE_FULL, "clone stack overflow: clones dropped");
    if (status & ERR_NEIGHBOR)
        return fail(nullptr, REED_E_NEIGHBOR,
                    "a neighbour list outgrew its overflow row or the overflow rows ran out (see nb_overflow): "
                    "forces were incomplete");
    return REED_OK;
}
