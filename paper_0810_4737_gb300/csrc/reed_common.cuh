// reed_common.cuh -- device-side parameter block, buffers, math helpers and
// the counter-based random streams of the REED-MD track stepper.
//
// Units: Angstrom, eV, amu; time unit tau = sqrt(amu A^2/eV) = 10.1805 fs
// (the paper's Fig. "dt_E" quotes the time unit as 10.18 fs).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "reed.h"

#define REED_TAU_FS 10.180505710
#define REED_E2 14.399645       // e^2 / (4 pi eps0), eV A
#define REED_BOHR 0.529177      // A
#define REED_PI 3.14159265358979323846

#define REED_MAX_BASIS 12
#define REED_MAX_THR 16
#define REED_MAX_WARPS 16
#define REED_MAXNB 12           // Tersoff neighbours per atom held in shared memory
#define REED_MAXNB_PAIR 64      // pair-potential neighbours per atom held in shared memory
#define REED_FAST_NB 4          // Tersoff atoms with at most this many list neighbours take the unrolled path
#define REED_BF_STRIDE 13       // row stride of the per-bond force rows (odd: lanes hit distinct banks)
// An atom with more list neighbours than its shared-memory row holds keeps
// its whole list in an overflow row in global memory (per CTA, rebuilt with
// the lists); only beyond these limits is a run refused (REED_E_NEIGHBOR).
#define REED_SPILL_ROWS 32      // overflow rows per CTA
#define REED_SPILL_TERSOFF 64   // entries of a Tersoff overflow row
#define REED_SPILL_PAIR 192     // entries of a pair-list overflow row
#define REED_MAX_HOT 30         // Tersoff partial refresh: atoms whose lists one refresh recomputes
#define REED_MAX_STALE 128      // ... and atoms whose grid bins may be stale since the last full build

// neighbour-list capacity per atom in shared memory, and of an overflow row
__host__ __device__ constexpr int maxnb(int tt) { return tt == REED_TT_BUCKINGHAM ? REED_MAXNB_PAIR : REED_MAXNB; }
__host__ __device__ constexpr int spill_width(int tt)
{
    return tt == REED_TT_BUCKINGHAM ? REED_SPILL_PAIR : (tt == REED_TT_TERSOFF ? REED_SPILL_TERSOFF : 0);
}

// slot flags carried in pos.w (exact small integers in either precision):
//   w = species (0/1) for an integrated atom, species + 2 for a frozen atom,
//   -1 for an empty slot (cell above the surface).
#define REED_W_EMPTY (-1)

enum { REED_NCOUNT = 30 };
enum { REED_NRED = 9 };   // per-warp partial sums of a force pass
// cycle counters of the step phases (thread 0 of every CTA, summed)
enum { PH_ION = 0, PH_MOVE, PH_BUILD, PH_PASS1, PH_FORCE, PH_ADMIN, REED_NPHASE };
#define C_PHASE0 C_SPARE
enum {
    C_PRIMARIES = 0, C_CLONES, C_TRACKS, C_STEPS, C_PAIRS, C_BONDS, C_SHIFTS, C_REBUILDS,
    C_DROPPED, C_NBOVF, C_FAILED, C_STOP, C_BACK, C_TRUNC, C_CAPOVF, C_TRIPLETS, C_MOVED, C_SPILLED, C_REFRESH,
    C_NLCHECK, C_SPARE
};   // C_SPARE .. C_SPARE + REED_NPHASE - 1 hold the phase clocks, then C_CLS0 ..
     // C_CLS0 + 3 the Tersoff centre evaluations by class
#define C_CLS0 (C_SPARE + REED_NPHASE)
static_assert(C_CLS0 + 4 == REED_NCOUNT, "counter layout");
enum { W_STOPPED = 0, W_BACK, W_TRUNC, W_FAILED };

// Hot-loop parameters in the arithmetic type of the force pass (float for
// the mixed form, double for the plain FP64 path), so that no conversion is
// executed per pair.
template <typename R> struct HotParams {
    R a;                          // lattice constant
    R invM2[2];
    // ion-target
    R rc2, rt, inv_tw, zk[2], zia[2], lam_inv;
    R spline_c[6], spline_ctr[6], spline_invh;
    // Tersoff
    R tA, tB, tl1, tl2, tbn, tn, tmhn, tc2, td2, th, tRmD, tcut, tq, tdq, tR, tc2d2;
    R t_blo, t_binvw, t_zk, t_zia, rlist2, skin;
    R g_lo, g_inv;   // neighbour-search grid: low corner (anchor frame) and bins per A
    R de_max;        // energy term of the adaptive step (0 = off)
    R dx_min;        // shortest step of the fastest particle the energy term may impose
    // Buckingham
    R bA[3], brho_inv[3], bC[3], b_lo, b_binvw, b_rt, b_rinvw, b_rc2, b_zk[3], b_zia[3];
    // ion step
    R dt_max, dx_max, e_stop, M1, invM1, gamma, gamma0, s_loc, rho0_inv, anchor_lo, anchor_hi;
};

// Everything a launch needs, passed by value (__grid_constant__).
struct DevParams {
    HotParams<float> hf;
    HotParams<double> hd;
    // lattice and window (Sec. 2 "Second")
    int kind, n, margin, nb, na, nspec, half_n;   // half_n = n / 2
    int bulk;                                      // 1: infinite crystal, vacancy at the origin site
    int g_nb, g_nbins;                             // neighbour-search grid: bins per axis, in all
    // damage feedback: the cumulative map new cells read (null = off)
    const double* fb_map;
    int fb_n;
    double fb_vox, fb_half, fb_zhalf, fb_dose, fb_atoms, fb_ec, sigma_am;
    double a, inv_a, sigma, anchor_shift;          // anchor_shift = 0.5 for even n
    double bas[REED_MAX_BASIS][3];
    int bspec[REED_MAX_BASIS];
    double Z2[2], M2[2], invM2[2];
    // ion
    double Z1, M1, invM1;
    // ion-target ZBL with taper (Sec. 2 "First")
    double rc, rt, rc2, inv_tw;
    double zk[2], zia[2];           // Z1 Z2 e^2, 1/a_U per target species
    int spline_on;
    double spline_c[6], spline_ctr[6], spline_invh;   // B-spline weights, centres (ln r), 1/width
    // target-target
    int tt;
    double tA, tB, tl1, tl2, tbn, tn, tc2, td2, th, tR, tD, tcut, tc2d2;
    double t_blo, t_bhi, t_zk, t_zia;  // Tersoff->ZBL blend, Si-Si ZBL
    double bA[3], brho_inv[3], bC[3];
    double b_rt, b_rc, b_lo, b_hi;
    double b_zk[3], b_zia[3];
    int bond_cap;                      // neighbour-list rows (Tersoff: needed atoms)
    int nl_check;                      // compare every list with a brute-force search after each build
    int act_cap;                       // integrated atoms a window can hold (rows of the per-bond forces)
    // electronic stopping (Sec. 2 "Third")
    double gamma, s_loc, rho0_inv, lam_inv;
    int rho_on;
    // integrator (Sec. 2, Fig. "dt_E")
    double dt_max, dx_max, e_stop, de_max, dx_min;
    long long step_cap;
    long long pool_polls;   // polls of the clone pool by an idle CTA before it gives up
    // beam
    double v0, tilt, rot_lo, rot_span, cos_tmax;
    int beam_mode;
    // rare-event enhancement (Sec. 2)
    int nthr;
    double thr[REED_MAX_THR];
    int thr_from_device;               // read the depths from DevBuf::thr (adaptive epochs)
    // cumulative damage map: dn^3 voxels of dvox, origin (-dhalf, -dhalf, -dzhalf)
    // with dzhalf = 0 (surface target) or dhalf (bulk target)
    int dn;
    double dvox, dhalf, dzhalf, dmin;
    // truncated-segment adjoint: segment length, checkpoint spacing, ring size
    int adjoint, adj_seg, adj_every, adj_nck;
    long long stop_after;              // stop handing out primaries after this many tracks (0: never)
    // tallies
    int nbins;
    double bin_w;
    // run
    unsigned long long seed;
    long long n_primaries, first_id;
    int trace_tracks, trace_steps;
    int record;
    long long record_cap;
};

struct DevBuf {
    double* hist;                   // nbins + 3 (under, over, back)
    unsigned long long* counters;   // REED_NCOUNT
    unsigned long long* splits;     // clones made at each cloning level (REED_MAX_THR), then clones
                                    // taken from the pool; may be null
    // shared clone pool (may be null): CTAs that run out of work take clones
    // that busy CTAs donate while some CTA is idle
    unsigned char* pool;            // pool_slots x entry_bytes
    unsigned* pool_state;           // per slot: POOL_EMPTY / WRITING / FULL / READING
    unsigned* pool_ctl;             // [0] idle CTAs, [1] records reserved or held, [2] records published
    int pool_slots;
    double* wsum;                   // W_*
    unsigned long long* next;       // primary queue head
    reed_track_record* records;
    unsigned long long* record_count;
    double* trace;                  // trace_tracks * trace_steps * 8
    int* trace_anchor;              // trace_tracks * trace_steps * 3
    unsigned char* stacks;          // per-CTA clone stacks
    size_t stack_stride, entry_bytes;
    int stack_depth;
    int* status;                    // [0] OR of error bits
    const double* thr;              // cloning depths of this launch (adaptive epochs)
    double* damage;                 // dn^3 + 1 (overflow) voxels, or null
    unsigned char* adj;             // per-CTA adjoint scratch (checkpoints, steps, block states)
    size_t adj_stride;
    double* grads;                  // 8 per track record: dz/dtheta
    unsigned long long* finished;   // tracks finished in this run (stop rule)
    unsigned char* spill;           // per-CTA neighbour-list overflow rows (target models), or null
    size_t spill_stride;
};

enum { ERR_QUEUE = 1, ERR_NONFINITE = 2, ERR_NEIGHBOR = 4, ERR_TIMEOUT = 8 };

// ---------------------------------------------------------------------------
// Precision-generic vector and math helpers.  The FP32 forms use the SFU
// (ex2/lg2/rsqrt/sin/cos approximations of the PTX ISA); the FP64 forms call
// the CUDA double-precision functions.
// ---------------------------------------------------------------------------
template <typename R> struct alignas(16) V4 { R x, y, z, w; };

template <typename R> __device__ __forceinline__ const HotParams<R>& hot(const DevParams& P);
template <> __device__ __forceinline__ const HotParams<float>& hot<float>(const DevParams& P) { return P.hf; }
template <> __device__ __forceinline__ const HotParams<double>& hot<double>(const DevParams& P) { return P.hd; }

__device__ __forceinline__ float sfu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sfu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename R> struct Mth;
template <> struct Mth<float> {
    static constexpr float LOG2E = 1.4426950408889634f;
    __device__ static __forceinline__ float exp(float x) { return sfu_ex2(x * LOG2E); }
    // exp(-c x) with c already multiplied by log2(e)
    __device__ static __forceinline__ float exp2n(float x) { return sfu_ex2(x); }
    __device__ static __forceinline__ float rsqrt(float x) { return sfu_rsqrt(x); }
    __device__ static __forceinline__ float log(float x) { return sfu_lg2(x) * 0.6931471805599453f; }
    __device__ static __forceinline__ float pow(float x, float y) { return sfu_ex2(y * sfu_lg2(x)); }
    __device__ static __forceinline__ float sin(float x) { return __sinf(x); }
    __device__ static __forceinline__ float cos(float x) { return __cosf(x); }
    __device__ static __forceinline__ float rcp(float x) { return sfu_rcp(x); }
};
template <> struct Mth<double> {
    static constexpr double LOG2E = 1.4426950408889634;
    __device__ static __forceinline__ double exp(double x) { return ::exp(x); }
    __device__ static __forceinline__ double exp2n(double x) { return ::exp2(x); }
    __device__ static __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    __device__ static __forceinline__ double log(double x) { return ::log(x); }
    __device__ static __forceinline__ double pow(double x, double y) { return ::pow(x, y); }
    __device__ static __forceinline__ double sin(double x) { return ::sin(x); }
    __device__ static __forceinline__ double cos(double x) { return ::cos(x); }
    __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
};

// ---------------------------------------------------------------------------
// Counter-based random streams.
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products with multipliers 0xD2511F53 / 0xCD9E8D57, key
// bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        uint32_t a0 = hi1 ^ c[1] ^ k0, a2 = hi0 ^ c[3] ^ k1;
        c[0] = a0; c[1] = lo1; c[2] = a2; c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) used to derive stream keys.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Philox key of track `id` under `seed`.
__host__ __device__ __forceinline__ uint64_t track_key(uint64_t seed, uint64_t id)
{
    return mix64(seed + 0x9E3779B97F4A7C15ull * (id + 1ull));
}
// Id of the clone a track spawns when it passes cloning level `level`.
__host__ __device__ __forceinline__ uint64_t clone_id(uint64_t parent, int level)
{
    return mix64(parent ^ (0xD1B54A32D192ED03ull * (uint64_t)(level + 1)));
}

#define REED_TAG_CELL 1u
#define REED_TAG_LAUNCH 2u
#define REED_TAG_DAMAGE 3u

__device__ __forceinline__ void draw4(uint64_t key, int ix, int iy, int iz, uint32_t word, uint32_t out[4])
{
    out[0] = (uint32_t)ix; out[1] = (uint32_t)iy; out[2] = (uint32_t)iz; out[3] = word;
    philox10(out, (uint32_t)key, (uint32_t)(key >> 32));
}

__device__ __forceinline__ double unit_open(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

// Three normals from one Philox block by the Box-Muller transform.
__device__ __forceinline__ void box_muller3(const uint32_t w[4], double g[3])
{
    double r1 = sqrt(-2.0 * log(unit_open(w[0])));
    double r2 = sqrt(-2.0 * log(unit_open(w[2])));
    double s1, c1, c2;
    sincospi(2.0 * unit_open(w[1]), &s1, &c1);
    c2 = cospi(2.0 * unit_open(w[3]));
    g[0] = r1 * c1;
    g[1] = r1 * s1;
    g[2] = r2 * c2;
}

// The same three normals in FP32 (the mixed form's thermal offsets; FP64
// transcendentals are slow on this part).  -ln u is taken from 1 - u when u
// is near 1 so that small radii keep their relative accuracy.
__device__ __forceinline__ float neg_log_unit(uint32_t w)
{
    if (w >= 0x80000000u) {
        const float e = ((float)(0xFFFFFFFFu - w) + 0.5f) * 2.3283064365386963e-10f;   // 1 - u
        return -log1pf(-e);
    }
    return -logf(((float)w + 0.5f) * 2.3283064365386963e-10f);
}

__device__ __forceinline__ void box_muller3f(const uint32_t w[4], float g[3])
{
    const float r1 = sqrtf(2.0f * neg_log_unit(w[0]));
    const float r2 = sqrtf(2.0f * neg_log_unit(w[2]));
    float s1, c1;
    sincospif(2.0f * (((float)w[1] + 0.5f) * 2.3283064365386963e-10f), &s1, &c1);
    const float c2 = cospif(2.0f * (((float)w[3] + 0.5f) * 2.3283064365386963e-10f));
    g[0] = r1 * c1;
    g[1] = r1 * s1;
    g[2] = r2 * c2;
}

// ---------------------------------------------------------------------------
// Warp reductions (fixed butterfly order: results are reproducible).
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
