// reed_track.cuh -- the persistent REED-MD track stepper.
//
// One CTA owns one ion track at a time.  The track's window of n^3 unit cells
// (Sec. 2 "Second", Fig. "moving cell") lives in shared memory in a ring
// layout: the atom of basis b in the cell whose absolute index is c sits in
// slot ((c_x mod n) n + (c_y mod n)) n + (c_z mod n)) * nb + b, so a window
// move rewrites only the n^2 cells of one face.  Atom coordinates are kept
// relative to the corner of the anchor cell (the ion's cell for odd n, its
// nearest cell corner for even n) and re-based when the anchor moves; the
// ion itself is kept in absolute FP64 coordinates.
//
// A CTA takes primaries from a device counter (the paper's host hands out
// ions, Sec. 3).  When a track first passes a cloning depth (Sec. 2, Fig.
// "split") its complete state is pushed onto the CTA's own stack in global
// memory and the track continues with half the weight; the clone is run by
// the same CTA when the track ends (depth first, so the stack never holds
// more entries than there are cloning depths and no CTA ever waits on
// another).  Results go straight into device tallies with atomics (the
// paper's result messages, Sec. 3).
//
// One step (kick-drift-kick with adaptive dt, Sec. 2):
//   prologue  (thread 0, FP64) dt from the fastest particle, ion half kick +
//             drift, window anchor check;
//   phase A   (all threads) re-anchor moved cells, atom half kick + drift;
//   forces    (all threads) ion-target ZBL, target-target terms, second half
//             kick of the atoms, per-warp partial sums;
//   epilogue  (thread 0) ion force reduction, ion second half kick, end /
//             cloning checks, then straight into the next prologue.
#pragma once

#include "reed_physics.cuh"

enum { SRC_NONE = 0, SRC_PRIMARY = 1, SRC_CLONE = 2, SRC_STOLEN = 3 };
enum { POOL_EMPTY = 0, POOL_WRITING = 1, POOL_FULL = 2, POOL_READING = 3 };

enum { EV_NONE = 0, EV_END = 1, EV_CLONE = 2, EV_CKPT = 3 };

// Ion state as stored in shared memory and in clone records.  Position,
// time and the energy given to electronic stopping are FP64 accumulators;
// velocity, force and the step arithmetic are in the force-pass type R, so
// the mixed form executes only a handful of FP64 additions per step.
template <typename R> struct alignas(16) IonState {
    double x[3];          // absolute position, A
    double t, e_elec;     // time (tau), energy removed by the drag (eV)
    R v[3], f[3];         // velocity (A/tau), conservative force (eV/A)
    R vlo[3];             // FP32 form: the rounding error carried with v (v + vlo, see add_velocity)
    R rho, vmax2;         // local density at x; fastest atom's speed^2
    R pmax;               // largest |F . v| over the integrated atoms (energy term of dt)
    long long steps;
    unsigned long long id, primary, key;
    int A[3];
    int level;
};

template <typename R> struct TrackShared {
    IonState<R> ion;
    R dt;
    R rel[3];             // ion position relative to the anchor corner A a
    R zthr, zback, zsurf; // next cloning depth, backscatter plane, surface in the anchor frame
    double thr[REED_MAX_THR];  // this track's cloning depths (frozen while it runs)
    int nthr;
    // adjoint workspace
    int on1, on2;
    long long rec_index;
    R xbi[3], vbi[3], ubi[3], vh[3], irel[3], vub, k1;
    double gth[8];
    R adj_red[REED_MAX_WARPS][12];
    int Aold[3];
    int shift, event, status, src, top, nclone, slot;
    int need_count, active_count;
    int nspill;           // overflow rows taken by the current lists
    int ncls[4];          // Tersoff: slots per centre-pass class, in `order` (see ters_centres)
    unsigned long long cls_sum[4];   // centre evaluations per class, summed over passes (thread 0)
    // Tersoff partial refreshes: atoms whose bins are stale since the last
    // full build (atom order), and the atoms refreshed now
    int nstale, nhot;
    uint16_t stale[REED_MAX_STALE];
    uint16_t hot[REED_MAX_HOT];
    int scan[4][REED_MAX_WARPS];
    long long pidx;
    R red[REED_MAX_WARPS][REED_NRED];
    R path2[REED_MAX_WARPS][2];   // per warp: the two longest atom paths since the list build
};

template <typename R> struct V2 { R a, b; };

// Shared-memory carve-up for a window of na atoms.  Target neighbour lists
// are kept only for "needed" atoms -- integrated atoms (slots 0 ..
// active_count-1) and, for Tersoff, the atoms bonded to them -- at most cap
// of them, addressed through need_map (atom -> slot) and slot_atom.  The
// neighbour search bins atoms on a grid of nbins cells (bin_count is all
// zero between builds).  Tersoff adds, per list entry, the position of the
// centre in the neighbour's own list (rev), the order in which the centre
// pass visits the slots, and for each integrated atom (at most act of them)
// one force row: entry q holds the force that the bonds centred on its q-th
// neighbour exert on it.

template <typename R, int TT> struct Layout {
    static __host__ __device__ size_t align(size_t x) { return (x + 15) & ~(size_t)15; }
    static __host__ __device__ size_t shared_bytes() { return align(sizeof(TrackShared<R>)); }
    static __host__ __device__ size_t atoms_bytes(int na) { return 3 * align(sizeof(V4<R>) * na); }
    static __host__ __device__ size_t nbr_bytes(int na, int cap, int nbins)
    {
        if (TT == REED_TT_NONE) return 0;
        return align(sizeof(uint16_t) * na) +            // need_map
               align(sizeof(uint16_t) * na) +            // binned (atoms in bin order)
               align(sizeof(uint16_t) * (nbins + 1)) +   // bin_start
               align(sizeof(unsigned) * nbins) +         // bin_count
               align(sizeof(uint16_t) * cap) +           // slot_atom
               align(cap) +                              // nnb
               align(sizeof(uint16_t) * cap * maxnb(TT));     // nbr
    }
    static __host__ __device__ size_t bond_bytes(int cap, int act, int na = 0)
    {
        if (TT != REED_TT_TERSOFF) return 0;
        return 2 * align(sizeof(unsigned) * (size_t)((na + 31) / 32)) + // stale and hot bits
               align(sizeof(unsigned) * (size_t)cap) +                 // refresh marks per slot
               align((size_t)cap * REED_MAXNB) +                       // rev
               align(sizeof(uint16_t) * cap) +                         // order
               3 * align(sizeof(R) * (size_t)act * REED_BF_STRIDE);    // per-bond forces (x, y, z)
    }
    static __host__ __device__ size_t adj_bytes(int na, int adj) { return adj ? 2 * align(sizeof(V4<R>) * na) : 0; }
    static __host__ __device__ size_t total(int na, int cap, int adj = 0, int nbins = 0, int act = 0)
    {
        return shared_bytes() + atoms_bytes(na) + nbr_bytes(na, cap, nbins) + bond_bytes(cap, act, na) +
               adj_bytes(na, adj);
    }
    // bytes of one clone record: ion header + pos, vel, frc
    static __host__ __device__ size_t entry_bytes(int na) { return align(sizeof(IonState<R>)) + atoms_bytes(na); }
    // per-CTA overflow rows in global memory: neighbours (and, for Tersoff,
    // the reverse entries and the per-bond forces of an integrated atom)
    static __host__ __device__ size_t spill_bytes()
    {
        constexpr size_t W = (size_t)spill_width(TT), N = REED_SPILL_ROWS;
        if (TT == REED_TT_NONE) return 0;
        size_t b = align(sizeof(uint16_t) * N * W);
        if (TT == REED_TT_TERSOFF) b += align(N * W) + align(sizeof(R) * 3 * N * W);
        return b;
    }
};

#define REED_NO_SLOT 0xFFFFu
#define REED_PENDING 0xFFFEu
#define REED_NO_REV 0xFFu

template <typename R, int TT> struct Win {
    TrackShared<R>* S;
    V4<R>* pos;
    V4<R>* vel;
    V4<R>* frc;
    uint16_t* need_map;   // atom -> list slot
    uint16_t* binned;     // present atoms in bin order (atom order inside a bin)
    uint16_t* bin_start;  // bin -> first entry in binned (nbins + 1)
    unsigned* bin_count;  // scratch of the build, zero between builds
    uint16_t* slot_atom;  // list slot -> atom
    uint8_t* nnb;         // neighbours per slot
    uint16_t* nbr;        // neighbour atoms per slot
    unsigned* sbits;      // Tersoff: atoms whose grid bin is stale (one bit each)
    unsigned* hbits;      // Tersoff: atoms refreshed by the current partial refresh
    unsigned* tmask;      // Tersoff refresh, per slot: bit 31 = row rebuilt or loses a hot atom, bit t < 30 =
                          //   gains hot atom t, bit 30 = lists a changed row
    uint8_t* rev;         // Tersoff: per slot and neighbour, the centre's entry in the neighbour's list
    uint16_t* order;      // Tersoff: slots in the order the centre pass takes them
    R* bfx;               // Tersoff: per integrated slot and list entry, the force of the
    R* bfy;               //   bonds centred on that neighbour (row stride REED_BF_STRIDE)
    R* bfz;
    uint16_t* sp_nbr;     // overflow rows in global memory (may be null)
    uint8_t* sp_rev;
    R* sp_bf;             // x, y, z blocks of REED_SPILL_TERSOFF per row
    V4<R>* xbar;          // adjoint of positions (adjoint runs)
    V4<R>* vbar;          // adjoint of velocities
    // Neighbour q of list slot k is nbr[k * nb_slot + q * nb_q]: slot-major for
    // Tersoff (a thread walks its own short list), neighbour-major for the
    // 64-entry pair lists (consecutive slots, i.e. lanes, hit consecutive words).
    // A slot with more neighbours than the shared row holds keeps its whole
    // list in an overflow row; entry 0 of the shared row is then that row's index.
    int nb_slot, nb_q, act_cap;
    // zero the bin counters (all threads; a barrier must follow)
    __device__ void clear_grid(const DevParams& P)
    {
        if (bin_count)
            for (int b = threadIdx.x; b < P.g_nbins; b += blockDim.x) bin_count[b] = 0u;
    }
    __device__ Win(unsigned char* base, int na, int cap, int adj = 0, int nbins = 0, int act = 0,
                   unsigned char* spill = nullptr)
        : nb_slot(TT == REED_TT_BUCKINGHAM ? 1 : maxnb(TT)), nb_q(TT == REED_TT_BUCKINGHAM ? cap : 1), act_cap(act)
    {
        using L = Layout<R, TT>;
        S = reinterpret_cast<TrackShared<R>*>(base);
        size_t o = L::shared_bytes();
        size_t ab = L::align(sizeof(V4<R>) * na);
        pos = reinterpret_cast<V4<R>*>(base + o);
        vel = reinterpret_cast<V4<R>*>(base + o + ab);
        frc = reinterpret_cast<V4<R>*>(base + o + 2 * ab);
        o += 3 * ab;
        need_map = nullptr;
        binned = nullptr;
        bin_start = nullptr;
        bin_count = nullptr;
        slot_atom = nullptr;
        nnb = nullptr;
        nbr = nullptr;
        sbits = hbits = tmask = nullptr;
        rev = nullptr;
        order = nullptr;
        bfx = bfy = bfz = nullptr;
        sp_nbr = nullptr;
        sp_rev = nullptr;
        sp_bf = nullptr;
        if constexpr (TT != REED_TT_NONE) {
            need_map = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * na);
            binned = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * na);
            bin_start = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * (nbins + 1));
            bin_count = reinterpret_cast<unsigned*>(base + o);
            o += L::align(sizeof(unsigned) * nbins);
            slot_atom = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * cap);
            nnb = base + o;
            o += L::align(cap);
            nbr = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * cap * maxnb(TT));
            if (spill) sp_nbr = reinterpret_cast<uint16_t*>(spill);
        }
        if constexpr (TT == REED_TT_TERSOFF) {
            const size_t bw = L::align(sizeof(unsigned) * (size_t)((na + 31) / 32));
            sbits = reinterpret_cast<unsigned*>(base + o);
            hbits = reinterpret_cast<unsigned*>(base + o + bw);
            o += 2 * bw;
            tmask = reinterpret_cast<unsigned*>(base + o);
            o += L::align(sizeof(unsigned) * (size_t)cap);
            rev = base + o;
            o += L::align((size_t)cap * REED_MAXNB);
            order = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * cap);
            const size_t fb = L::align(sizeof(R) * (size_t)act * REED_BF_STRIDE);
            bfx = reinterpret_cast<R*>(base + o);
            bfy = reinterpret_cast<R*>(base + o + fb);
            bfz = reinterpret_cast<R*>(base + o + 2 * fb);
            o += 3 * fb;
            if (spill) {
                constexpr size_t W = REED_SPILL_TERSOFF, N = REED_SPILL_ROWS;
                sp_rev = spill + L::align(sizeof(uint16_t) * N * W);
                sp_bf = reinterpret_cast<R*>(spill + L::align(sizeof(uint16_t) * N * W) + L::align(N * W));
            }
        }
        xbar = vbar = nullptr;
        if (adj) {
            xbar = reinterpret_cast<V4<R>*>(base + o);
            vbar = reinterpret_cast<V4<R>*>(base + o + L::align(sizeof(V4<R>) * na));
        }
    }
    // list of slot k with m entries: its shared row, or its overflow row
    __device__ __forceinline__ const uint16_t* list(int k, int m) const
    {
        return m <= maxnb(TT) ? nbr + (size_t)k * nb_slot : sp_nbr + (size_t)nbr[(size_t)k * nb_slot] * spill_width(TT);
    }
    __device__ __forceinline__ uint8_t* rev_row(int k, int m) const
    {
        return m <= REED_MAXNB ? rev + (size_t)k * REED_MAXNB : sp_rev + (size_t)nbr[(size_t)k * REED_MAXNB] * REED_SPILL_TERSOFF;
    }
    // force of the bonds centred on entry e's atom on the integrated atom of slot s
    __device__ __forceinline__ void bf_store(int s, int e, R fx, R fy, R fz) const
    {
        if (nnb[s] <= REED_MAXNB) {
            const int o = s * REED_BF_STRIDE + e;
            bfx[o] = fx;
            bfy[o] = fy;
            bfz[o] = fz;
        } else {
            R* b = sp_bf + (size_t)nbr[(size_t)s * REED_MAXNB] * 3 * REED_SPILL_TERSOFF;
            b[e] = fx;
            b[REED_SPILL_TERSOFF + e] = fy;
            b[2 * REED_SPILL_TERSOFF + e] = fz;
        }
    }
};

__device__ __forceinline__ int pmod(int x, int n)
{
    int r = x % n;
    return r < 0 ? r + n : r;
}

// slot coordinates of atom slot i
__device__ __forceinline__ void slot_coords(const DevParams& P, int i, int s[3], int& b)
{
    b = i % P.nb;
    int cell = i / P.nb;
    s[2] = cell % P.n;
    s[1] = (cell / P.n) % P.n;
    s[0] = cell / (P.n * P.n);
}

// Create the atom of slot i for a window anchored at A (Sec. 2: new cells
// are a perfect lattice plus a statistical realisation; Sec. 4.1: Gaussian
// thermal displacements).  Cells with z index < 0 are above the surface of a
// surface target; a bulk target fills space and lacks the atom of the site
// the recoil starts from (basis atom 0 of cell (0,0,0)).
template <typename R>
__device__ void make_atom(const DevParams& P, uint64_t key, int i, const int A[3], V4<R>& p, V4<R>& v)
{
    int s[3], b;
    slot_coords(P, i, s, b);
    int c[3], active = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int L = A[d] - P.half_n;
        int o = pmod(s[d] - L, P.n);
        c[d] = L + o;
        if (o < P.margin || o > P.n - 1 - P.margin) active = 0;
    }
    v.x = v.y = v.z = v.w = R(0);
    if (P.bulk ? (b == 0 && c[0] == 0 && c[1] == 0 && c[2] == 0) : c[2] < 0) {
        p.x = p.y = p.z = R(0);
        p.w = R(REED_W_EMPTY);
        return;
    }
    // damage feedback (reading of the paper's cumulative damage feedback):
    // the cell is amorphous, with the wider offsets, with probability
    // 1 - exp(-e / e_crit), e = dose * D / N for the map's voxel D holding
    // the cell's centre and N lattice atoms per voxel
    double sig = P.sigma;
    if (P.fb_map) {
        const double cc[3] = {(c[0] + 0.5) * P.a + P.fb_half, (c[1] + 0.5) * P.a + P.fb_half,
                              (c[2] + 0.5) * P.a + P.fb_zhalf};
        int vv[3];
        bool in = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vv[d] = (int)floor(cc[d] / P.fb_vox);
            in = in && vv[d] >= 0 && vv[d] < P.fb_n;
        }
        if (in) {
            const double D = P.fb_map[((size_t)vv[0] * P.fb_n + vv[1]) * P.fb_n + vv[2]];
            const double e = P.fb_dose * D / P.fb_atoms;
            const double pam = 1.0 - exp(-e / P.fb_ec);
            uint32_t w[4];
            draw4(key, c[0], c[1], c[2], REED_TAG_DAMAGE, w);
            if (unit_open(w[0]) < pam) sig = P.sigma_am;
        }
    }
    double g[3] = {0.0, 0.0, 0.0};
    if (sig > 0.0) {
        uint32_t w[4];
        draw4(key, c[0], c[1], c[2], ((uint32_t)b << 4) | REED_TAG_CELL, w);
        if constexpr (sizeof(R) == 4) {
            float gf[3];
            box_muller3f(w, gf);
            g[0] = gf[0];
            g[1] = gf[1];
            g[2] = gf[2];
        } else {
            box_muller3(w, g);
        }
    }
    p.x = R(((double)(c[0] - A[0]) + P.bas[b][0]) * P.a + sig * g[0]);
    p.y = R(((double)(c[1] - A[1]) + P.bas[b][1]) * P.a + sig * g[1]);
    p.z = R(((double)(c[2] - A[2]) + P.bas[b][2]) * P.a + sig * g[2]);
    p.w = R(P.bspec[b] + (active ? 0 : 2));
}

// Move slot i from a window anchored at Aold to one anchored at Anew: if its
// cell is still inside, re-base the coordinates (and update the frozen flag),
// else replace it by the atom of the cell that entered the window.
template <typename R>
__device__ __forceinline__ bool reanchor_atom(const DevParams& P, const HotParams<R>& H, uint64_t key, int i,
                                              const int Aold[3], const int Anew[3], V4<R>& p, V4<R>& v,
                                              V4<R>& f)
{
    int s[3], b;
    slot_coords(P, i, s, b);
    bool keep = true;
    int active = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int Lo = Aold[d] - P.half_n;
        int c = Lo + pmod(s[d] - Lo, P.n);
        int on = c - (Anew[d] - P.half_n);
        if (on < 0 || on >= P.n) keep = false;
        if (on < P.margin || on > P.n - 1 - P.margin) active = 0;
    }
    if (!keep) {
        make_atom<R>(P, key, i, Anew, p, v);
        f.x = f.y = f.z = f.w = R(0);
        return true;
    }
    if (p.w < R(0)) return false;
    p.x -= R(Anew[0] - Aold[0]) * H.a;
    p.y -= R(Anew[1] - Aold[1]) * H.a;
    p.z -= R(Anew[2] - Aold[2]) * H.a;
    int sp = ((int)p.w) & 1;
    p.w = R(sp + (active ? 0 : 2));
    return false;
}

template <typename R> __device__ __forceinline__ bool is_present(const V4<R>& p) { return p.w >= R(0); }
template <typename R> __device__ __forceinline__ int species_of(const V4<R>& p);

// Cumulative damage (reading of the paper's shared damage information): an
// atom leaving the simulation -- its cell dropped, or the track ended --
// deposits w * KE into the voxel holding it when KE > dmin.  p is relative to
// the anchor A.
template <typename R>
__device__ __forceinline__ void deposit_damage(const DevParams& P, const DevBuf& B, const V4<R>& p, const V4<R>& v,
                                               const int A[3], double w)
{
    if (!B.damage || p.w < R(0)) return;
    const double ke = 0.5 * P.M2[((int)p.w) & 1] * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
    if (!(ke > P.dmin)) return;
    const double x = (double)p.x + (double)A[0] * P.a, y = (double)p.y + (double)A[1] * P.a,
                 z = (double)p.z + (double)A[2] * P.a;
    const int ix = (int)floor((x + P.dhalf) / P.dvox), iy = (int)floor((y + P.dhalf) / P.dvox),
              iz = (int)floor((z + P.dzhalf) / P.dvox);
    const size_t n = (size_t)P.dn;
    size_t cell = n * n * n;   // overflow
    if (ix >= 0 && iy >= 0 && iz >= 0 && ix < P.dn && iy < P.dn && iz < P.dn) cell = ((size_t)ix * n + iy) * n + iz;
    atomicAdd(&B.damage[cell], w * ke);
}
template <typename R> __device__ __forceinline__ bool is_active(const V4<R>& p) { return p.w >= R(0) && p.w < R(2); }
template <typename R> __device__ __forceinline__ int species_of(const V4<R>& p) { return ((int)p.w) & 1; }

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Target neighbour lists.  Rebuilt at track start, after a window move and
// when the two longest atom paths since the last build add up to more than
// the skin (a pair can then have closed in from beyond the list radius).
// Candidates come from a grid over the window whose bins are at least one
// list radius wide: atoms closer than that sit in the same or adjacent bins.
// Bin indices are clamped to the grid, which keeps that property for atoms
// that have left the window's volume.  Inside a bin atoms are kept in atom
// order, so lists do not depend on thread timing.
// Integrated atoms get list slots first; atoms bonded to them next.
// Called by all threads right after a barrier; ends with a barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int floor_int(float x) { return __float2int_rd(x); }
__device__ __forceinline__ int floor_int(double x) { return __double2int_rd(x); }

template <typename R>
__device__ __forceinline__ int grid_axis(const DevParams& P, const HotParams<R>& H, R x)
{
    return min(max(floor_int((x - H.g_lo) * H.g_inv), 0), P.g_nb - 1);
}

template <typename R>
__device__ __forceinline__ int grid_bin(const DevParams& P, const HotParams<R>& H, const V4<R>& p)
{
    return (grid_axis<R>(P, H, p.x) * P.g_nb + grid_axis<R>(P, H, p.y)) * P.g_nb + grid_axis<R>(P, H, p.z);
}

// Squared distance in a fixed operation order (no contraction), so that a
// pair's list test gives the same answer from both ends in every list
// builder: the lists are symmetric.
__device__ __forceinline__ float list_d2(const V4<float>& a, const V4<float>& b)
{
    const float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}
__device__ __forceinline__ double list_d2(const V4<double>& a, const V4<double>& b)
{
    const double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y), dz = __dsub_rn(b.z, a.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ bool bit_of(const unsigned* b, int i) { return (b[i >> 5] >> (i & 31)) & 1u; }

// Appends neighbours to the list of one slot: the shared row, then -- past
// its capacity -- a whole overflow row in global memory; past that, entries
// are dropped and counted in `overflow` (which fails the run).
template <typename R, int TT> struct ListWriter {
    uint16_t* out;
    int oq;
    uint16_t* sp = nullptr;
    bool asked = false;
    int cnt = 0;
    __device__ ListWriter(Win<R, TT>& W, int slot) : out(W.nbr + (size_t)slot * W.nb_slot), oq(W.nb_q) {}
    __device__ __forceinline__ void add(Win<R, TT>& W, int j, int& overflow)
    {
        constexpr int NS = maxnb(TT), NW = spill_width(TT);
        if (cnt < NS) {
            out[(size_t)cnt * oq] = (uint16_t)j;
            ++cnt;
            return;
        }
        if (!asked && W.sp_nbr) {
            asked = true;
            const int r = atomicAdd(&W.S->nspill, 1);
            if (r < REED_SPILL_ROWS) {
                sp = W.sp_nbr + (size_t)r * NW;
                for (int e = 0; e < NS; ++e) sp[e] = out[(size_t)e * oq];
                out[0] = (uint16_t)r;
            }
        }
        if (sp && cnt < NW) {
            sp[cnt] = (uint16_t)j;
            ++cnt;
        } else {
            ++overflow;
        }
    }
};

// Neighbours of atom i within the list radius, in bin order, into list slot
// `slot`.  Past the shared row's capacity the list moves to an overflow row
// in global memory; past that row's capacity (or with no row left) the
// entries are dropped and counted in `overflow`, which fails the run.
// MODE 0: every atom; atoms whose bins are stale (Tersoff partial refreshes)
// are skipped in the bins and tested from the stale set instead.  MODE 1
// (lists of atoms that became needed in a partial refresh): frozen atoms from
// the bins, then the atoms being refreshed.
template <typename R, int TT, int MODE = 0>
__device__ __forceinline__ int list_of(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int i, int slot,
                                      int& overflow)
{
    const V4<R> pi = W.pos[i];
    ListWriter<R, TT> L(W, slot);
    bool skip_stale = false;
    if constexpr (TT == REED_TT_TERSOFF) skip_stale = MODE == 0 && W.S->nstale > 0;
    const int nb = P.g_nb;
    const int bx = grid_axis<R>(P, H, pi.x), by = grid_axis<R>(P, H, pi.y), bz = grid_axis<R>(P, H, pi.z);
    const int z0 = max(bz - 1, 0), z1 = min(bz + 1, nb - 1);
    // (candidates are read four at a time so that their loads overlap: the
    // search is bound by shared-memory latency, not by arithmetic)
    for (int cx = max(bx - 1, 0); cx <= min(bx + 1, nb - 1); ++cx) {
        for (int cy = max(by - 1, 0); cy <= min(by + 1, nb - 1); ++cy) {
            // bins z0..z1 of one (x, y) column are consecutive in binned[]
            const int col = (cx * nb + cy) * nb;
            const int q1 = W.bin_start[col + z1 + 1];
            for (int q0 = W.bin_start[col + z0]; q0 < q1; q0 += 4) {
                int jj[4];
                V4<R> pp[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) jj[u] = q0 + u < q1 ? (int)W.binned[q0 + u] : i;
#pragma unroll
                for (int u = 0; u < 4; ++u) pp[u] = W.pos[jj[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = jj[u];
                    if (j == i) continue;
                    const V4<R> pj = pp[u];
                    if (MODE == 1 && is_active(pj)) continue;
                    if (skip_stale && bit_of(W.sbits, j)) continue;
                    if (!(list_d2(pi, pj) < H.rlist2)) continue;
                    L.add(W, j, overflow);
                    if (TT == REED_TT_TERSOFF && !is_active(pj) && W.need_map[j] == REED_NO_SLOT)
                        W.need_map[j] = (uint16_t)REED_PENDING;
                }
            }
        }
    }
    if constexpr (TT == REED_TT_TERSOFF) {
        const int ns = MODE == 0 ? (skip_stale ? W.S->nstale : 0) : W.S->nhot;
        const uint16_t* set = MODE == 0 ? W.S->stale : W.S->hot;
        for (int t = 0; t < ns; ++t) {
            const int j = set[t];
            if (j == i) continue;
            const V4<R> pj = W.pos[j];
            if (!(list_d2(pi, pj) < H.rlist2)) continue;
            L.add(W, j, overflow);
            if (!is_active(pj) && W.need_map[j] == REED_NO_SLOT) W.need_map[j] = (uint16_t)REED_PENDING;
        }
    }
    return L.cnt;
}

// The same search by one warp (all 32 lanes call it with the same i; Tersoff
// lists): lanes take the candidates in the order list_of visits them (bin
// columns, then the stale or hot set), ballots keep that order.  Used where
// a few lists are built while the rest of the CTA waits.  An overflow row
// the slot held before is reused.
template <typename R, int TT, int MODE>
__device__ int list_of_warp(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int i, int slot, int& overflow)
{
    constexpr int NS = REED_MAXNB, NW = REED_SPILL_TERSOFF;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const V4<R> pi = W.pos[i];
    const bool skip_stale = MODE == 0 && W.S->nstale > 0;
    const int nb = P.g_nb;
    const int bx = grid_axis<R>(P, H, pi.x), by = grid_axis<R>(P, H, pi.y), bz = grid_axis<R>(P, H, pi.z);
    const int z0 = max(bz - 1, 0), z1 = min(bz + 1, nb - 1);
    // the candidate columns: ranges [qs, qs + len) of binned[], in visiting order
    int qs[9], pre[10];
    pre[0] = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const int cx = bx - 1 + c / 3, cy = by - 1 + c % 3;
        int a = 0, b = 0;
        if (cx >= 0 && cx < nb && cy >= 0 && cy < nb) {
            const int col = (cx * nb + cy) * nb;
            a = W.bin_start[col + z0];
            b = W.bin_start[col + z1 + 1];
        }
        qs[c] = a;
        pre[c + 1] = pre[c] + (b - a);
    }
    const int nbin = pre[9];
    const int nset = MODE == 0 ? (skip_stale ? W.S->nstale : 0) : W.S->nhot;
    const uint16_t* set = MODE == 0 ? W.S->stale : W.S->hot;
    const int total_c = nbin + nset, nit = (total_c + 31) >> 5;
    // sweep 1: count
    int total = 0;
    for (int it = 0; it < nit; ++it) {
        const int t = lane + 32 * it;
        bool hit = false;
        if (t < total_c) {
            int j;
            if (t < nbin) {
                int q = 0;
#pragma unroll
                for (int u = 0; u < 9; ++u)
                    if (t >= pre[u] && t < pre[u + 1]) q = qs[u] + (t - pre[u]);
                j = W.binned[q];
            } else {
                j = set[t - nbin];
            }
            if (j != i) {
                const V4<R> pj = W.pos[j];
                hit = !(MODE == 1 && t < nbin && is_active(pj)) && !(t < nbin && skip_stale && bit_of(W.sbits, j)) &&
                      list_d2(pi, pj) < H.rlist2;
            }
        }
        total += __popc(__ballot_sync(FULL, hit));
    }
    // storage: the shared row, or an overflow row (the slot's previous one if it had one)
    uint16_t* out = W.nbr + (size_t)slot * REED_MAXNB;
    const int old_m = W.nnb[slot];
    const int old_r = old_m > NS ? (int)out[0] : -1;
    uint16_t* dst = out;
    int cap = NS, r = -1;
    if (total > NS) {
        r = old_r;
        if (r < 0) {
            r = REED_SPILL_ROWS;
            if (lane == 0 && W.sp_nbr) r = atomicAdd(&W.S->nspill, 1);
            r = __shfl_sync(FULL, r, 0);
        }
        if (r < REED_SPILL_ROWS && W.sp_nbr) {
            dst = W.sp_nbr + (size_t)r * NW;
            cap = NW;
        }
    }
    __syncwarp();
    // sweep 2: write in order, mark frozen neighbours without a row
    int w = 0;
    for (int it = 0; it < nit; ++it) {
        const int t = lane + 32 * it;
        bool hit = false;
        int j = i;
        V4<R> pj = pi;
        if (t < total_c) {
            if (t < nbin) {
                int q = 0;
#pragma unroll
                for (int u = 0; u < 9; ++u)
                    if (t >= pre[u] && t < pre[u + 1]) q = qs[u] + (t - pre[u]);
                j = W.binned[q];
            } else {
                j = set[t - nbin];
            }
            if (j != i) {
                pj = W.pos[j];
                hit = !(MODE == 1 && t < nbin && is_active(pj)) && !(t < nbin && skip_stale && bit_of(W.sbits, j)) &&
                      list_d2(pi, pj) < H.rlist2;
            }
        }
        const unsigned bal = __ballot_sync(FULL, hit);
        if (hit) {
            const int e = w + __popc(bal & ((1u << lane) - 1u));
            if (e < cap) dst[e] = (uint16_t)j;
            if (!is_active(pj) && W.need_map[j] == REED_NO_SLOT) W.need_map[j] = (uint16_t)REED_PENDING;
        }
        w += __popc(bal);
    }
    __syncwarp();
    if (lane == 0) {
        if (cap == NW) out[0] = (uint16_t)r;
        if (total > cap) overflow += total - cap;
    }
    return min(total, cap);
}

// Block-wide exclusive prefix sums of two per-thread counts (threads own
// contiguous chunks, so the result follows their order).  Writes each
// thread's offsets and returns the totals.  All threads must call it.
template <typename R>
__device__ __forceinline__ void block_scan2(TrackShared<R>* S, int c0, int c1, int& o0, int& o1, int& t0, int& t1)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x0 = c0, x1 = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
        if (lane >= o) {
            x0 += y0;
            x1 += y1;
        }
    }
    __syncthreads();
    if (lane == 31) {
        S->scan[0][wid] = x0;
        S->scan[1][wid] = x1;
    }
    __syncthreads();
    int b0 = 0, b1 = 0;
    t0 = 0;
    t1 = 0;
    for (int w = 0; w < nw; ++w) {
        if (w == wid) {
            b0 = t0;
            b1 = t1;
        }
        t0 += S->scan[0][w];
        t1 += S->scan[1][w];
    }
    o0 = b0 + x0 - c0;
    o1 = b1 + x1 - c1;
}

// The same for four counts (c[], offsets o[], totals t[]).
template <typename R>
__device__ __forceinline__ void block_scan4(TrackShared<R>* S, const int c[4], int o[4], int t[4])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = c[i];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int y = __shfl_up_sync(0xffffffffu, x[i], d);
            if (lane >= d) x[i] += y;
        }
    }
    __syncthreads();
    if (lane == 31)
#pragma unroll
        for (int i = 0; i < 4; ++i) S->scan[i][wid] = x[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int b = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w == wid) b = tot;
            tot += S->scan[i][w];
        }
        o[i] = b + x[i] - c[i];
        t[i] = tot;
    }
}

// Centre-pass class of a Tersoff slot with m list neighbours: one thread
// (unrolled, m <= REED_FAST_NB), or a group of 8, 16 or 32 lanes.
__device__ __forceinline__ int centre_class(int m) { return m <= REED_FAST_NB ? 0 : (m <= 8 ? 1 : (m <= 16 ? 2 : 3)); }

// Reverse entries of the slots [k0, k1) (all threads): where the centre of
// slot k sits in the list of each integrated neighbour (lists are
// symmetric: the same distance test from both ends), so the centre pass can
// leave its force there.  SELECTIVE: only the rows whose slot is marked
// (chg[slot] != 0) are recomputed.  (Four entries
// at a time, and the neighbour's list four entries at a time, so that the
// dependent shared-memory loads overlap.)
template <typename R, int TT, bool SELECTIVE>
__device__ __forceinline__ void reverse_entries(Win<R, TT>& W, int k0, int k1, int nact_slots, int& overflow,
                                                const unsigned* chg = nullptr)
{
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const int a = W.slot_atom[k], m = W.nnb[k];
        if (SELECTIVE && chg[k] == 0u) continue;
        const uint16_t* row = W.list(k, m);
        uint8_t* rv = W.rev_row(k, m);
        for (int q0 = 0; q0 < m; q0 += 4) {
            unsigned sp[4];
            int mp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) sp[u] = q0 + u < m ? (unsigned)W.need_map[row[q0 + u]] : REED_NO_SLOT;
#pragma unroll
            for (int u = 0; u < 4; ++u) mp[u] = sp[u] < (unsigned)nact_slots ? (int)W.nnb[sp[u]] : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (q0 + u >= m) break;
                uint8_t e = (uint8_t)REED_NO_REV;
                if (sp[u] < (unsigned)nact_slots) {
                    const uint16_t* prow = W.list((int)sp[u], mp[u]);
                    for (int t0 = 0; t0 < mp[u] && e == (uint8_t)REED_NO_REV; t0 += 4) {
                        int pv[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) pv[v] = t0 + v < mp[u] ? (int)prow[t0 + v] : -1;
#pragma unroll
                        for (int v = 3; v >= 0; --v)
                            if (pv[v] == a) e = (uint8_t)(t0 + v);
                    }
                    if (e == (uint8_t)REED_NO_REV) ++overflow;   // only with a truncated list
                }
                rv[q0 + u] = e;
            }
        }
    }
}

// The order of the centre pass (all threads; ends with a barrier): the slots
// class by class (see ters_centres), in slot order inside a class.
template <typename R, int TT> __device__ void centre_order(Win<R, TT>& W, int nneed)
{
    TrackShared<R>* S = W.S;
    const int kc = (nneed + blockDim.x - 1) / blockDim.x;
    const int k0 = min(nneed, (int)threadIdx.x * kc), k1 = min(nneed, k0 + kc);
    int c[4] = {0, 0, 0, 0}, o[4], t[4];
    for (int k = k0; k < k1; ++k) {
        const int cl = centre_class(W.nnb[k]);
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] += cl == i;
    }
    block_scan4<R>(S, c, o, t);
    o[1] += t[0];
    o[2] += t[0] + t[1];
    o[3] += t[0] + t[1] + t[2];
    for (int k = k0; k < k1; ++k) {
        const int cl = centre_class(W.nnb[k]);
        int dst = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (cl == i) dst = o[i]++;
        W.order[dst] = (uint16_t)k;
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) S->ncls[i] = t[i];
    __syncthreads();
}

// The end of a full Tersoff list build (all threads, after the lists and a
// barrier; ends with a barrier): clears the pending marks, fills the reverse
// entries and the order of the centre pass.
template <typename R, int TT>
__device__ void finish_tersoff_lists(const DevParams& P, Win<R, TT>& W, int nact_slots, int nneed, int& overflow)
{
    // (pending marks set by these last lists are not needed: clear them)
    for (int i = threadIdx.x; i < P.na; i += blockDim.x)
        if (W.need_map[i] == REED_PENDING) W.need_map[i] = (uint16_t)REED_NO_SLOT;
    __syncthreads();
    reverse_entries<R, TT, false>(W, 0, nneed, nact_slots, overflow);
    centre_order<R, TT>(W, nneed);
}

template <typename R, int TT>
__device__ void build_neighbours(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int& overflow,
                                 int& cap_overflow, unsigned long long& spilled)
{
    const int na = P.na, nbins = P.g_nbins;
    TrackShared<R>* S = W.S;
    const int chunk = (na + blockDim.x - 1) / blockDim.x;
    const int i0 = min(na, (int)threadIdx.x * chunk), i1 = min(na, i0 + chunk);
    const int bchunk = (nbins + blockDim.x - 1) / blockDim.x;
    const int j0 = min(nbins, (int)threadIdx.x * bchunk), j1 = min(nbins, j0 + bchunk);
    if (threadIdx.x == 0) S->nspill = 0;
    if constexpr (TT == REED_TT_TERSOFF) {   // every bin is current again
        for (int w = threadIdx.x; w < (na + 31) >> 5; w += blockDim.x) W.sbits[w] = W.hbits[w] = 0u;
        for (int k = threadIdx.x; k < P.bond_cap; k += blockDim.x) W.tmask[k] = 0u;
        if (threadIdx.x == 0) S->nstale = S->nhot = 0;
    }
    // bin populations and integrated atoms of this thread's chunk
    int nact = 0;
    for (int i = i0; i < i1; ++i) {
        const V4<R> p = W.pos[i];
        W.need_map[i] = (uint16_t)REED_NO_SLOT;
        if (is_present(p)) {
            atomicAdd(&W.bin_count[grid_bin<R>(P, H, p)], 1u);
            nact += is_active(p) ? 1 : 0;
            W.vel[i].w = R(0);   // path length since the list was built
        }
    }
    __syncthreads();
    int nbin_atoms = 0;
    for (int j = j0; j < j1; ++j) nbin_atoms += (int)W.bin_count[j];
    int ob, oa, tot_b, tot_a;
    block_scan2<R>(S, nbin_atoms, nact, ob, oa, tot_b, tot_a);
    for (int j = j0; j < j1; ++j) {
        W.bin_start[j] = (uint16_t)ob;
        ob += (int)W.bin_count[j];
    }
    if (threadIdx.x == 0) W.bin_start[nbins] = (uint16_t)tot_b;
    for (int i = i0; i < i1; ++i) {
        if (!is_active(W.pos[i])) continue;
        if (oa < P.bond_cap) {
            W.need_map[i] = (uint16_t)oa;
            W.slot_atom[oa] = (uint16_t)i;
        } else {
            ++cap_overflow;
        }
        ++oa;
    }
    const int nact_slots = min(tot_a, P.bond_cap);
    if (threadIdx.x == 0) S->active_count = nact_slots;
    __syncthreads();
    // scatter into the bins (the counters run back down to zero)
    for (int i = i0; i < i1; ++i) {
        const V4<R> p = W.pos[i];
        if (!is_present(p)) continue;
        const int b = grid_bin<R>(P, H, p);
        const unsigned k = atomicSub(&W.bin_count[b], 1u) - 1u;
        W.binned[W.bin_start[b] + k] = (uint16_t)i;
    }
    __syncthreads();
    // atom order inside each bin
    for (int j = threadIdx.x; j < nbins; j += blockDim.x) {
        const int q0 = W.bin_start[j], q1 = W.bin_start[j + 1];
        for (int q = q0 + 1; q < q1; ++q) {
            const uint16_t v = W.binned[q];
            int r = q - 1;
            while (r >= q0 && W.binned[r] > v) {
                W.binned[r + 1] = W.binned[r];
                --r;
            }
            W.binned[r + 1] = v;
        }
    }
    __syncthreads();
    // lists of integrated atoms; their other neighbours become pending
    for (int k = threadIdx.x; k < nact_slots; k += blockDim.x) {
        const int i = W.slot_atom[k];
        W.nnb[k] = (uint8_t)list_of<R, TT>(P, H, W, i, k, overflow);
    }
    __syncthreads();
    if constexpr (TT != REED_TT_TERSOFF) {
        // pair potentials need lists of the integrated atoms only
        if (threadIdx.x == 0) {
            S->need_count = nact_slots;
            spilled += (unsigned long long)min(S->nspill, REED_SPILL_ROWS);
        }
        __syncthreads();
        return;
    }
    // slots for the pending atoms, in atom order after the integrated ones
    int npend = 0;
    for (int i = i0; i < i1; ++i) npend += W.need_map[i] == REED_PENDING;
    int op, dummy, tot_pend, dummy_t;
    block_scan2<R>(S, npend, 0, op, dummy, tot_pend, dummy_t);
    op += nact_slots;
    for (int i = i0; i < i1; ++i) {
        if (W.need_map[i] != REED_PENDING) continue;
        if (op < P.bond_cap) {
            W.need_map[i] = (uint16_t)op;
            W.slot_atom[op] = (uint16_t)i;
        } else {
            W.need_map[i] = (uint16_t)REED_NO_SLOT;
            ++cap_overflow;
        }
        ++op;
    }
    const int nneed = min(nact_slots + tot_pend, P.bond_cap);
    __syncthreads();
    for (int k = nact_slots + threadIdx.x; k < nneed; k += blockDim.x) {
        const int i = W.slot_atom[k];
        W.nnb[k] = (uint8_t)list_of<R, TT>(P, H, W, i, k, overflow);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S->need_count = nneed;
        spilled += (unsigned long long)min(S->nspill, REED_SPILL_ROWS);
    }
    finish_tersoff_lists<R, TT>(P, W, nact_slots, nneed, overflow);
}

// ---------------------------------------------------------------------------
// Partial refresh of the Tersoff lists (no window move since the last full
// build; all threads, after a barrier; ends with a barrier).  Only the
// integrated atoms whose path since their last list exceeds a quarter of the
// skin ("hot") get new lists; every other list keeps its entries, drops those
// of hot atoms and gains the hot atoms that now list it.  A pair of atoms
// that are both not hot has moved by at most half the skin since its status
// was last evaluated, so the lists still hold every pair within the cutoff.
// The grid bins are those of the last full build: atoms that have been hot
// since then ("stale") are tested from the stale set; every other atom has
// moved by at most a quarter of the skin, and bins at least r_list + skin/2
// wide keep it in the 27 bins around any point within r_list of it.  A
// frozen atom that becomes needed gets the frozen atoms and the hot atoms
// within the list radius: an integrated atom that is not hot cannot list it
// (else it would have been needed already), so both ends agree.  Returns
// false, before changing any list, when the sets or the list rows would
// overflow; the caller then builds from scratch.
// ---------------------------------------------------------------------------
template <typename R, int TT>
__device__ bool refresh_lists(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int& overflow,
                              unsigned long long& spilled)
{
    const int na = P.na, tid = threadIdx.x, lane = tid & 31, nw = blockDim.x >> 5, wid = tid >> 5;
    TrackShared<R>* S = W.S;
    // (refreshing every atom past a quarter of the skin leaves the rest at most
    // a quarter each, so the next refresh comes only after the two fastest have
    // moved another half skin)
    const R thr = R(0.25) * H.skin;
    const int nact = S->active_count, nneed0 = S->need_count, nstale0 = S->nstale, nsp0 = S->nspill;
    // hot atoms, among the integrated ones (slot order is atom order)
    const int kc = (nact + blockDim.x - 1) / blockDim.x;
    const int k0 = min(nact, tid * kc), k1 = min(nact, k0 + kc);
    int c[4] = {0, 0, 0, 0}, o[4], t4[4];
    for (int k = k0; k < k1; ++k) {
        const int i = W.slot_atom[k];
        if (W.vel[i].w > thr) {
            ++c[0];
            c[1] += bit_of(W.sbits, i) ? 0 : 1;
        }
    }
    block_scan4<R>(S, c, o, t4);
    const int nhot = t4[0];
    if (nhot == 0 || nhot > REED_MAX_HOT || nstale0 + t4[1] > REED_MAX_STALE || S->nspill > REED_SPILL_ROWS / 2) {
        __syncthreads();
        return false;   // (overflow rows are only reclaimed by a full build)
    }
    {
        int oh = o[0], os = nstale0 + o[1];
        for (int k = k0; k < k1; ++k) {
            const int i = W.slot_atom[k];
            if (!(W.vel[i].w > thr)) continue;
            S->hot[oh++] = (uint16_t)i;
            atomicOr(&W.hbits[i >> 5], 1u << (i & 31));
            if (!bit_of(W.sbits, i)) {
                S->stale[os++] = (uint16_t)i;   // (atom order among the new ones)
                atomicOr(&W.sbits[i >> 5], 1u << (i & 31));
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        S->nhot = nhot;
        S->nstale = nstale0 + t4[1];
    }
    // rows that will lose a hot atom: the old neighbours of the hot atoms
    for (int t = wid; t < nhot; t += nw) {
        const int kh = W.need_map[S->hot[t]], mh = W.nnb[kh];
        const uint16_t* rh = W.list(kh, mh);
        for (int q = lane; q < mh; q += 32) {
            const unsigned sj = W.need_map[rh[q]];
            if (sj < REED_PENDING) atomicOr(&W.tmask[sj], 1u << 31);
        }
    }
    __syncthreads();
    // new lists of the hot atoms (one warp each)
    for (int t = wid; t < nhot; t += nw) {
        const int h = S->hot[t];
        const int k = W.need_map[h];
        const int m = list_of_warp<R, TT, 0>(P, H, W, h, k, overflow);
        if (lane == 0) W.nnb[k] = (uint8_t)m;
    }
    __syncthreads();
    // frozen atoms that became needed must fit; nothing has changed yet
    // that a full build would not redo
    const int chunk = (na + blockDim.x - 1) / blockDim.x;
    const int i0 = min(na, tid * chunk), i1 = min(na, i0 + chunk);
    int np = 0;
    for (int i = i0; i < i1; ++i) np += W.need_map[i] == REED_PENDING;
    int op, dummy, tp, dummy_t;
    block_scan2<R>(S, np, 0, op, dummy, tp, dummy_t);
    if (nneed0 + tp > P.bond_cap) {
        __syncthreads();
        return false;
    }
    // rows that gain a hot atom: the new neighbours of the hot atoms (hot
    // rows are rebuilt whole, rows of atoms that became needed are new)
    for (int t = wid; t < nhot; t += nw) {
        const int kh = W.need_map[S->hot[t]], mh = W.nnb[kh];
        const uint16_t* rh = W.list(kh, mh);
        for (int q = lane; q < mh; q += 32) {
            const unsigned sj = W.need_map[rh[q]];
            if (sj < REED_PENDING) atomicOr(&W.tmask[sj], 1u << t);
        }
    }
    __syncthreads();
    // the marked rows: drop the hot atoms, append those that list this atom
    for (int k = tid; k < nneed0; k += blockDim.x) {
        const unsigned mk = W.tmask[k];
        if (!mk) continue;
        const int a = W.slot_atom[k];
        if (bit_of(W.hbits, a)) continue;
        const unsigned add = mk & 0x7fffffffu;
        const int m = W.nnb[k];
        const uint16_t* row = W.list(k, m);
        if (m <= maxnb(TT)) {   // in place in the shared row (entries only move down)
            ListWriter<R, TT> L(W, k);
            for (int q = 0; q < m; ++q) {
                const int j = row[q];
                if (!bit_of(W.hbits, j)) L.out[L.cnt++] = (uint16_t)j;
            }
            for (int t = 0; t < nhot; ++t)
                if ((add >> t) & 1u) L.add(W, S->hot[t], overflow);
            W.nnb[k] = (uint8_t)L.cnt;
        } else {                // in place in the overflow row; back to the shared row if it fits
            uint16_t* sp = const_cast<uint16_t*>(row);
            int w = 0;
            for (int q = 0; q < m; ++q) {
                const int j = row[q];
                if (!bit_of(W.hbits, j)) sp[w++] = (uint16_t)j;
            }
            for (int t = 0; t < nhot; ++t) {
                if (!((add >> t) & 1u)) continue;
                if (w < REED_SPILL_TERSOFF) sp[w++] = S->hot[t];
                else ++overflow;
            }
            if (w <= maxnb(TT))
                for (int e = 0; e < w; ++e) W.nbr[(size_t)k * REED_MAXNB + e] = sp[e];
            W.nnb[k] = (uint8_t)w;
        }
    }
    // slots of the frozen atoms that became needed, in atom order
    op += nneed0;
    for (int i = i0; i < i1; ++i) {
        if (W.need_map[i] != REED_PENDING) continue;
        W.need_map[i] = (uint16_t)op;
        W.slot_atom[op] = (uint16_t)i;
        W.tmask[op] = 1u << 31;   // (a new row)
        ++op;
    }
    const int nneed = nneed0 + tp;
    __syncthreads();
    for (int k = nneed0 + wid; k < nneed; k += nw) {
        const int i = W.slot_atom[k];
        if (lane == 0) W.nnb[k] = 0;   // (no overflow row to reuse)
        __syncwarp();
        const int m = list_of_warp<R, TT, 1>(P, H, W, i, k, overflow);
        if (lane == 0) W.nnb[k] = (uint8_t)m;
    }
    for (int t = tid; t < nhot; t += blockDim.x) W.tmask[W.need_map[S->hot[t]]] |= 1u << 31;   // (rebuilt rows)
    __syncthreads();
    if (tid == 0) {
        S->need_count = nneed;
        spilled += (unsigned long long)(min(S->nspill, REED_SPILL_ROWS) - min(nsp0, REED_SPILL_ROWS));
    }
    // (pending marks set by the new rows' lists are not needed: clear them)
    for (int i = i0; i < i1; ++i)
        if (W.need_map[i] == REED_PENDING) W.need_map[i] = (uint16_t)REED_NO_SLOT;
    // reverse entries: of the changed rows, and of the rows listed in them
    // (lists are symmetric, so those are the rows that point into them)
    for (int k = tid; k < nneed; k += blockDim.x) {
        if (!(W.tmask[k] & ~(1u << 30))) continue;
        const int m = W.nnb[k];
        const uint16_t* row = W.list(k, m);
        for (int q = 0; q < m; ++q) {
            const unsigned sj = W.need_map[row[q]];
            if (sj < (unsigned)nneed) atomicOr(&W.tmask[sj], 1u << 30);
        }
    }
    __syncthreads();
    reverse_entries<R, TT, true>(W, 0, nneed, nact, overflow, W.tmask);
    __syncthreads();
    centre_order<R, TT>(W, nneed);
    // the hot atoms start new paths; the marks are cleared
    for (int k = tid; k < nneed; k += blockDim.x) W.tmask[k] = 0u;
    for (int t = tid; t < nhot; t += blockDim.x) {
        const int h = S->hot[t];
        W.vel[h].w = R(0);
        atomicAnd(&W.hbits[h >> 5], ~(1u << (h & 31)));
    }
    __syncthreads();
    return true;
}

// Self-check of the Tersoff lists (option nl_check; all threads, ends with a
// barrier): every pair of a needed atom with an atom within `r2ok` must be
// listed, and no listed pair may be farther than r_list + skin.  Counts the
// differences.
template <typename R, int TT>
__device__ void check_lists(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, R r2ok, unsigned long long& errors)
{
    if constexpr (TT != REED_TT_TERSOFF) return;   // (the pair lists are neighbour-major)
    const R rmax = Mth<R>::rsqrt(H.rlist2);
    const R lim = H.rlist2 * (R(1) + H.skin * rmax) * (R(1) + H.skin * rmax);   // (r_list + skin)^2
    const int nneed = W.S->need_count;
    unsigned long long e = 0;
    for (int k = threadIdx.x; k < nneed; k += blockDim.x) {
        const int a = W.slot_atom[k], m = W.nnb[k];
        const uint16_t* row = W.list(k, m);
        const V4<R> pa = W.pos[a];
        for (int j = 0; j < P.na; ++j) {
            if (j == a || !is_present(W.pos[j])) continue;
            if (!(list_d2(pa, W.pos[j]) < r2ok)) continue;
            bool found = false;
            for (int q = 0; q < m; ++q) found = found || row[q] == j;
            e += found ? 0 : 1;
        }
        for (int q = 0; q < m; ++q) e += list_d2(pa, W.pos[row[q]]) < lim ? 0 : 1;
    }
    errors += e;
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tersoff forces, one centre at a time.  The energy of the bonds centred on
// atom a,
//     E_a = 1/2 sum_j V(r_j, b_j),   b_j = b(zeta_j),
//     zeta_j = sum_{k != j} fc(r_k) g(c_jk),   c_jk = u_j . u_k,
// (j, k over a's neighbours, u_j the unit vector from a to j) depends on the
// positions of a and its neighbours only.  With P_j = 1/2 dV_j/db db_j/dzeta
// and Q_j = 1/2 dV_j/dr, the force it exerts on neighbour p is
//     F_p = -u_p [Q_p + fc'(r_p) sum_{j != p} P_j g(c_jp)]
//           - (1 / r_p) sum_{j != p} [P_j fc(r_p) + P_p fc(r_j)] g'(c_jp) (u_j - c_jp u_p)
// and on a itself -sum_p F_p.  The centre pass evaluates every needed atom
// once and leaves F_p in the force row of each integrated neighbour p (at
// a's entry in p's list) and -sum_p F_p in frc[a] when a is integrated; the
// force phase then sums each integrated atom's row in list order.  Every
// term is written by one thread and summed in a fixed order, so results do
// not depend on thread timing.
// ---------------------------------------------------------------------------

// Atoms with at most REED_FAST_NB neighbours: everything in registers
// (unrolled; missing neighbours have fc = P = Q = 0 and contribute nothing).
template <typename R, int TT>
__device__ __forceinline__ R ters_centre_fast(const HotParams<R>& H, Win<R, TT>& W, int k, int m, int nact,
                                              unsigned long long& triplets)
{
    constexpr int M = REED_FAST_NB;
    const int a = W.slot_atom[k];
    const V4<R> pa = W.pos[a];
    const uint16_t* row = W.nbr + (size_t)k * REED_MAXNB;
    const uint8_t* rv = W.rev + (size_t)k * REED_MAXNB;
    R ux[M], uy[M], uz[M], ir[M], rr[M], fc[M], dfc[M];
    int idx[M];
    int npos = 0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        ux[q] = uy[q] = uz[q] = ir[q] = rr[q] = fc[q] = dfc[q] = R(0);
        idx[q] = -1;
        if (q < m) {
            idx[q] = row[q];
            const V4<R> pq = W.pos[idx[q]];
            const R dx = pq.x - pa.x, dy = pq.y - pa.y, dz = pq.z - pa.z;
            const R r2 = dx * dx + dy * dy + dz * dz;
            ir[q] = Mth<R>::rsqrt(r2);
            rr[q] = r2 * ir[q];
            ux[q] = dx * ir[q];
            uy[q] = dy * ir[q];
            uz[q] = dz * ir[q];
            fc[q] = ters_fc<R>(H, rr[q], dfc[q]);
            npos += (fc[q] > R(0) || dfc[q] != R(0)) ? 1 : 0;
        }
    }
    if (m > 1) triplets += (unsigned long long)((m - 1) * npos);
    // angle terms of every pair of neighbours
    R c[M][M], g[M][M], dg[M][M];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int p = q + 1; p < M; ++p) {
            c[q][p] = ux[q] * ux[p] + uy[q] * uy[p] + uz[q] * uz[p];
            g[q][p] = ters_g<R>(H, c[q][p], dg[q][p]);
        }
    // bond orders, bond energies and their derivatives
    R P[M], Q[M];
    R E = R(0);
#pragma unroll
    for (int q = 0; q < M; ++q) {
        R zeta = R(0);
#pragma unroll
        for (int p = 0; p < M; ++p)
            if (p != q) zeta += fc[p] * (p < q ? g[p][q] : g[q][p]);
        P[q] = Q[q] = R(0);
        if (q < m && (fc[q] > R(0) || dfc[q] != R(0))) {
            R db, V, dV, pfa;
            const R b = ters_b<R>(H, zeta, db);
            ters_pair<R>(H, rr[q], fc[q], dfc[q], b, V, dV, pfa);
            P[q] = R(0.5) * pfa * db;
            Q[q] = R(0.5) * dV;
            E += R(0.5) * V;
        }
    }
    // forces on the neighbours
    R fx[M], fy[M], fz[M];
#pragma unroll
    for (int p = 0; p < M; ++p) {
        R sg = R(0);
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (j != p) sg += P[j] * (j < p ? g[j][p] : g[p][j]);
        const R A = Q[p] + dfc[p] * sg;
        fx[p] = -A * ux[p];
        fy[p] = -A * uy[p];
        fz[p] = -A * uz[p];
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
        for (int p = j + 1; p < M; ++p) {
            const R w = (P[j] * fc[p] + P[p] * fc[j]) * dg[j][p];
            const R wp = w * ir[p], wj = w * ir[j], cc = c[j][p];
            fx[p] -= wp * (ux[j] - cc * ux[p]);
            fy[p] -= wp * (uy[j] - cc * uy[p]);
            fz[p] -= wp * (uz[j] - cc * uz[p]);
            fx[j] -= wj * (ux[p] - cc * ux[j]);
            fy[j] -= wj * (uy[p] - cc * uy[j]);
            fz[j] -= wj * (uz[p] - cc * uz[j]);
        }
    R ax = R(0), ay = R(0), az = R(0);
#pragma unroll
    for (int p = 0; p < M; ++p) {
        ax -= fx[p];
        ay -= fy[p];
        az -= fz[p];
        if (p < m) {
            const unsigned s = W.need_map[idx[p]];
            if (s < (unsigned)nact && rv[p] != (uint8_t)REED_NO_REV) W.bf_store((int)s, rv[p], fx[p], fy[p], fz[p]);
        }
    }
    if (k < nact) {
        V4<R> f;
        f.x = ax;
        f.y = ay;
        f.z = az;
        f.w = R(0);
        W.frc[a] = f;
    }
    return E;
}

// More than REED_FAST_NB neighbours (lists in shared memory or in an
// overflow row): a group of G lanes per centre (G = 8, 16 or 32; lane l of
// the group owns neighbours l and, for G = 32, l + 32).  The terms a lane
// needs from the other neighbours are broadcast with shuffles inside the
// group; sums over the group use the fixed butterfly order.  All 32 lanes of
// the warp call it together, each group with its own slot k (k < 0: idle).
template <typename R, int TT, int G>
__device__ R ters_centre_group(const HotParams<R>& H, Win<R, TT>& W, int k, int nact, unsigned long long& triplets)
{
    constexpr int NH = G == 32 ? 2 : 1;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1);
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int m = k >= 0 ? (int)W.nnb[k] : 0;
    const int mmax = (int)__reduce_max_sync(FULL, (unsigned)m);
    int a = 0;
    V4<R> pa = {R(0), R(0), R(0), R(0)};
    const uint16_t* row = nullptr;
    const uint8_t* rv = nullptr;
    if (k >= 0) {
        a = W.slot_atom[k];
        pa = W.pos[a];
        row = W.list(k, m);
        rv = W.rev_row(k, m);
    }
    // per-neighbour terms of this lane's neighbours
    R ux[NH], uy[NH], uz[NH], ir[NH], rr[NH], fc[NH], dfc[NH], P[NH], Q[NH], fx[NH], fy[NH], fz[NH];
    int id[NH];
    bool ok[NH];
    int npos = 0;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const int q = lg + G * h;
        ok[h] = q < m;
        ux[h] = uy[h] = uz[h] = ir[h] = rr[h] = fc[h] = dfc[h] = P[h] = Q[h] = R(0);
        fx[h] = fy[h] = fz[h] = R(0);
        id[h] = -1;
        if (ok[h]) {
            id[h] = row[q];
            const V4<R> pq = W.pos[id[h]];
            const R dx = pq.x - pa.x, dy = pq.y - pa.y, dz = pq.z - pa.z;
            const R r2 = dx * dx + dy * dy + dz * dz;
            ir[h] = Mth<R>::rsqrt(r2);
            rr[h] = r2 * ir[h];
            ux[h] = dx * ir[h];
            uy[h] = dy * ir[h];
            uz[h] = dz * ir[h];
            fc[h] = ters_fc<R>(H, rr[h], dfc[h]);
        }
        npos += __popc(__ballot_sync(FULL, ok[h] && (fc[h] > R(0) || dfc[h] != R(0))) & gmask);
    }
    if (lg == 0 && m > 1) triplets += (unsigned long long)((m - 1) * npos);
    // bond orders of this lane's bonds
    R zeta[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) zeta[h] = R(0);
    for (int p = 0; p < mmax; ++p) {
        const int src = p & (G - 1), hp = NH == 2 ? (p >> 5) : 0;
        const R vx = __shfl_sync(FULL, hp ? ux[NH - 1] : ux[0], src, G);
        const R vy = __shfl_sync(FULL, hp ? uy[NH - 1] : uy[0], src, G);
        const R vz = __shfl_sync(FULL, hp ? uz[NH - 1] : uz[0], src, G);
        const R fp = __shfl_sync(FULL, hp ? fc[NH - 1] : fc[0], src, G);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            if (!ok[h] || p >= m || lg + G * h == p || fp == R(0)) continue;
            R dg;
            zeta[h] += fp * ters_g<R>(H, ux[h] * vx + uy[h] * vy + uz[h] * vz, dg);
        }
    }
    R E = R(0);
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        if (ok[h] && (fc[h] > R(0) || dfc[h] != R(0))) {
            R db, V, dV, pfa;
            const R b = ters_b<R>(H, zeta[h], db);
            ters_pair<R>(H, rr[h], fc[h], dfc[h], b, V, dV, pfa);
            P[h] = R(0.5) * pfa * db;
            Q[h] = R(0.5) * dV;
            E += R(0.5) * V;
        }
    }
    // forces on this lane's neighbours
    R sg[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) sg[h] = R(0);
    for (int j = 0; j < mmax; ++j) {
        const int src = j & (G - 1), hj = NH == 2 ? (j >> 5) : 0;
        const R vx = __shfl_sync(FULL, hj ? ux[NH - 1] : ux[0], src, G);
        const R vy = __shfl_sync(FULL, hj ? uy[NH - 1] : uy[0], src, G);
        const R vz = __shfl_sync(FULL, hj ? uz[NH - 1] : uz[0], src, G);
        const R fj = __shfl_sync(FULL, hj ? fc[NH - 1] : fc[0], src, G);
        const R Pj = __shfl_sync(FULL, hj ? P[NH - 1] : P[0], src, G);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            if (!ok[h] || j >= m || lg + G * h == j) continue;
            const R cc = vx * ux[h] + vy * uy[h] + vz * uz[h];
            R dg;
            const R g = ters_g<R>(H, cc, dg);
            sg[h] += Pj * g;
            const R w = (Pj * fc[h] + P[h] * fj) * dg * ir[h];
            fx[h] -= w * (vx - cc * ux[h]);
            fy[h] -= w * (vy - cc * uy[h]);
            fz[h] -= w * (vz - cc * uz[h]);
        }
    }
    R ax = R(0), ay = R(0), az = R(0);
#pragma unroll
    for (int h = 0; h < NH; ++h) {
        const R A = Q[h] + dfc[h] * sg[h];
        fx[h] -= A * ux[h];
        fy[h] -= A * uy[h];
        fz[h] -= A * uz[h];
        ax -= fx[h];
        ay -= fy[h];
        az -= fz[h];
        if (ok[h]) {
            const unsigned s = W.need_map[id[h]];
            const uint8_t e = rv[lg + G * h];
            if (s < (unsigned)nact && e != (uint8_t)REED_NO_REV) W.bf_store((int)s, e, fx[h], fy[h], fz[h]);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(FULL, ax, o);
        ay += __shfl_xor_sync(FULL, ay, o);
        az += __shfl_xor_sync(FULL, az, o);
        E += __shfl_xor_sync(FULL, E, o);
    }
    if (lg == 0 && k >= 0 && k < nact) {
        V4<R> f;
        f.x = ax;
        f.y = ay;
        f.z = az;
        f.w = R(0);
        W.frc[a] = f;
    }
    return (lg == 0 && k >= 0) ? E : R(0);
}

// The centre pass over every needed slot (all threads; a barrier must follow).
// `order` holds the slots class by class: ncls[0] with at most REED_FAST_NB
// neighbours (one thread each, unrolled), then ncls[1] with up to 8 (groups
// of 8 lanes, four centres per warp), ncls[2] with up to 16 (two per warp)
// and ncls[3] with more (one per warp).  The group tasks are dealt to the
// warps from the last one down (the last warps have the fewest one-thread
// slots).  Returns this thread's share of the Tersoff energy.
template <typename R, int TT>
__device__ R ters_centres(const HotParams<R>& H, Win<R, TT>& W, unsigned long long& triplets)
{
    const int nact = W.S->active_count;
    const int n0 = W.S->ncls[0], n1 = W.S->ncls[1], n2 = W.S->ncls[2], n3 = W.S->ncls[3];
    R E = R(0);
    for (int j = threadIdx.x; j < n0; j += blockDim.x) {
        const int k = W.order[j];
        E += ters_centre_fast<R, TT>(H, W, k, W.nnb[k], nact, triplets);
    }
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t1 = (n1 + 3) / 4, t2 = (n2 + 1) / 2, ntask = t1 + t2 + n3;
    for (int t = nw - 1 - w; t < ntask; t += nw) {
        if (t < t1) {
            const int j = 4 * t + (lane >> 3);
            E += ters_centre_group<R, TT, 8>(H, W, j < n1 ? (int)W.order[n0 + j] : -1, nact, triplets);
        } else if (t < t1 + t2) {
            const int j = 2 * (t - t1) + (lane >> 4);
            E += ters_centre_group<R, TT, 16>(H, W, j < n2 ? (int)W.order[n0 + n1 + j] : -1, nact, triplets);
        } else {
            E += ters_centre_group<R, TT, 32>(H, W, (int)W.order[n0 + n1 + n2 + (t - t1 - t2)], nact, triplets);
        }
    }
    return E;
}

// Sum of the force row of the integrated atom in slot k (list order).
template <typename R, int TT>
__device__ __forceinline__ void ters_gather(const Win<R, TT>& W, int k, R& Fx, R& Fy, R& Fz)
{
    const int m = W.nnb[k];
    R fx = R(0), fy = R(0), fz = R(0);
    if (m <= REED_MAXNB) {
        const int o = k * REED_BF_STRIDE;
        for (int q = 0; q < m; ++q) {
            fx += W.bfx[o + q];
            fy += W.bfy[o + q];
            fz += W.bfz[o + q];
        }
    } else {
        const R* b = W.sp_bf + (size_t)W.nbr[(size_t)k * REED_MAXNB] * 3 * REED_SPILL_TERSOFF;
        for (int q = 0; q < m; ++q) {
            fx += b[q];
            fy += b[REED_SPILL_TERSOFF + q];
            fz += b[2 * REED_SPILL_TERSOFF + q];
        }
    }
    Fx += fx;
    Fy += fy;
    Fz += fz;
}

// Buckingham / short-range pair forces on atom i from its list (each pair is
// visited from both ends; the energy is halved).
template <typename R, int TT>
__device__ R pair_force(const HotParams<R>& H, Win<R, TT>& W, int i, int k, R& Fx, R& Fy, R& Fz)
{
    const int m = W.nnb[k];
    const V4<R> pi = W.pos[i];
    const int si = species_of(pi);
    const uint16_t* nb = W.list(k, m);
    const int oq = m <= maxnb(TT) ? W.nb_q : 1;   // an overflow row is contiguous
    R E = R(0);
    for (int q = 0; q < m; ++q) {
        const V4<R> pj = W.pos[nb[(size_t)q * oq]];
        R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        R r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= H.b_rc2) continue;
        R U;
        R g = buck_pair<R>(H, si + species_of(pj), r2, U);
        Fx += g * dx;
        Fy += g * dy;
        Fz += g * dz;
        E += R(0.5) * U;
    }
    return E;
}

// Partial sums reduced per step.
template <typename R> struct Partial {
    R fx, fy, fz, rho, vmax2, epot;
    int pairs, bonds;
    R pmax;
};

// Per-thread work counters (algorithmic units of a step, see stats).
struct WorkCount {
    unsigned long long triplets = 0;   // Tersoff bond-angle terms (one per zeta term)
    unsigned long long moved = 0;      // integrated atom updates
    unsigned long long spilled = 0;    // overflow rows taken by list builds (thread 0)
    unsigned long long refreshes = 0;  // Tersoff partial refreshes (thread 0)
    unsigned long long nl_errors = 0;  // list self-check differences (all threads)
};

// Force evaluation over the whole window; with KICK the second half kick is
// applied to integrated atoms and their speed^2 reduced for the next dt.
// Writes W.frc of every present atom.  With target-target terms the
// integrated atoms are visited through their list slots (balanced across
// threads); the others only contribute ion-target pairs.
// The ion-target part of one atom's force pass at its current position p,
// and (integrated atoms) the second half kick: the operations of atom_force
// for an atom without target-target terms, on values held in registers.
template <typename R>
__device__ __forceinline__ void ion_atom_step(const DevParams& P, const HotParams<R>& H, const TrackShared<R>* S,
                                              const V4<R>& p, V4<R>& v, bool act, R hdt, V4<R>& f, Partial<R>& out)
{
    R fx = R(0), fy = R(0), fz = R(0);
    const R dx = p.x - S->rel[0], dy = p.y - S->rel[1], dz = p.z - S->rel[2];
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < H.rc2) {
        R U, rw;
        const R g = ion_pair<R>(H, P.spline_on, P.rho_on, species_of(p), r2, U, rw);
        fx -= g * dx;
        fy -= g * dy;
        fz -= g * dz;
        out.fx += g * dx;
        out.fy += g * dy;
        out.fz += g * dz;
        out.rho += rw;
        out.epot += U;
        out.pairs += 1;
    }
    f.x = fx;
    f.y = fy;
    f.z = fz;
    f.w = R(0);
    if (act) {
        const R kk = hdt * H.invM2[species_of(p)];
        v.x += kk * fx;
        v.y += kk * fy;
        v.z += kk * fz;
        out.vmax2 = max(out.vmax2, v.x * v.x + v.y * v.y + v.z * v.z);
        if (H.de_max > R(0)) out.pmax = max(out.pmax, fabs(fx * v.x + fy * v.y + fz * v.z));
    }
}

template <typename R, int TT, bool KICK>
__device__ __forceinline__ void atom_force(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int i, int k,
                                           R hdt, Partial<R>& out, bool want_energy)
{
    const R ix = W.S->rel[0], iy = W.S->rel[1], iz = W.S->rel[2];
    V4<R> p = W.pos[i];
    const bool act = is_active(p);
    R fx = R(0), fy = R(0), fz = R(0);
    if (TT == REED_TT_TERSOFF && act && k >= 0) {   // the bonds centred on i, from the centre pass
        const V4<R> f1 = W.frc[i];
        fx = f1.x;
        fy = f1.y;
        fz = f1.z;
    }
    const R dx = p.x - ix, dy = p.y - iy, dz = p.z - iz;
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < H.rc2) {
        R U, rw;
        const R g = ion_pair<R>(H, P.spline_on, P.rho_on, species_of(p), r2, U, rw);
        fx -= g * dx;
        fy -= g * dy;
        fz -= g * dz;
        out.fx += g * dx;
        out.fy += g * dy;
        out.fz += g * dz;
        out.rho += rw;
        out.epot += U;
        out.pairs += 1;
    }
    if (k >= 0) {
        if constexpr (TT == REED_TT_TERSOFF) {
            if (act) {
                ters_gather<R, TT>(W, k, fx, fy, fz);
                out.bonds += W.nnb[k];
            }
        }
        if constexpr (TT == REED_TT_BUCKINGHAM) {
            if (act || want_energy) {
                out.epot += pair_force<R, TT>(H, W, i, k, fx, fy, fz);
                out.bonds += W.nnb[k];
            }
        }
    }
    V4<R> f;
    f.x = fx;
    f.y = fy;
    f.z = fz;
    f.w = R(0);
    W.frc[i] = f;
    if (KICK && act) {
        V4<R> v = W.vel[i];
        const R kk = hdt * H.invM2[species_of(p)];
        v.x += kk * fx;
        v.y += kk * fy;
        v.z += kk * fz;
        W.vel[i] = v;
        out.vmax2 = max(out.vmax2, v.x * v.x + v.y * v.y + v.z * v.z);
        if (H.de_max > R(0)) out.pmax = max(out.pmax, fabs(fx * v.x + fy * v.y + fz * v.z));
    }
}

template <typename R, int TT, bool KICK>
__device__ void force_phase(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, R hdt, Partial<R>& out,
                            bool want_energy)
{
    if constexpr (TT == REED_TT_NONE) {
        for (int i = threadIdx.x; i < P.na; i += blockDim.x)
            if (is_present(W.pos[i])) atom_force<R, TT, KICK>(P, H, W, i, -1, hdt, out, want_energy);
    } else {
        // integrated atoms through their slots, then every other present atom
        const int nact = W.S->active_count;
        for (int k = threadIdx.x; k < nact; k += blockDim.x)
            atom_force<R, TT, KICK>(P, H, W, W.slot_atom[k], k, hdt, out, want_energy);
        for (int i = threadIdx.x; i < P.na; i += blockDim.x) {
            const V4<R> p = W.pos[i];
            if (!is_present(p)) continue;
            if (KICK && !is_active(p)) {
                // a frozen atom during a step: only its pair with the ion
                // matters (its own force is never used)
                const R dx = p.x - W.S->rel[0], dy = p.y - W.S->rel[1], dz = p.z - W.S->rel[2];
                const R r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < H.rc2) {
                    R U, rw;
                    const R g = ion_pair<R>(H, P.spline_on, P.rho_on, species_of(p), r2, U, rw);
                    out.fx += g * dx;
                    out.fy += g * dy;
                    out.fz += g * dz;
                    out.rho += rw;
                    out.epot += U;
                    out.pairs += 1;
                }
                continue;
            }
            const unsigned sl = W.need_map[i];
            if (is_active(p) && sl < (unsigned)nact) continue;   // done above
            const int k = (sl < REED_PENDING && want_energy) ? (int)sl : -1;
            atom_force<R, TT, KICK>(P, H, W, i, k, hdt, out, want_energy);
        }
    }
}

// Block-reduce the partials into S->red row 0 (thread 0 reads them).
template <typename R, int TT>
__device__ __forceinline__ void reduce_partials(Win<R, TT>& W, Partial<R>& q)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R fx = warp_sum(q.fx), fy = warp_sum(q.fy), fz = warp_sum(q.fz), rho = warp_sum(q.rho);
    R vm = warp_max(q.vmax2), ep = warp_sum(q.epot), pm = warp_max(q.pmax);
    int pr = warp_sum(q.pairs), bd = warp_sum(q.bonds);
    if (lane == 0) {
        R* row = W.S->red[wid];
        row[0] = fx; row[1] = fy; row[2] = fz; row[3] = rho; row[4] = vm; row[5] = ep;
        row[6] = R(pr); row[7] = R(bd); row[8] = pm;
    }
}

// Sum the per-warp partials (thread 0), fixed order; rows 4 and 8 are maxima.
template <typename R, int TT>
__device__ __forceinline__ void gather_partials(Win<R, TT>& W, R out[REED_NRED])
{
    const int nw = (blockDim.x + 31) >> 5;
    R acc[REED_NRED];
#pragma unroll
    for (int c = 0; c < REED_NRED; ++c) acc[c] = R(0);
    for (int w = 0; w < nw; ++w) {
        const R* row = W.S->red[w];
        for (int c = 0; c < REED_NRED; ++c) {
            if (c == 4 || c == 8) acc[c] = max(acc[c], row[c]);
            else acc[c] += row[c];
        }
    }
    for (int c = 0; c < REED_NRED; ++c) out[c] = acc[c];
}

// Depth of the ion for the tallies and the cloning depths: z below a
// surface, or the distance from the starting site in a bulk target.
template <typename R> __device__ __forceinline__ double track_depth(const DevParams& P, const IonState<R>& I)
{
    if (!P.bulk) return I.x[2];
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(I.x[0], I.x[0]), __dmul_rn(I.x[1], I.x[1])), __dmul_rn(I.x[2], I.x[2])));
}

// Depth bin tally and per-track record of a finished track (Sec. 3: result
// messages become atomics on device tallies).
template <typename R>
__device__ long long finish_track(const DevParams& P, const DevBuf& B, const IonState<R>& I, int status)
{
    long long kept = -1;
    const double w = ldexp(1.0, -I.level);
    if (status >= REED_TRACK_STOPPED && status <= REED_TRACK_TRUNCATED)
        atomicAdd(&B.counters[C_STOP + status - REED_TRACK_STOPPED], 1ull);
    const double z = track_depth(P, I);
    if (status == REED_TRACK_STOPPED) {
        int bin;
        if (z < 0.0) bin = P.nbins;
        else {
            double q = floor(z / P.bin_w);
            bin = q >= (double)P.nbins ? P.nbins + 1 : (int)q;
        }
        atomicAdd(&B.hist[bin], w);
        atomicAdd(&B.wsum[W_STOPPED], w);
    } else if (status == REED_TRACK_BACKSCATTERED) {
        atomicAdd(&B.hist[P.nbins + 2], w);
        atomicAdd(&B.wsum[W_BACK], w);
    } else if (status == REED_TRACK_TRUNCATED) {
        atomicAdd(&B.wsum[W_TRUNC], w);
    } else {
        atomicAdd(&B.wsum[W_FAILED], w);
    }
    if (P.stop_after > 0) atomicAdd(B.finished, 1ull);
    if (P.record) {
        unsigned long long k = atomicAdd(B.record_count, 1ull);
        if ((long long)k < P.record_cap) {
            reed_track_record r;
            r.id = I.id;
            r.primary = I.primary;
            r.z = z;
            r.t = I.t;
            r.steps = I.steps;
            r.level = I.level;
            r.status = status;
            B.records[k] = r;
            kept = (long long)k;
        }
    }
    return kept;
}

// Add a half kick to the ion's velocity.  In FP32 the sum is kept as two
// floats, v + vlo (Knuth's TwoSum), so that increments of a few ulp -- the drag
// on an MeV ion over its 0.05 A steps -- do not round systematically: with a
// plain FP32 sum the 85 MeV Kr drag-only range came out 0.7 % short, with the
// two-float sum within 1e-6.
template <typename R> __device__ __forceinline__ void add_velocity(IonState<R>& I, int d, R inc)
{
    if constexpr (sizeof(R) == 4) {
        const float a = I.v[d], b = __fadd_rn(inc, I.vlo[d]);
        const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
        I.vlo[d] = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        I.v[d] = s;
    } else {
        I.v[d] += inc;
    }
}

// Launch a primary (Sec. 2; lateral position uniform in the (0,0) surface
// cell, start at z = -rc; or a recoil from the origin site of a bulk target,
// the on-lattice ions of Sec. 4.1).
template <typename R> __device__ void launch_primary(const DevParams& P, IonState<R>& I, long long pidx)
{
    I.id = (unsigned long long)(P.first_id + pidx);
    I.primary = I.id;
    I.key = track_key(P.seed, I.id);
    uint32_t w[4];
    draw4(I.key, 0, 0, 0, REED_TAG_LAUNCH, w);
    double th, ph;
    if (P.beam_mode == REED_BEAM_CONE) {
        const double ct = 1.0 - unit_open(w[2]) * (1.0 - P.cos_tmax);
        th = acos(ct);
        ph = 2.0 * REED_PI * unit_open(w[3]);
    } else if (P.beam_mode == REED_BEAM_RECOIL) {
        // uniform over the sphere: cos(theta) uniform in (-1, 1)
        th = acos(1.0 - 2.0 * unit_open(w[2]));
        ph = 2.0 * REED_PI * unit_open(w[3]);
    } else {
        th = P.tilt;
        ph = P.rot_lo + P.rot_span * unit_open(w[2]);
    }
    if (P.beam_mode == REED_BEAM_RECOIL) {   // on the site of basis atom 0 of cell (0,0,0)
        I.x[0] = P.bas[0][0] * P.a;
        I.x[1] = P.bas[0][1] * P.a;
        I.x[2] = P.bas[0][2] * P.a;
    } else {
        I.x[0] = P.a * unit_open(w[0]);
        I.x[1] = P.a * unit_open(w[1]);
        I.x[2] = -P.rc;
    }
    const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
    I.v[0] = R(P.v0 * st * cp);
    I.v[1] = R(P.v0 * st * sp);
    I.v[2] = R(P.v0 * ct);
    I.vlo[0] = I.vlo[1] = I.vlo[2] = R(0);
    I.f[0] = I.f[1] = I.f[2] = R(0);
    I.rho = R(0);
    I.vmax2 = R(0);
    I.pmax = R(0);
    I.t = 0.0;
    I.e_elec = 0.0;
    I.steps = 0;
    I.level = 0;
    for (int d = 0; d < 3; ++d) I.A[d] = (int)floor(I.x[d] / P.a + P.anchor_shift);
}

// Anchor-frame quantities from the FP64 position (track start, window move,
// cloning): the ion's offset from the anchor corner and the depths that the
// per-step checks compare against.
template <typename R> __device__ void set_frame(const DevParams& P, TrackShared<R>* S)
{
    const IonState<R>& I = S->ion;
    for (int d = 0; d < 3; ++d) S->rel[d] = R(I.x[d] - (double)I.A[d] * P.a);
    const double z0 = (double)I.A[2] * P.a;
    if (P.bulk) {   // no surface; the depth checks run on the distance from the start
        S->zthr = I.level < S->nthr ? R(-1e30) : R(1e30);
        S->zback = R(-1e30);
        S->zsurf = R(-1e30);
        return;
    }
    S->zthr = I.level < S->nthr ? R(S->thr[I.level] - z0) : R(1e30);
    S->zback = R(-P.rc - z0);
    S->zsurf = R(-z0);
}

// Electronic drag coefficient (Sec. 2 "Third"): F_e = -k v with
// k = gamma (1 + s_loc (rho / rho0 - 1)) inside the target (z >= 0).
template <typename R> __device__ __forceinline__ R drag_k(const HotParams<R>& H, const TrackShared<R>* S)
{
    if (S->rel[2] < S->zsurf) return R(0);
    return H.gamma * (R(1) + H.s_loc * (S->ion.rho * H.rho0_inv - R(1)));
}

// Prologue of a step (thread 0): dt from the fastest particle, ion half kick
// and drift, window anchor check (Fig. "moving cell": the main cell follows
// the ion).  FP64 work: the position and energy accumulations only.
template <typename R> __device__ void ion_prologue(const DevParams& P, const HotParams<R>& H, TrackShared<R>* S)
{
    IonState<R>& I = S->ion;
    const R v2 = I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2];
    const R vmax = sqrt(max(v2, I.vmax2));
    R dt = H.dt_max;
    if (vmax * dt > H.dx_max) dt = H.dx_max / vmax;
    if (H.de_max > R(0)) {   // energy term: |dE_kin| <= de_max per step for every particle
        const R pw = max(fabs(I.f[0] * I.v[0] + I.f[1] * I.v[1] + I.f[2] * I.v[2]), I.pmax);
        if (pw * dt > H.de_max) {
            dt = H.de_max / pw;
            if (vmax * dt < H.dx_min) dt = H.dx_min / vmax;   // a step that moves nothing stalls
        }
    }
    const R kd = drag_k<R>(H, S);
    S->on1 = S->rel[2] >= S->zsurf;
    const R h = R(0.5) * dt * H.invM1;
    R de = R(0);
    for (int d = 0; d < 3; ++d) {
        const R fe = -kd * I.v[d];
        de -= fe * I.v[d];
        add_velocity<R>(I, d, h * (I.f[d] + fe));
    }
    I.e_elec += (double)(R(0.5) * dt * de);
    int moved = 0;
    for (int d = 0; d < 3; ++d) {
        const R dx = dt * I.v[d];
        I.x[d] += (double)dx;
        S->rel[d] += dx;
        S->Aold[d] = I.A[d];
        // the ion leaves its anchor cell when rel leaves [-h a, (1-h) a)
        if (S->rel[d] >= H.anchor_hi || S->rel[d] < H.anchor_lo) {
            I.A[d] = (int)floor(I.x[d] / P.a + P.anchor_shift);
            moved = 1;
        }
    }
    if (moved) set_frame<R>(P, S);
    S->shift = moved;
    S->dt = dt;
}

// Epilogue (thread 0): ion second half kick, end and cloning checks.
// Returns EV_NONE / EV_END / EV_CLONE; sets S->status and S->nclone.
template <typename R>
__device__ int ion_epilogue(const DevParams& P, const HotParams<R>& H, TrackShared<R>* S, const R red[REED_NRED])
{
    IonState<R>& I = S->ion;
    const R dt = S->dt;
    I.f[0] = red[0];
    I.f[1] = red[1];
    I.f[2] = red[2];
    I.rho = red[3];
    I.vmax2 = red[4];
    I.pmax = red[8];
    const R kd = drag_k<R>(H, S);
    S->on2 = S->rel[2] >= S->zsurf;
    const R h = R(0.5) * dt * H.invM1;
    R de = R(0);
    for (int d = 0; d < 3; ++d) {
        const R fe = -kd * I.v[d];
        de -= fe * I.v[d];
        add_velocity<R>(I, d, h * (I.f[d] + fe));
    }
    I.e_elec += (double)(R(0.5) * dt * de);
    I.t += (double)dt;
    I.steps += 1;
    const R E = R(0.5) * H.M1 * (I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2]);
    int st = 0;
    if (!isfinite(E) || !isfinite(S->rel[0] + S->rel[1] + S->rel[2])) st = REED_TRACK_FAILED;
    else if (E < H.e_stop) st = REED_TRACK_STOPPED;
    else if (S->rel[2] < S->zback && I.v[2] < R(0)) st = REED_TRACK_BACKSCATTERED;
    else if (I.steps >= P.step_cap) st = REED_TRACK_TRUNCATED;
    S->status = st;
    if (st) return EV_END;
    int nc = 0;
    if (S->rel[2] >= S->zthr) {
        // passed one (or more) cloning depths: count them on the FP64 depth
        const double z = track_depth(P, I);
        while (I.level + nc < S->nthr && z >= S->thr[I.level + nc]) ++nc;
    }
    S->nclone = nc;
    return nc ? EV_CLONE : EV_NONE;
}

// Copy the window (pos, vel, frc) between shared memory and a clone record.
// ---------------------------------------------------------------------------
// Shared clone pool (the paper's host handing returned clones to whichever
// client is free, Sec. 3).  Lock-free: a slot is claimed with one CAS and no
// CTA ever waits for a particular other CTA; an idle CTA polls the pool with a
// bounded number of sleeps.  Records pass through L2 only (they are written
// and read by different SMs).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pool_claim(const DevBuf& B, unsigned from, unsigned to)
{
    const int n = B.pool_slots;
    const int start = (int)((blockIdx.x * 2654435761u) % (unsigned)n);
    for (int j = 0; j < n; ++j) {
        int s = start + j;
        if (s >= n) s -= n;
        if (*(volatile unsigned*)&B.pool_state[s] != from) continue;
        if (atomicCAS(&B.pool_state[s], from, to) == from) return s;
    }
    return -1;
}

template <typename R, int TT>
__device__ __forceinline__ void copy_window_cg(const DevParams& P, Win<R, TT>& W, const unsigned char* rec)
{
    using L = Layout<R, TT>;
    const uint4* g = reinterpret_cast<const uint4*>(rec + L::align(sizeof(IonState<R>)));
    const int na = P.na, w = (int)(sizeof(V4<R>) / sizeof(uint4));
    uint4* pos = reinterpret_cast<uint4*>(W.pos);
    uint4* vel = reinterpret_cast<uint4*>(W.vel);
    uint4* frc = reinterpret_cast<uint4*>(W.frc);
    for (int i = threadIdx.x; i < na * w; i += blockDim.x) {
        pos[i] = __ldcg(g + i);
        vel[i] = __ldcg(g + na * w + i);
        frc[i] = __ldcg(g + 2 * na * w + i);
    }
}

template <typename R, int TT>
__device__ __forceinline__ void copy_window(const DevParams& P, Win<R, TT>& W, unsigned char* rec, bool to_rec)
{
    using L = Layout<R, TT>;
    V4<R>* g = reinterpret_cast<V4<R>*>(rec + L::align(sizeof(IonState<R>)));
    const int na = P.na;
    if (to_rec) {
        for (int i = threadIdx.x; i < na; i += blockDim.x) {
            g[i] = W.pos[i];
            g[na + i] = W.vel[i];
            g[2 * na + i] = W.frc[i];
        }
    } else {
        for (int i = threadIdx.x; i < na; i += blockDim.x) {
            W.pos[i] = g[i];
            W.vel[i] = g[na + i];
            W.frc[i] = g[2 * na + i];
        }
    }
}

// Forces + (optionally) target bookkeeping at the start of a track.
template <typename R, int TT>
__device__ void initial_forces(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, unsigned long long& ctr_bonds,
                               unsigned long long& ctr_rebuild, int& nbovf, int& capovf, WorkCount& wc)
{
    if constexpr (TT != REED_TT_NONE) {
        build_neighbours<R, TT>(P, H, W, nbovf, capovf, wc.spilled);
        if (threadIdx.x == 0) ++ctr_rebuild;
        __syncthreads();
        if (P.nl_check) check_lists<R, TT>(P, H, W, H.rlist2, wc.nl_errors);
    }
    if constexpr (TT == REED_TT_TERSOFF) {
        ters_centres<R, TT>(H, W, wc.triplets);
        __syncthreads();
    }
    Partial<R> q = {R(0), R(0), R(0), R(0), R(0), R(0), 0, 0};
    force_phase<R, TT, false>(P, H, W, R(0), q, false);
    reduce_partials<R, TT>(W, q);
    __syncthreads();
    if (threadIdx.x == 0) {
        R red[REED_NRED];
        gather_partials<R, TT>(W, red);
        IonState<R>& I = W.S->ion;
        I.f[0] = red[0];
        I.f[1] = red[1];
        I.f[2] = red[2];
        I.rho = red[3];
        ctr_bonds += (unsigned long long)red[7];
    }
    __syncthreads();
}

#include "reed_adjoint.cuh"

// ---------------------------------------------------------------------------
// The persistent kernel.  ADJ (target model NONE only) adds the checkpoints,
// the step records and the reverse pass of the truncated-segment adjoint.
// The second launch bound is the number of CTAs per SM the shared memory of
// the workloads allows, so registers are budgeted for that occupancy.
// ---------------------------------------------------------------------------
template <typename R, int TT, bool ADJ>
constexpr int track_min_ctas()
{
    if (TT == REED_TT_NONE) return sizeof(R) == 4 ? (ADJ ? 2 : 3) : (ADJ ? 1 : 2);
    return TT == REED_TT_TERSOFF && sizeof(R) == 4 ? 2 : 1;
}

// Threads per track at most: 512 for the pair-list model (one track fills an
// SM's shared memory, so its warps are all the SM gets), else 256.
template <int TT> constexpr int track_max_threads() { return TT == REED_TT_BUCKINGHAM ? 512 : 256; }

template <typename R, int TT, bool ADJ>
__global__ void __launch_bounds__((track_max_threads<TT>()), (track_min_ctas<R, TT, ADJ>())) reed_track_kernel(
    const __grid_constant__ DevParams P, const __grid_constant__ DevBuf B)
{
    static_assert(!ADJ || TT == REED_TT_NONE, "the adjoint runs without target-target forces");
    extern __shared__ __align__(16) unsigned char smem[];
    Win<R, TT> W(smem, P.na, P.bond_cap, ADJ ? 1 : 0, P.g_nbins, P.act_cap,
                 B.spill ? B.spill + (size_t)blockIdx.x * B.spill_stride : nullptr);
    TrackShared<R>* S = W.S;
    const HotParams<R>& H = hot<R>(P);
    const int tid = threadIdx.x;
    unsigned char* adjbase = (ADJ && B.adj) ? B.adj + (size_t)blockIdx.x * B.adj_stride : nullptr;
    unsigned char* stack = B.stacks ? B.stacks + (size_t)blockIdx.x * B.stack_stride : nullptr;

    // thread-0 counters, flushed at exit
    unsigned long long c_prim = 0, c_clone = 0, c_tracks = 0, c_steps = 0, c_pairs = 0, c_bonds = 0,
                       c_shift = 0, c_rebuild = 0, c_drop = 0, c_fail = 0;
    int nbovf = 0, capovf = 0;
    WorkCount wc;
    // phase clocks (thread 0): time between consecutive barriers of a step
    unsigned long long ph[REED_NPHASE] = {0, 0, 0, 0, 0, 0};
    long long t_mark = clock64();
    auto lap = [&](int phase) {
        if (tid == 0) {
            const long long now = clock64();
            ph[phase] += (unsigned long long)(now - t_mark);
            t_mark = now;
        }
    };
    if (tid == 0) {
        S->top = 0;
        for (int c = 0; c < 4; ++c) S->cls_sum[c] = 0;
    }
    W.clear_grid(P);

    for (;;) {
        // ---- acquire a track: own clone stack first, then a new primary
        if (tid == 0) {
            S->nthr = P.nthr;
            for (int k = 0; k < P.nthr; ++k) S->thr[k] = P.thr_from_device ? B.thr[k] : P.thr[k];
            if (S->top > 0) {
                S->src = SRC_CLONE;
            } else if (P.stop_after > 0 &&
                       (long long)(*(volatile unsigned long long*)B.finished) >= P.stop_after) {
                S->src = SRC_NONE;   // enough tracks collected: hand out no more primaries
            } else {
                unsigned long long k = atomicAdd(B.next, 1ull);
                S->pidx = (long long)k;
                S->src = ((long long)k < P.n_primaries) ? SRC_PRIMARY : SRC_NONE;
            }
            if (S->src == SRC_NONE && B.pool) {
                // out of work: take a donated clone, or stop once every CTA is
                // idle and no record is reserved or held
                bool idle = false;
                for (long long it = 0;; ++it) {
                    // scan the slots only when some record is published
                    const int sl = *(volatile unsigned*)&B.pool_ctl[2] > 0u ? pool_claim(B, POOL_FULL, POOL_READING) : -1;
                    if (sl >= 0) {
                        atomicSub(&B.pool_ctl[2], 1u);
                        if (idle) atomicSub(&B.pool_ctl[0], 1u);
                        S->slot = sl;
                        S->src = SRC_STOLEN;
                        break;
                    }
                    if (!idle) {
                        atomicAdd(&B.pool_ctl[0], 1u);
                        idle = true;
                    }
                    if (*(volatile unsigned*)&B.pool_ctl[0] >= gridDim.x && *(volatile unsigned*)&B.pool_ctl[1] == 0u)
                        break;
                    if (it >= P.pool_polls) {
                        atomicOr(B.status, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(it < 64 ? 500u : 4000u);
                }
            }
        }
        __syncthreads();
        const int src = S->src;
        if (src == SRC_NONE) break;
        if (src == SRC_PRIMARY) {
            if (tid == 0) {
                launch_primary<R>(P, S->ion, S->pidx);
                set_frame<R>(P, S);
                ++c_prim;
            }
            __syncthreads();
            const uint64_t key = S->ion.key;
            int A[3] = {S->ion.A[0], S->ion.A[1], S->ion.A[2]};
            for (int i = tid; i < P.na; i += blockDim.x) {
                V4<R> p, v, f;
                make_atom<R>(P, key, i, A, p, v);
                f.x = f.y = f.z = f.w = R(0);
                W.pos[i] = p;
                W.vel[i] = v;
                W.frc[i] = f;
            }
            __syncthreads();
            initial_forces<R, TT>(P, H, W, c_bonds, c_rebuild, nbovf, capovf, wc);
            if constexpr (TT == REED_TT_NONE) {
                if (ADJ && adjbase) {   // checkpoint of the state before step 0
                    save_state<R, TT>(P, W, adjbase);
                    __syncthreads();
                }
            }
        } else if (src == SRC_STOLEN) {
            const unsigned char* rec = B.pool + (size_t)S->slot * B.entry_bytes;
            if (tid == 0) {
                __threadfence();
                const uint4* h = reinterpret_cast<const uint4*>(rec);
                uint4* d = reinterpret_cast<uint4*>(&S->ion);
                for (int k = 0; k < (int)(sizeof(IonState<R>) / sizeof(uint4)); ++k) d[k] = __ldcg(h + k);
                set_frame<R>(P, S);
            }
            copy_window_cg<R, TT>(P, W, rec);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicExch(&B.pool_state[S->slot], (unsigned)POOL_EMPTY);
                atomicSub(&B.pool_ctl[1], 1u);
                if (B.splits) atomicAdd(&B.splits[REED_MAX_THR], 1ull);
            }
            if constexpr (TT != REED_TT_NONE) {
                build_neighbours<R, TT>(P, H, W, nbovf, capovf, wc.spilled);
                if (tid == 0) ++c_rebuild;
            }
            __syncthreads();
        } else {
            unsigned char* rec = stack + (size_t)(S->top - 1) * B.entry_bytes;
            if (tid == 0) {
                S->ion = *reinterpret_cast<const IonState<R>*>(rec);
                set_frame<R>(P, S);
            }
            copy_window<R, TT>(P, W, rec, false);
            __syncthreads();
            if (tid == 0) S->top -= 1;
            if constexpr (TT != REED_TT_NONE) {
                build_neighbours<R, TT>(P, H, W, nbovf, capovf, wc.spilled);
                if (tid == 0) ++c_rebuild;
            }
            __syncthreads();
        }
        const bool tracing = (src == SRC_PRIMARY) && (S->pidx < P.trace_tracks);
        const long long pidx = S->pidx;

        // ---- step loop
        bool need_prologue = true;
        lap(PH_ADMIN);
        for (;;) {
            if (need_prologue) {
                if (tid == 0) ion_prologue<R>(P, H, S);
                __syncthreads();
                lap(PH_ION);
            }
            const R dt = R(S->dt), hdt = R(0.5) * R(S->dt);
            const int shift = S->shift;
            const uint64_t key = S->ion.key;
            Partial<R> q = {R(0), R(0), R(0), R(0), R(0), R(0), 0, 0};
            if constexpr (TT == REED_TT_NONE) {
                // no target-target forces: each atom's whole step (re-anchor,
                // half kick, drift, ion-target force, half kick) in one pass,
                // the same operations as the separate phases of the other models
                for (int i = tid; i < P.na; i += blockDim.x) {
                    V4<R> p = W.pos[i], v = W.vel[i], f = W.frc[i];
                    // half kick and drift of the atoms integrated before the
                    // window moves, then the move (a step's kick and drift
                    // precede its window update)
                    if (is_active(p)) {
                        ++wc.moved;
                        const R k = hdt * H.invM2[species_of(p)];
                        v.x += k * f.x;
                        v.y += k * f.y;
                        v.z += k * f.z;
                        p.x += dt * v.x;
                        p.y += dt * v.y;
                        p.z += dt * v.z;
                    }
                    if (shift) {
                        const V4<R> p0 = p, v0 = v;
                        if (reanchor_atom<R>(P, H, key, i, S->Aold, S->ion.A, p, v, f))
                            deposit_damage<R>(P, B, p0, v0, S->Aold, ldexp(1.0, -S->ion.level));
                    }
                    if (!is_present(p)) {
                        if (shift) {
                            W.pos[i] = p;
                            W.vel[i] = v;
                            W.frc[i] = f;
                        }
                        continue;
                    }
                    const bool act = is_active(p);
                    ion_atom_step<R>(P, H, W.S, p, v, act, hdt, f, q);
                    W.pos[i] = p;
                    W.vel[i] = v;
                    W.frc[i] = f;
                }
                reduce_partials<R, TT>(W, q);
                __syncthreads();
                lap(PH_FORCE);
            } else {
            // phase A: first half kick + drift of the atoms integrated before
            // the window moves, then the move (a step's kick and drift precede
            // its window update: an atom entering the integrated region is
            // first kicked at the end of this step, one leaving it still
            // moves in this step)
            R pm1 = R(0), pm2 = R(0);   // this thread's two longest paths
            for (int i = tid; i < P.na; i += blockDim.x) {
                V4<R> p = W.pos[i];
                const bool act = is_active(p);
                if (!act && !shift) continue;   // frozen atoms do not move
                V4<R> v = W.vel[i], f = W.frc[i];
                if (act) {
                    ++wc.moved;
                    const R k = hdt * H.invM2[species_of(p)];
                    v.x += k * f.x;
                    v.y += k * f.y;
                    v.z += k * f.z;
                    const R sx = dt * v.x, sy = dt * v.y, sz = dt * v.z;
                    p.x += sx;
                    p.y += sy;
                    p.z += sz;
                    if constexpr (TT != REED_TT_NONE) {
                        { const R l2 = sx * sx + sy * sy + sz * sz; if (l2 > R(0)) v.w += l2 * Mth<R>::rsqrt(l2); }
                        if (v.w > pm1) {
                            pm2 = pm1;
                            pm1 = v.w;
                        } else if (v.w > pm2) {
                            pm2 = v.w;
                        }
                    }
                }
                if (shift) {
                    const V4<R> p0 = p, v0 = v;
                    if (reanchor_atom<R>(P, H, key, i, S->Aold, S->ion.A, p, v, f))
                        deposit_damage<R>(P, B, p0, v0, S->Aold, ldexp(1.0, -S->ion.level));
                }
                W.pos[i] = p;
                W.vel[i] = v;
                if (shift) W.frc[i] = f;
            }
            if constexpr (TT != REED_TT_NONE) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const R q1 = __shfl_xor_sync(0xffffffffu, pm1, o), q2 = __shfl_xor_sync(0xffffffffu, pm2, o);
                    pm2 = fmax(fmin(pm1, q1), fmax(pm2, q2));
                    pm1 = fmax(pm1, q1);
                }
                if ((tid & 31) == 0) {
                    S->path2[tid >> 5][0] = pm1;
                    S->path2[tid >> 5][1] = pm2;
                }
                __syncthreads();
                lap(PH_MOVE);
                // every thread merges the per-warp pairs in the same order
                R m1 = R(0), m2 = R(0);
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    const R q1 = S->path2[w][0], q2 = S->path2[w][1];
                    m2 = fmax(fmin(m1, q1), fmax(m2, q2));
                    m1 = fmax(m1, q1);
                }
                if (shift || m1 + m2 > H.skin) {
                    bool refreshed = false;
                    if constexpr (TT == REED_TT_TERSOFF) {
                        if (!shift) refreshed = refresh_lists<R, TT>(P, H, W, nbovf, wc.spilled);
                    }
                    if (!refreshed) build_neighbours<R, TT>(P, H, W, nbovf, capovf, wc.spilled);
                    __syncthreads();
                    if (tid == 0) ++(refreshed ? wc.refreshes : c_rebuild);
                    if (P.nl_check)
                        check_lists<R, TT>(P, H, W, refreshed ? H.tcut * H.tcut : H.rlist2, wc.nl_errors);
                    lap(PH_BUILD);
                }
                if constexpr (TT == REED_TT_TERSOFF) {
                    ters_centres<R, TT>(H, W, wc.triplets);
                    __syncthreads();
                    lap(PH_PASS1);
                    if (tid == 0)
                        for (int c = 0; c < 4; ++c) S->cls_sum[c] += (unsigned)S->ncls[c];
                }
            }
            force_phase<R, TT, true>(P, H, W, hdt, q, false);
            reduce_partials<R, TT>(W, q);
            __syncthreads();
            lap(PH_FORCE);
            }
            if (tid == 0) {
                R red[REED_NRED];
                gather_partials<R, TT>(W, red);
                c_pairs += (unsigned long long)red[6];
                c_bonds += (unsigned long long)red[7];
                c_shift += shift;
                ++c_steps;
                int ev = ion_epilogue<R>(P, H, S, red);
                if (tracing && S->ion.steps <= P.trace_steps) {
                    const IonState<R>& I = S->ion;
                    size_t o = (size_t)pidx * P.trace_steps + (size_t)(I.steps - 1);
                    double* t8 = B.trace + 8 * o;
                    t8[0] = I.x[0]; t8[1] = I.x[1]; t8[2] = I.x[2]; t8[3] = I.t;
                    t8[4] = I.v[0]; t8[5] = I.v[1]; t8[6] = I.v[2]; t8[7] = S->dt;
                    int* a3 = B.trace_anchor + 3 * o;
                    a3[0] = I.A[0]; a3[1] = I.A[1]; a3[2] = I.A[2];
                }
                if (adjbase) {
                    // frozen quantities of this step; checkpoints every adj_every steps
                    StepRec<R>* ring = reinterpret_cast<StepRec<R>*>(adjbase + (size_t)P.adj_nck * B.entry_bytes);
                    StepRec<R> sr;
                    sr.dt = S->dt;
                    sr.A[0] = S->ion.A[0];
                    sr.A[1] = S->ion.A[1];
                    sr.A[2] = S->ion.A[2];
                    sr.flags = (S->on1 ? 1 : 0) | (S->on2 ? 2 : 0) | (shift ? 4 : 0);
                    ring[(S->ion.steps - 1) % REED_STEP_RING] = sr;
                    if (ev == EV_NONE && S->ion.steps % P.adj_every == 0) ev = EV_CKPT;
                }
                S->event = ev;
                if (ev == EV_NONE) ion_prologue<R>(P, H, S);
            }
            __syncthreads();
            lap(PH_ION);
            const int ev = S->event;
            if (ev == EV_NONE) {
                need_prologue = false;
                continue;
            }
            need_prologue = true;
            if (ev == EV_END) break;
            if (ev == EV_CKPT) {
                if constexpr (TT == REED_TT_NONE) {
                    save_state<R, TT>(P, W, adjbase + (size_t)((S->ion.steps / P.adj_every) % P.adj_nck) * B.entry_bytes);
                    __syncthreads();
                }
                continue;
            }
            // ---- cloning (Sec. 2): push one record per level passed
            const int nc = S->nclone;
            __syncthreads();
            for (int c = 0; c < nc; ++c) {
                // some CTA is idle: donate this clone to the pool instead
                if (tid == 0) {
                    S->slot = -1;
                    if (B.pool && *(volatile unsigned*)&B.pool_ctl[0] > 0u) {
                        atomicAdd(&B.pool_ctl[1], 1u);   // counted before the slot is visible
                        S->slot = pool_claim(B, POOL_EMPTY, POOL_WRITING);
                        if (S->slot < 0) atomicSub(&B.pool_ctl[1], 1u);
                    }
                }
                __syncthreads();
                if (S->slot >= 0) {
                    unsigned char* rec = B.pool + (size_t)S->slot * B.entry_bytes;
                    if (tid == 0) {
                        IonState<R>& I = S->ion;
                        I.level += 1;
                        IonState<R> C = I;
                        C.id = clone_id(I.id, I.level);
                        C.key = track_key(P.seed, C.id);
                        *reinterpret_cast<IonState<R>*>(rec) = C;
                        ++c_clone;
                        if (B.splits) atomicAdd(&B.splits[min(I.level, REED_MAX_THR) - 1], 1ull);
                    }
                    copy_window<R, TT>(P, W, rec, true);
                    __threadfence();
                    __syncthreads();
                    if (tid == 0) {
                        atomicExch(&B.pool_state[S->slot], (unsigned)POOL_FULL);
                        atomicAdd(&B.pool_ctl[2], 1u);
                    }
                    __syncthreads();
                    continue;
                }
                if (S->top >= B.stack_depth || stack == nullptr) {
                    if (tid == 0) {
                        c_drop += (unsigned long long)(nc - c);
                        atomicOr(B.status, ERR_QUEUE);
                        // the track still passes the levels (its depths stay in step with its
                        // weight 2^-level), so the dropped clones' weight is lost from the
                        // profile; the run reports REED_E_QUEUE_FULL
                        S->ion.level += nc - c;
                    }
                    __syncthreads();
                    break;
                }
                unsigned char* rec = stack + (size_t)S->top * B.entry_bytes;
                if (tid == 0) {
                    IonState<R>& I = S->ion;
                    I.level += 1;
                    IonState<R> C = I;
                    C.id = clone_id(I.id, I.level);
                    C.key = track_key(P.seed, C.id);
                    *reinterpret_cast<IonState<R>*>(rec) = C;
                    ++c_clone;
                    if (B.splits) atomicAdd(&B.splits[min(I.level, REED_MAX_THR) - 1], 1ull);
                }
                copy_window<R, TT>(P, W, rec, true);
                __syncthreads();
                if (tid == 0) S->top += 1;
                __syncthreads();
            }
            if (tid == 0) set_frame<R>(P, S);   // next cloning depth
            __syncthreads();
        }
        // ---- track finished
        lap(PH_ADMIN);
        if (B.damage) {
            const int A[3] = {S->ion.A[0], S->ion.A[1], S->ion.A[2]};
            const double wgt = ldexp(1.0, -S->ion.level);
            for (int i = tid; i < P.na; i += blockDim.x) {
                const V4<R> p = W.pos[i];
                if (is_active(p)) deposit_damage<R>(P, B, p, W.vel[i], A, wgt);
            }
            __syncthreads();
        }
        if (tid == 0) {
            if (S->status == REED_TRACK_FAILED) {
                ++c_fail;
                atomicOr(B.status, ERR_NONFINITE);
            }
            S->rec_index = finish_track<R>(P, B, S->ion, S->status);
            ++c_tracks;
        }
        __syncthreads();
        if constexpr (ADJ) {
            // truncated-segment sensitivities of the final depth
            if (adjbase && B.grads && S->rec_index >= 0) {
                double g[REED_NTHETA] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (S->status == REED_TRACK_STOPPED) {
                    AdjScratch<R, TT> A(adjbase, P, B.entry_bytes);
                    adjoint_track<R, TT>(P, H, W, A, g);
                }
                if (tid == 0)
                    for (int k = 0; k < REED_NTHETA; ++k) B.grads[(size_t)S->rec_index * REED_NTHETA + k] = g[k];
                __syncthreads();
            }
        }
    }
    if (nbovf || capovf) atomicOr(B.status, ERR_NEIGHBOR);
    // flush counters
    int ov = nbovf, oc = capovf;
    for (int o = 16; o > 0; o >>= 1) {
        ov += __shfl_xor_sync(0xffffffffu, ov, o);
        oc += __shfl_xor_sync(0xffffffffu, oc, o);
    }
    if ((tid & 31) == 0 && ov) atomicAdd(&B.counters[C_NBOVF], (unsigned long long)ov);
    if ((tid & 31) == 0 && oc) atomicAdd(&B.counters[C_CAPOVF], (unsigned long long)oc);
    unsigned long long tr = wc.triplets, mv = wc.moved;
    for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
        mv += __shfl_xor_sync(0xffffffffu, mv, o);
    }
    if ((tid & 31) == 0) {
        if (tr) atomicAdd(&B.counters[C_TRIPLETS], tr);
        atomicAdd(&B.counters[C_MOVED], mv);
    }
    if (tid == 0 && wc.spilled) atomicAdd(&B.counters[C_SPILLED], wc.spilled);
    if (tid == 0 && wc.refreshes) atomicAdd(&B.counters[C_REFRESH], wc.refreshes);
    if (TT == REED_TT_TERSOFF && tid == 0)
        for (int c = 0; c < 4; ++c)
            if (S->cls_sum[c]) atomicAdd(&B.counters[C_CLS0 + c], S->cls_sum[c]);
    if (wc.nl_errors) atomicAdd(&B.counters[C_NLCHECK], wc.nl_errors);
    if (tid == 0) {
        atomicAdd(&B.counters[C_PRIMARIES], c_prim);
        atomicAdd(&B.counters[C_CLONES], c_clone);
        atomicAdd(&B.counters[C_TRACKS], c_tracks);
        atomicAdd(&B.counters[C_STEPS], c_steps);
        atomicAdd(&B.counters[C_PAIRS], c_pairs);
        atomicAdd(&B.counters[C_BONDS], c_bonds);
        atomicAdd(&B.counters[C_SHIFTS], c_shift);
        atomicAdd(&B.counters[C_REBUILDS], c_rebuild);
        atomicAdd(&B.counters[C_DROPPED], c_drop);
        atomicAdd(&B.counters[C_FAILED], c_fail);
        lap(PH_ADMIN);
        for (int k = 0; k < REED_NPHASE; ++k) atomicAdd(&B.counters[C_PHASE0 + k], ph[k]);
    }
}
