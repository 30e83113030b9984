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

enum { SRC_NONE = 0, SRC_PRIMARY = 1, SRC_CLONE = 2 };
enum { EV_NONE = 0, EV_END = 1, EV_CLONE = 2 };

// Ion state (FP64) as stored in shared memory and in clone records.
struct IonState {
    double x[3], v[3], f[3];
    double rho, t, e_elec, vmax2;
    long long steps;
    unsigned long long id, primary, key;
    int A[3];
    int level;
};

template <typename R> struct TrackShared {
    IonState ion;
    double dt;
    R rel[3];
    int Aold[3];
    int shift, rebuild, event, status, src, top, nclone, need_count;
    long long pidx;
    R red[REED_MAX_WARPS][8];
};

template <typename R> struct V2 { R a, b; };

// Shared-memory carve-up for a window of na atoms.  Tersoff bond data is
// stored only for "needed" atoms (integrated, or bonded to an integrated
// atom), at most bond_cap of them, through a compact index need_map.
template <typename R, int TT> struct Layout {
    static __host__ __device__ size_t align(size_t x) { return (x + 15) & ~(size_t)15; }
    static __host__ __device__ size_t shared_bytes() { return align(sizeof(TrackShared<R>)); }
    static __host__ __device__ size_t atoms_bytes(int na) { return 3 * align(sizeof(V4<R>) * na); }
    static __host__ __device__ size_t nbr_bytes(int na)
    {
        return TT == REED_TT_NONE ? 0 : align(sizeof(uint16_t) * na * REED_MAXNB) + align(na) +
                                            align(sizeof(uint16_t) * na);
    }
    static __host__ __device__ size_t bond_bytes(int bond_cap)
    {
        return TT == REED_TT_TERSOFF ? align(sizeof(V2<R>) * bond_cap * REED_MAXNB) : 0;
    }
    static __host__ __device__ size_t total(int na, int bond_cap)
    {
        return shared_bytes() + atoms_bytes(na) + nbr_bytes(na) + bond_bytes(bond_cap);
    }
    // bytes of one clone record: ion header + pos, vel, frc
    static __host__ __device__ size_t entry_bytes(int na) { return align(sizeof(IonState)) + atoms_bytes(na); }
};

#define REED_NO_SLOT 0xFFFFu

template <typename R, int TT> struct Win {
    TrackShared<R>* S;
    V4<R>* pos;
    V4<R>* vel;
    V4<R>* frc;
    uint16_t* nbr;
    uint8_t* nnb;
    uint16_t* need_map;
    V2<R>* bond;
    __device__ Win(unsigned char* base, int na)
    {
        using L = Layout<R, TT>;
        S = reinterpret_cast<TrackShared<R>*>(base);
        size_t o = L::shared_bytes();
        size_t ab = L::align(sizeof(V4<R>) * na);
        pos = reinterpret_cast<V4<R>*>(base + o);
        vel = reinterpret_cast<V4<R>*>(base + o + ab);
        frc = reinterpret_cast<V4<R>*>(base + o + 2 * ab);
        o += 3 * ab;
        nbr = nullptr;
        nnb = nullptr;
        need_map = nullptr;
        bond = nullptr;
        if constexpr (TT != REED_TT_NONE) {
            nbr = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * na * REED_MAXNB);
            nnb = reinterpret_cast<uint8_t*>(base + o);
            o += L::align(na);
            need_map = reinterpret_cast<uint16_t*>(base + o);
            o += L::align(sizeof(uint16_t) * na);
        }
        if constexpr (TT == REED_TT_TERSOFF) bond = reinterpret_cast<V2<R>*>(base + o);
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
// thermal displacements).  Cells with z index < 0 are above the surface.
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
    if (c[2] < 0) {
        p.x = p.y = p.z = R(0);
        p.w = R(REED_W_EMPTY);
        return;
    }
    double g[3] = {0.0, 0.0, 0.0};
    if (P.sigma > 0.0) {
        uint32_t w[4];
        draw4(key, c[0], c[1], c[2], ((uint32_t)b << 4) | REED_TAG_CELL, w);
        box_muller3(w, g);
    }
    p.x = R(((double)(c[0] - A[0]) + P.bas[b][0]) * P.a + P.sigma * g[0]);
    p.y = R(((double)(c[1] - A[1]) + P.bas[b][1]) * P.a + P.sigma * g[1]);
    p.z = R(((double)(c[2] - A[2]) + P.bas[b][2]) * P.a + P.sigma * g[2]);
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
template <typename R> __device__ __forceinline__ bool is_active(const V4<R>& p) { return p.w >= R(0) && p.w < R(2); }
template <typename R> __device__ __forceinline__ int species_of(const V4<R>& p) { return ((int)p.w) & 1; }

// ---------------------------------------------------------------------------
// Target neighbour lists (Tersoff / pair terms): all present atoms within
// rlist = cutoff + skin (brute force over the window).  nnb[i] holds the
// count; need_map[i] the compact bond-storage slot of atoms that are
// integrated or bonded to an integrated atom (REED_NO_SLOT otherwise).
// Called by all threads right after a barrier.
template <typename R, int TT>
__device__ void build_neighbours(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, int& overflow)
{
    const int na = P.na;
    if (threadIdx.x == 0) W.S->need_count = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        V4<R> pi = W.pos[i];
        W.need_map[i] = (uint16_t)REED_NO_SLOT;
        if (!is_present(pi)) {
            W.nnb[i] = 0;
            continue;
        }
        int cnt = 0;
        bool need = is_active(pi);
        for (int j = 0; j < na; ++j) {
            if (j == i) continue;
            V4<R> pj = W.pos[j];
            if (!is_present(pj)) continue;
            R dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < H.rlist2) {
                if (cnt < REED_MAXNB) {
                    W.nbr[i * REED_MAXNB + cnt] = (uint16_t)j;
                    ++cnt;
                } else {
                    ++overflow;
                }
                need = need || is_active(pj);
            }
        }
        W.nnb[i] = (uint8_t)cnt;
        if (TT == REED_TT_TERSOFF && need) {
            int slot = atomicAdd(&W.S->need_count, 1);
            if (slot < P.bond_cap) W.need_map[i] = (uint16_t)slot;
            else ++overflow;
        }
        W.vel[i].w = R(0);   // path length since the list was built
    }
}

// Tersoff pass 1 for atom a: for each bond (a, b) of its list store
// {pre_ab = 1/2 dV_ab/db * db/dzeta_ab, dV_ab/dr} and return 1/2 sum V_ab.
template <typename R, int TT>
__device__ R ters_pass1(const HotParams<R>& H, Win<R, TT>& W, int a)
{
    const int m = W.nnb[a];
    V2<R>* bond = W.bond + (size_t)W.need_map[a] * REED_MAXNB;
    const V4<R> pa = W.pos[a];
    R dx[REED_MAXNB], dy[REED_MAXNB], dz[REED_MAXNB], r[REED_MAXNB], ir[REED_MAXNB], fc[REED_MAXNB];
#pragma unroll
    for (int q = 0; q < REED_MAXNB; ++q) {
        if (q < m) {
            V4<R> pb = W.pos[W.nbr[a * REED_MAXNB + q]];
            dx[q] = pb.x - pa.x;
            dy[q] = pb.y - pa.y;
            dz[q] = pb.z - pa.z;
            R r2 = dx[q] * dx[q] + dy[q] * dy[q] + dz[q] * dz[q];
            ir[q] = Mth<R>::rsqrt(r2);
            r[q] = r2 * ir[q];
            R dfc;
            fc[q] = ters_fc<R>(H, r[q], dfc);
        }
    }
    R E = R(0);
#pragma unroll
    for (int q = 0; q < REED_MAXNB; ++q) {
        if (q < m) {
            R zeta = R(0);
#pragma unroll
            for (int k = 0; k < REED_MAXNB; ++k) {
                if (k < m && k != q && fc[k] > R(0)) {
                    R c = (dx[q] * dx[k] + dy[q] * dy[k] + dz[q] * dz[k]) * ir[q] * ir[k];
                    R dg;
                    zeta += fc[k] * ters_g<R>(H, c, dg);
                }
            }
            R db;
            R b = ters_b<R>(H, zeta, db);
            R V, dV, pfa;
            ters_pair<R>(H, r[q], b, V, dV, pfa);
            V2<R> out;
            out.a = R(0.5) * pfa * db;
            out.b = dV;
            bond[q] = out;
            E += R(0.5) * V;
        }
    }
    return E;
}

// Tersoff pass 2: force on atom i gathered from every term of the energy
// that depends on its position (bonds of i, bonds to i, and bonds of its
// neighbours in which i is the third atom).
template <typename R, int TT>
__device__ void ters_pass2(const HotParams<R>& H, Win<R, TT>& W, int i, R& Fx, R& Fy, R& Fz)
{
    const int m = W.nnb[i];
    if (W.need_map[i] == REED_NO_SLOT) return;
    const V2<R>* bond_i = W.bond + (size_t)W.need_map[i] * REED_MAXNB;
    const V4<R> pi = W.pos[i];
    R ux[REED_MAXNB], uy[REED_MAXNB], uz[REED_MAXNB], r[REED_MAXNB], fc[REED_MAXNB], dfc[REED_MAXNB];
#pragma unroll
    for (int q = 0; q < REED_MAXNB; ++q) {
        if (q < m) {
            V4<R> pb = W.pos[W.nbr[i * REED_MAXNB + q]];
            R dx = pb.x - pi.x, dy = pb.y - pi.y, dz = pb.z - pi.z;
            R r2 = dx * dx + dy * dy + dz * dz;
            R irr = Mth<R>::rsqrt(r2);
            r[q] = r2 * irr;
            ux[q] = dx * irr;
            uy[q] = dy * irr;
            uz[q] = dz * irr;
            fc[q] = ters_fc<R>(H, r[q], dfc[q]);
        }
    }
    R fx = R(0), fy = R(0), fz = R(0);
    // bonds (i, b): radial part and i as the centre of zeta_ib
#pragma unroll
    for (int q = 0; q < REED_MAXNB; ++q) {
        if (q < m) {
            V2<R> bq = bond_i[q];
            R h = R(0.5) * bq.b;
            fx += h * ux[q];
            fy += h * uy[q];
            fz += h * uz[q];
            R gx = R(0), gy = R(0), gz = R(0);   // d zeta_iq / d x_i
            if (bq.a != R(0)) {
#pragma unroll
                for (int k = 0; k < REED_MAXNB; ++k) {
                    if (k < m && k != q && (fc[k] > R(0))) {
                        R c = ux[q] * ux[k] + uy[q] * uy[k] + uz[q] * uz[k];
                        R dg, g = ters_g<R>(H, c, dg);
                        R irq = Mth<R>::rcp(r[q]), irk = Mth<R>::rcp(r[k]);
                        // d c / d x_i = -[(u_k - c u_q)/r_q + (u_q - c u_k)/r_k]
                        R cx = (ux[k] - c * ux[q]) * irq + (ux[q] - c * ux[k]) * irk;
                        R cy = (uy[k] - c * uy[q]) * irq + (uy[q] - c * uy[k]) * irk;
                        R cz = (uz[k] - c * uz[q]) * irq + (uz[q] - c * uz[k]) * irk;
                        R t = fc[k] * dg;
                        gx += -dfc[k] * g * ux[k] - t * cx;
                        gy += -dfc[k] * g * uy[k] - t * cy;
                        gz += -dfc[k] * g * uz[k] - t * cz;
                    }
                }
                fx -= bq.a * gx;
                fy -= bq.a * gy;
                fz -= bq.a * gz;
            }
        }
    }
    // bonds (a, i) and (a, b) for each neighbour a of i
#pragma unroll
    for (int q = 0; q < REED_MAXNB; ++q) {
        if (q < m) {
            const int a = W.nbr[i * REED_MAXNB + q];
            const int ma = W.nnb[a];
            if (W.need_map[a] == REED_NO_SLOT) continue;
            const V2<R>* bond_a = W.bond + (size_t)W.need_map[a] * REED_MAXNB;
            const V4<R> pa = W.pos[a];
            // unit vector a -> i and its length
            const R vx = -ux[q], vy = -uy[q], vz = -uz[q];
            const R irai = Mth<R>::rcp(r[q]);
            R ax = R(0), ay = R(0), az = R(0);   // sum fc(r_ab) g'(c) t  (d zeta_ai / d x_i)
            R pre_ai = R(0), dV_ai = R(0);
            for (int p = 0; p < ma; ++p) {
                const int b = W.nbr[a * REED_MAXNB + p];
                const V2<R> bab = bond_a[p];
                if (b == i) {
                    pre_ai = bab.a;
                    dV_ai = bab.b;
                    continue;
                }
                const V4<R> pb = W.pos[b];
                R dx = pb.x - pa.x, dy = pb.y - pa.y, dz = pb.z - pa.z;
                R r2 = dx * dx + dy * dy + dz * dz;
                R irab = Mth<R>::rsqrt(r2);
                R rab = r2 * irab;
                R wx = dx * irab, wy = dy * irab, wz = dz * irab;
                R c = vx * wx + vy * wy + vz * wz;
                R dg, g = ters_g<R>(H, c, dg);
                R tx = (wx - c * vx) * irai, ty = (wy - c * vy) * irai, tz = (wz - c * vz) * irai;
                R dfab, fab = ters_fc<R>(H, rab, dfab);
                ax += fab * dg * tx;
                ay += fab * dg * ty;
                az += fab * dg * tz;
                // i as the third atom of zeta_ab
                R s1 = dfc[q] * g, s2 = fc[q] * dg;
                fx -= bab.a * (s1 * vx + s2 * tx);
                fy -= bab.a * (s1 * vy + s2 * ty);
                fz -= bab.a * (s1 * vz + s2 * tz);
            }
            fx -= pre_ai * ax;
            fy -= pre_ai * ay;
            fz -= pre_ai * az;
            R h = R(0.5) * dV_ai;
            fx += h * ux[q];
            fy += h * uy[q];
            fz += h * uz[q];
        }
    }
    Fx += fx;
    Fy += fy;
    Fz += fz;
}

// Buckingham / short-range pair forces on atom i from its list (each pair is
// visited from both ends; the energy is halved).
template <typename R, int TT>
__device__ R pair_force(const HotParams<R>& H, Win<R, TT>& W, int i, R& Fx, R& Fy, R& Fz)
{
    const int m = W.nnb[i];
    const V4<R> pi = W.pos[i];
    const int si = species_of(pi);
    R E = R(0);
    for (int q = 0; q < m; ++q) {
        const V4<R> pj = W.pos[W.nbr[i * REED_MAXNB + q]];
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
};

// Force evaluation over the whole window; with KICK the second half kick is
// applied to integrated atoms and their speed^2 reduced for the next dt.
// Writes W.frc for every present atom.
template <typename R, int TT, bool KICK>
__device__ void force_phase(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, R hdt, Partial<R>& out,
                            bool want_energy)
{
    const R ix = W.S->rel[0], iy = W.S->rel[1], iz = W.S->rel[2];
    for (int i = threadIdx.x; i < P.na; i += blockDim.x) {
        V4<R> p = W.pos[i];
        if (!is_present(p)) continue;
        const bool act = is_active(p);
        R fx = R(0), fy = R(0), fz = R(0);
        const R dx = p.x - ix, dy = p.y - iy, dz = p.z - iz;
        const R r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < H.rc2) {
            R U, rw;
            const R g = ion_pair<R>(H, P.spline_on, P.rho_on, species_of(p), r2, U, rw);
            fx = -g * dx;
            fy = -g * dy;
            fz = -g * dz;
            out.fx += g * dx;
            out.fy += g * dy;
            out.fz += g * dz;
            out.rho += rw;
            out.epot += U;
            out.pairs += 1;
        }
        if constexpr (TT == REED_TT_TERSOFF) {
            if (act) {
                ters_pass2<R, TT>(H, W, i, fx, fy, fz);
                out.bonds += W.nnb[i];
            }
        }
        if constexpr (TT == REED_TT_BUCKINGHAM) {
            if (act || want_energy) {
                out.epot += pair_force<R, TT>(H, W, i, fx, fy, fz);
                out.bonds += W.nnb[i];
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
            const R k = hdt * H.invM2[species_of(p)];
            v.x += k * fx;
            v.y += k * fy;
            v.z += k * fz;
            W.vel[i] = v;
            out.vmax2 = max(out.vmax2, v.x * v.x + v.y * v.y + v.z * v.z);
        }
    }
}

// Block-reduce the partials into S->red row 0 (thread 0 reads them).
template <typename R, int TT>
__device__ __forceinline__ void reduce_partials(Win<R, TT>& W, Partial<R>& q)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R fx = warp_sum(q.fx), fy = warp_sum(q.fy), fz = warp_sum(q.fz), rho = warp_sum(q.rho);
    R vm = warp_max(q.vmax2), ep = warp_sum(q.epot);
    int pr = warp_sum(q.pairs), bd = warp_sum(q.bonds);
    if (lane == 0) {
        R* row = W.S->red[wid];
        row[0] = fx; row[1] = fy; row[2] = fz; row[3] = rho; row[4] = vm; row[5] = ep;
        row[6] = R(pr); row[7] = R(bd);
    }
}

// Sum the per-warp partials (thread 0), fixed order.
template <typename R, int TT>
__device__ __forceinline__ void gather_partials(Win<R, TT>& W, double out[8])
{
    const int nw = (blockDim.x + 31) >> 5;
    for (int c = 0; c < 8; ++c) out[c] = 0.0;
    R acc[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int w = 0; w < nw; ++w) {
        const R* row = W.S->red[w];
        for (int c = 0; c < 8; ++c) {
            if (c == 4) acc[4] = max(acc[4], row[4]);
            else acc[c] += row[c];
        }
    }
    for (int c = 0; c < 8; ++c) out[c] = (double)acc[c];
}

// Depth bin tally and per-track record of a finished track (Sec. 3: result
// messages become atomics on device tallies).
static __device__ void finish_track(const DevParams& P, const DevBuf& B, const IonState& I, int status)
{
    const double w = ldexp(1.0, -I.level);
    if (status >= REED_TRACK_STOPPED && status <= REED_TRACK_TRUNCATED)
        atomicAdd(&B.counters[C_STOP + status - REED_TRACK_STOPPED], 1ull);
    if (status == REED_TRACK_STOPPED) {
        const double z = I.x[2];
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
    if (P.record) {
        unsigned long long k = atomicAdd(B.record_count, 1ull);
        if ((long long)k < P.record_cap) {
            reed_track_record r;
            r.id = I.id;
            r.primary = I.primary;
            r.z = I.x[2];
            r.t = I.t;
            r.steps = I.steps;
            r.level = I.level;
            r.status = status;
            B.records[k] = r;
        }
    }
}

// Launch a primary (Sec. 2; lateral position uniform in the (0,0) surface
// cell, start at z = -rc).
static __device__ void launch_primary(const DevParams& P, IonState& I, long long pidx)
{
    I.id = (unsigned long long)(P.first_id + pidx);
    I.primary = I.id;
    I.key = track_key(P.seed, I.id);
    uint32_t w[4];
    draw4(I.key, 0, 0, 0, REED_TAG_LAUNCH, w);
    double th, ph;
    if (P.beam_mode == REED_BEAM_CONE) {
        double ct = 1.0 - unit_open(w[2]) * (1.0 - P.cos_tmax);
        th = acos(ct);
        ph = 2.0 * REED_PI * unit_open(w[3]);
    } else {
        th = P.tilt;
        ph = P.rot_lo + P.rot_span * unit_open(w[2]);
    }
    I.x[0] = P.a * unit_open(w[0]);
    I.x[1] = P.a * unit_open(w[1]);
    I.x[2] = -P.rc;
    double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
    I.v[0] = P.v0 * st * cp;
    I.v[1] = P.v0 * st * sp;
    I.v[2] = P.v0 * ct;
    I.f[0] = I.f[1] = I.f[2] = 0.0;
    I.rho = 0.0;
    I.t = 0.0;
    I.e_elec = 0.0;
    I.vmax2 = 0.0;
    I.steps = 0;
    I.level = 0;
    for (int d = 0; d < 3; ++d) I.A[d] = (int)floor(I.x[d] / P.a + P.anchor_shift);
}

template <typename R> __device__ __forceinline__ void set_rel(const DevParams& P, TrackShared<R>* S)
{
    for (int d = 0; d < 3; ++d) S->rel[d] = R(S->ion.x[d] - (double)S->ion.A[d] * P.a);
}

// Prologue of a step (thread 0): dt, ion half kick + drift, anchor check.
template <typename R> __device__ void ion_prologue(const DevParams& P, TrackShared<R>* S)
{
    IonState& I = S->ion;
    const double v2 = I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2];
    const double vmax = sqrt(fmax(v2, I.vmax2));
    double dt = P.dt_max;
    if (vmax * dt > P.dx_max) dt = P.dx_max / vmax;
    const double kd = drag_coeff(P, I.x[2], I.rho);
    const double h = 0.5 * dt * P.invM1;
    for (int d = 0; d < 3; ++d) {
        const double fe = -kd * I.v[d];
        I.e_elec -= 0.5 * dt * fe * I.v[d];
        I.v[d] += h * (I.f[d] + fe);
    }
    int moved = 0;
    for (int d = 0; d < 3; ++d) {
        I.x[d] += dt * I.v[d];
        const int Ad = (int)floor(I.x[d] / P.a + P.anchor_shift);
        S->Aold[d] = I.A[d];
        if (Ad != I.A[d]) moved = 1;
        I.A[d] = Ad;
    }
    S->shift = moved;
    S->dt = dt;
    set_rel<R>(P, S);
}

// Epilogue (thread 0): ion second half kick, end and cloning checks.
// Returns EV_NONE / EV_END / EV_CLONE; sets S->status and S->nclone.
template <typename R> __device__ int ion_epilogue(const DevParams& P, TrackShared<R>* S, const double red[8])
{
    IonState& I = S->ion;
    const double dt = S->dt;
    I.f[0] = red[0];
    I.f[1] = red[1];
    I.f[2] = red[2];
    I.rho = red[3];
    I.vmax2 = red[4];
    const double kd = drag_coeff(P, I.x[2], I.rho);
    const double h = 0.5 * dt * P.invM1;
    for (int d = 0; d < 3; ++d) {
        const double fe = -kd * I.v[d];
        I.e_elec -= 0.5 * dt * fe * I.v[d];
        I.v[d] += h * (I.f[d] + fe);
    }
    I.t += dt;
    I.steps += 1;
    const double v2 = I.v[0] * I.v[0] + I.v[1] * I.v[1] + I.v[2] * I.v[2];
    const double E = 0.5 * P.M1 * v2;
    int st = 0;
    if (!isfinite(E) || !isfinite(I.x[0] + I.x[1] + I.x[2])) st = REED_TRACK_FAILED;
    else if (E < P.e_stop) st = REED_TRACK_STOPPED;
    else if (I.x[2] < -P.rc && I.v[2] < 0.0) st = REED_TRACK_BACKSCATTERED;
    else if (I.steps >= P.step_cap) st = REED_TRACK_TRUNCATED;
    S->status = st;
    if (st) return EV_END;
    int nc = 0;
    while (I.level + nc < P.nthr && I.x[2] >= P.thr[I.level + nc]) ++nc;
    S->nclone = nc;
    return nc ? EV_CLONE : EV_NONE;
}

// Copy the window (pos, vel, frc) between shared memory and a clone record.
template <typename R, int TT>
__device__ __forceinline__ void copy_window(const DevParams& P, Win<R, TT>& W, unsigned char* rec, bool to_rec)
{
    using L = Layout<R, TT>;
    V4<R>* g = reinterpret_cast<V4<R>*>(rec + L::align(sizeof(IonState)));
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
                               unsigned long long& ctr_rebuild, int& nbovf)
{
    if constexpr (TT != REED_TT_NONE) {
        build_neighbours<R, TT>(P, H, W, nbovf);
        if (threadIdx.x == 0) ++ctr_rebuild;
        __syncthreads();
    }
    if constexpr (TT == REED_TT_TERSOFF) {
        for (int a = threadIdx.x; a < P.na; a += blockDim.x)
            if (W.need_map[a] != REED_NO_SLOT) ters_pass1<R, TT>(H, W, a);
        __syncthreads();
    }
    Partial<R> q = {R(0), R(0), R(0), R(0), R(0), R(0), 0, 0};
    force_phase<R, TT, false>(P, H, W, R(0), q, false);
    reduce_partials<R, TT>(W, q);
    __syncthreads();
    if (threadIdx.x == 0) {
        double red[8];
        gather_partials<R, TT>(W, red);
        IonState& I = W.S->ion;
        I.f[0] = red[0];
        I.f[1] = red[1];
        I.f[2] = red[2];
        I.rho = red[3];
        ctr_bonds += (unsigned long long)red[7];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// The persistent kernel.
// ---------------------------------------------------------------------------
template <typename R, int TT>
__global__ void __launch_bounds__(256) reed_track_kernel(const __grid_constant__ DevParams P,
                                                         const __grid_constant__ DevBuf B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Win<R, TT> W(smem, P.na);
    TrackShared<R>* S = W.S;
    const HotParams<R>& H = hot<R>(P);
    const int tid = threadIdx.x;
    unsigned char* stack = B.stacks ? B.stacks + (size_t)blockIdx.x * B.stack_stride : nullptr;

    // thread-0 counters, flushed at exit
    unsigned long long c_prim = 0, c_clone = 0, c_tracks = 0, c_steps = 0, c_pairs = 0, c_bonds = 0,
                       c_shift = 0, c_rebuild = 0, c_drop = 0, c_fail = 0;
    int nbovf = 0;
    if (tid == 0) S->top = 0;

    for (;;) {
        // ---- acquire a track: own clone stack first, then a new primary
        if (tid == 0) {
            S->rebuild = 0;
            if (S->top > 0) {
                S->src = SRC_CLONE;
            } else {
                unsigned long long k = atomicAdd(B.next, 1ull);
                S->pidx = (long long)k;
                S->src = ((long long)k < P.n_primaries) ? SRC_PRIMARY : SRC_NONE;
            }
        }
        __syncthreads();
        const int src = S->src;
        if (src == SRC_NONE) break;
        if (src == SRC_PRIMARY) {
            if (tid == 0) {
                launch_primary(P, S->ion, S->pidx);
                set_rel<R>(P, S);
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
            initial_forces<R, TT>(P, H, W, c_bonds, c_rebuild, nbovf);
        } else {
            unsigned char* rec = stack + (size_t)(S->top - 1) * B.entry_bytes;
            if (tid == 0) {
                S->ion = *reinterpret_cast<const IonState*>(rec);
                set_rel<R>(P, S);
            }
            copy_window<R, TT>(P, W, rec, false);
            __syncthreads();
            if (tid == 0) S->top -= 1;
            if constexpr (TT != REED_TT_NONE) {
                build_neighbours<R, TT>(P, H, W, nbovf);
                if (tid == 0) ++c_rebuild;
            }
            __syncthreads();
        }
        const bool tracing = (src == SRC_PRIMARY) && (S->pidx < P.trace_tracks);
        const long long pidx = S->pidx;

        // ---- step loop
        bool need_prologue = true;
        for (;;) {
            if (need_prologue) {
                if (tid == 0) ion_prologue<R>(P, S);
                __syncthreads();
            }
            const R dt = R(S->dt), hdt = R(0.5) * R(S->dt);
            const int shift = S->shift;
            const uint64_t key = S->ion.key;
            // phase A: re-anchor and first half kick + drift of own atoms
            bool any_new = false;
            for (int i = tid; i < P.na; i += blockDim.x) {
                V4<R> p = W.pos[i], v = W.vel[i], f = W.frc[i];
                if (shift) any_new |= reanchor_atom<R>(P, H, key, i, S->Aold, S->ion.A, p, v, f);
                if (is_active(p)) {
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
                        if (v.w > H.skin_half) S->rebuild = 1;
                    }
                }
                W.pos[i] = p;
                W.vel[i] = v;
                if (shift) W.frc[i] = f;
            }
            (void)any_new;
            if constexpr (TT != REED_TT_NONE) {
                if (tid == 0 && shift) S->rebuild = 1;
                __syncthreads();
                if (S->rebuild) {
                    build_neighbours<R, TT>(P, H, W, nbovf);
                    __syncthreads();
                    if (tid == 0) {
                        S->rebuild = 0;
                        ++c_rebuild;
                    }
                }
                if constexpr (TT == REED_TT_TERSOFF) {
                    for (int a = tid; a < P.na; a += blockDim.x)
                        if (W.need_map[a] != REED_NO_SLOT) ters_pass1<R, TT>(H, W, a);
                    __syncthreads();
                }
            }
            Partial<R> q = {R(0), R(0), R(0), R(0), R(0), R(0), 0, 0};
            force_phase<R, TT, true>(P, H, W, hdt, q, false);
            reduce_partials<R, TT>(W, q);
            __syncthreads();
            if (tid == 0) {
                double red[8];
                gather_partials<R, TT>(W, red);
                c_pairs += (unsigned long long)red[6];
                c_bonds += (unsigned long long)red[7];
                c_shift += shift;
                ++c_steps;
                int ev = ion_epilogue<R>(P, S, red);
                if (tracing && S->ion.steps <= P.trace_steps) {
                    const IonState& I = S->ion;
                    size_t o = (size_t)pidx * P.trace_steps + (size_t)(I.steps - 1);
                    double* t8 = B.trace + 8 * o;
                    t8[0] = I.x[0]; t8[1] = I.x[1]; t8[2] = I.x[2]; t8[3] = I.t;
                    t8[4] = I.v[0]; t8[5] = I.v[1]; t8[6] = I.v[2]; t8[7] = S->dt;
                    int* a3 = B.trace_anchor + 3 * o;
                    a3[0] = I.A[0]; a3[1] = I.A[1]; a3[2] = I.A[2];
                }
                S->event = ev;
                if (ev == EV_NONE) ion_prologue<R>(P, S);
            }
            __syncthreads();
            const int ev = S->event;
            if (ev == EV_NONE) {
                need_prologue = false;
                continue;
            }
            need_prologue = true;
            if (ev == EV_END) break;
            // ---- cloning (Sec. 2): push one record per level passed
            const int nc = S->nclone;
            for (int c = 0; c < nc; ++c) {
                if (S->top >= B.stack_depth || stack == nullptr) {
                    if (tid == 0) {
                        c_drop += (unsigned long long)(nc - c);
                        atomicOr(B.status, ERR_QUEUE);
                        S->ion.level += nc - c;   // keep weights consistent: the track carries all levels
                    }
                    __syncthreads();
                    break;
                }
                unsigned char* rec = stack + (size_t)S->top * B.entry_bytes;
                if (tid == 0) {
                    IonState& I = S->ion;
                    I.level += 1;
                    IonState C = I;
                    C.id = clone_id(I.id, I.level);
                    C.key = track_key(P.seed, C.id);
                    *reinterpret_cast<IonState*>(rec) = C;
                    ++c_clone;
                }
                copy_window<R, TT>(P, W, rec, true);
                __syncthreads();
                if (tid == 0) S->top += 1;
                __syncthreads();
            }
        }
        // ---- track finished
        if (tid == 0) {
            if (S->status == REED_TRACK_FAILED) {
                ++c_fail;
                atomicOr(B.status, ERR_NONFINITE);
            }
            finish_track(P, B, S->ion, S->status);
            ++c_tracks;
        }
        __syncthreads();
    }
    if (nbovf) atomicOr(B.status, ERR_NEIGHBOR);
    // flush counters
    int ov = nbovf;
    for (int o = 16; o > 0; o >>= 1) ov += __shfl_xor_sync(0xffffffffu, ov, o);
    if ((tid & 31) == 0 && ov) atomicAdd(&B.counters[C_NBOVF], (unsigned long long)ov);
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
    }
}
