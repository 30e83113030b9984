// reed_adjoint.cuh -- reverse-mode sensitivities of a track's final depth
// to theta = (s_e, s_loc, c_1..c_6) over its truncated last segment.
//
// While a track runs with the adjoint on, its complete state is written to a
// per-CTA ring every `every` steps and each step's frozen quantities (dt,
// anchor after the step, drag on/off at both half kicks, window move) to a
// step ring.  When the track has stopped at step T, the segment starts at
// s0 = every * floor((T - seg) / every) (0 if T <= seg); the state at s0 is
// held fixed and so are the frozen quantities.  The gradient of z_T is then
// propagated backwards block by block: each block of `every` steps is
// re-run forward from its checkpoint (states kept in global scratch) and
// walked in reverse through the kick-drift-kick map:
//
//   v_h = v + (h/M)(F(x) + Fe(v, x)),  x' = x + dt v_h,
//   v'  = v_h + (h/M)(F(x') + Fe(v_h, x')),
//
// with F = -grad U (ion-target pairs U(r) = V_ZBL e^{c(r)} S(r)), so that
// the transposed Jacobian needs Hessian-vector products of the pair terms,
// dF/dc_k for the correction coefficients, and the drag's derivatives in
// s_e, s_loc and (through the local density) in the positions.  Cells
// created at a window move do not depend on earlier states: their adjoints
// are zero before the move.  Target-target forces and cloning are not part
// of this path (the workload is a ZBL-only window without splitting).
#pragma once

#include "reed_physics.cuh"

enum { REED_NTHETA = 8 };
#define REED_STEP_RING 256

// Frozen quantities of one step.
template <typename R> struct StepRec {
    R dt;
    int A[3];    // anchor after the step
    int flags;   // bit 0: drag on at the first half kick, bit 1: at the second, bit 2: window moved
};

// Quintic taper's second derivative.
template <typename R> __device__ __forceinline__ R taper_d2(R r, R lo, R inv_w)
{
    const R t = (r - lo) * inv_w;
    if (t <= R(0) || t >= R(1)) return R(0);
    return (R(-60) * t + R(180) * t * t - R(120) * t * t * t) * inv_w * inv_w;
}

// Ion-target pair: dU/dr, d2U/dr2, d(dU/dr)/dc_k and the density weight's
// radial derivative (dS/dr - S/lam) e^{-r/lam}.
template <typename R>
__device__ void ion_pair_d2(const HotParams<R>& H, int spline_on, int s, R r, R& dU, R& d2U, R dUdc[6], R& rhod)
{
    const R ir = R(1) / r;
    const R k = H.zk[s], ia = H.zia[s];
    const R x = r * ia;
    const R e0 = Mth<R>::exp2n(R(-3.19980 * 1.4426950408889634) * x);
    const R e1 = Mth<R>::exp2n(R(-0.94229 * 1.4426950408889634) * x);
    const R e2 = Mth<R>::exp2n(R(-0.40290 * 1.4426950408889634) * x);
    const R e3 = Mth<R>::exp2n(R(-0.20162 * 1.4426950408889634) * x);
    const R phi = R(0.18175) * e0 + R(0.50986) * e1 + R(0.28022) * e2 + R(0.02817) * e3;
    const R dphi = -(R(0.18175 * 3.19980) * e0 + R(0.50986 * 0.94229) * e1 + R(0.28022 * 0.40290) * e2 +
                     R(0.02817 * 0.20162) * e3);
    const R d2phi = R(0.18175 * 3.19980 * 3.19980) * e0 + R(0.50986 * 0.94229 * 0.94229) * e1 +
                    R(0.28022 * 0.40290 * 0.40290) * e2 + R(0.02817 * 0.20162 * 0.20162) * e3;
    const R V = k * phi * ir;
    const R V1 = k * ir * (dphi * ia - phi * ir);
    const R V2 = k * ir * (d2phi * ia * ia - R(2) * dphi * ia * ir + R(2) * phi * ir * ir);
    R c = R(0), c1 = R(0), c2 = R(0), Bk[6], B1k[6];
    const R lr = Mth<R>::log(r);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const R u = (lr - H.spline_ctr[i]) * H.spline_invh;
        R du;
        const R b = bspline3<R>(u, du);
        const R au = fabs(u);
        const R d2 = au >= R(2) ? R(0) : (au >= R(1) ? R(2) - au : R(-2) + R(3) * au);
        Bk[i] = b;
        B1k[i] = du * H.spline_invh * ir;
        if (spline_on) {
            c += H.spline_c[i] * b;
            c1 += H.spline_c[i] * B1k[i];
            c2 += H.spline_c[i] * (d2 * H.spline_invh * H.spline_invh - du * H.spline_invh) * ir * ir;
        }
    }
    const R E = spline_on ? Mth<R>::exp(c) : R(1);
    R dS;
    const R S = taper<R>(r, H.rt, H.inv_tw, dS);
    const R d2S = taper_d2<R>(r, H.rt, H.inv_tw);
    dU = V1 * E * S + V * E * c1 * S + V * E * dS;
    d2U = V2 * E * S + R(2) * V1 * E * c1 * S + R(2) * V1 * E * dS + V * E * (c1 * c1 + c2) * S +
          R(2) * V * E * c1 * dS + V * E * d2S;
#pragma unroll
    for (int i = 0; i < 6; ++i) dUdc[i] = Bk[i] * dU + V * E * S * B1k[i];
    rhod = (dS - S * H.lam_inv) * Mth<R>::exp(-r * H.lam_inv);
}

// Per-CTA adjoint scratch: checkpoint ring, step ring, block states.
template <typename R, int TT> struct AdjScratch {
    unsigned char* ring;
    StepRec<R>* steps;
    unsigned char* block;
    size_t entry;
    __device__ AdjScratch(unsigned char* base, const DevParams& P, size_t entry_bytes)
    {
        entry = entry_bytes;
        ring = base;
        steps = reinterpret_cast<StepRec<R>*>(base + (size_t)P.adj_nck * entry);
        block = base + (size_t)P.adj_nck * entry + Layout<R, TT>::align(sizeof(StepRec<R>) * REED_STEP_RING);
    }
    static __host__ __device__ size_t bytes(const DevParams& P, size_t entry_bytes)
    {
        return (size_t)P.adj_nck * entry_bytes + Layout<R, TT>::align(sizeof(StepRec<R>) * REED_STEP_RING) +
               (size_t)(P.adj_every + 1) * entry_bytes;
    }
};

// Partial sums of one adjoint pass (reduced per warp into S->red).
template <typename R> struct AdjPartial {
    R xb[3];      // ion position adjoint increment
    R dth[6];     // theta_bar increments for c_1..c_6
    R rhos[3];    // sum_j rho'_j rhat_j (drag gradient through the local density)
};

// One pass of the transposed step Jacobian at positions `pos` (global,
// anchor frame of `A`) with ion at `irel` (same frame): for every atom,
// ub_j = hm_j vbar_j; xbar_j -= K (ub_j - ub_i) - (v.ub_i) crho rho'_j rhat_j;
// returns the ion and theta partial sums.
template <typename R, int TT>
__device__ void adj_pass(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, const V4<R>* __restrict__ pos,
                         const R irel[3], R h, const R ubi[3], R vdot_ub, R crho, AdjPartial<R>& q)
{
    for (int j = threadIdx.x; j < P.na; j += blockDim.x) {
        const V4<R> p = pos[j];
        if (!is_present(p)) continue;
        const R dx = p.x - irel[0], dy = p.y - irel[1], dz = p.z - irel[2];
        const R r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= H.rc2) continue;
        const R r = sqrt(r2);
        const R ux = dx / r, uy = dy / r, uz = dz / r;
        R dU, d2U, dUdc[6], rhod;
        ion_pair_d2<R>(H, P.spline_on, species_of(p), r, dU, d2U, dUdc, rhod);
        V4<R> vb = W.vbar[j];
        const R hm = is_active(p) ? h * H.invM2[species_of(p)] : R(0);
        const R dbx = hm * vb.x - ubi[0], dby = hm * vb.y - ubi[1], dbz = hm * vb.z - ubi[2];
        const R ud = ux * dbx + uy * dby + uz * dbz;
        const R t = dU / r;
        const R kx = d2U * ux * ud + t * (dbx - ux * ud);
        const R ky = d2U * uy * ud + t * (dby - uy * ud);
        const R kz = d2U * uz * ud + t * (dbz - uz * ud);
        V4<R> xb = W.xbar[j];
        const R dr = vdot_ub * crho * rhod;
        xb.x -= kx + dr * ux;
        xb.y -= ky + dr * uy;
        xb.z -= kz + dr * uz;
        W.xbar[j] = xb;
        q.xb[0] += kx;
        q.xb[1] += ky;
        q.xb[2] += kz;
        q.rhos[0] += rhod * ux;
        q.rhos[1] += rhod * uy;
        q.rhos[2] += rhod * uz;
#pragma unroll
        for (int k = 0; k < 6; ++k) q.dth[k] -= dUdc[k] * ud;
    }
}

template <typename R, int TT> __device__ __forceinline__ void adj_reduce(Win<R, TT>& W, AdjPartial<R>& q)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R v[12] = {q.xb[0], q.xb[1], q.xb[2], q.dth[0], q.dth[1], q.dth[2], q.dth[3], q.dth[4], q.dth[5],
               q.rhos[0], q.rhos[1], q.rhos[2]};
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = warp_sum(v[c]);
    if (lane == 0)
        for (int c = 0; c < 12; ++c) W.S->adj_red[wid][c] = v[c];
}

template <typename R, int TT> __device__ __forceinline__ void adj_gather(Win<R, TT>& W, R out[12])
{
    const int nw = (blockDim.x + 31) >> 5;
    for (int c = 0; c < 12; ++c) out[c] = R(0);
    for (int w = 0; w < nw; ++w)
        for (int c = 0; c < 12; ++c) out[c] += W.S->adj_red[w][c];
}

// Was slot i replaced (its cell dropped) when the anchor moved Aold -> Anew?
__device__ __forceinline__ bool slot_replaced(const DevParams& P, int i, const int Aold[3], const int Anew[3])
{
    int s[3], b;
    slot_coords(P, i, s, b);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int Lo = Aold[d] - P.half_n;
        const int c = Lo + pmod(s[d] - Lo, P.n);
        const int on = c - (Anew[d] - P.half_n);
        if (on < 0 || on >= P.n) return true;
    }
    return false;
}

// Store / load the full state (ion + window) in the clone-record format.
template <typename R, int TT>
__device__ __forceinline__ void save_state(const DevParams& P, Win<R, TT>& W, unsigned char* rec)
{
    if (threadIdx.x == 0) *reinterpret_cast<IonState<R>*>(rec) = W.S->ion;
    copy_window<R, TT>(P, W, rec, true);
}
template <typename R, int TT>
__device__ __forceinline__ void load_state(const DevParams& P, Win<R, TT>& W, const unsigned char* rec)
{
    if (threadIdx.x == 0) W.S->ion = *reinterpret_cast<const IonState<R>*>(rec);
    copy_window<R, TT>(P, W, const_cast<unsigned char*>(rec), false);
}
template <typename R, int TT> __device__ __forceinline__ const V4<R>* state_pos(const unsigned char* rec)
{
    return reinterpret_cast<const V4<R>*>(rec + Layout<R, TT>::align(sizeof(IonState<R>)));
}

// One frozen forward step (replay): the recorded dt, anchor and drag flags;
// the arithmetic is that of the running step.
template <typename R, int TT>
__device__ void replay_step(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, const StepRec<R>& sr)
{
    TrackShared<R>* S = W.S;
    if (threadIdx.x == 0) {
        IonState<R>& I = S->ion;
        const R dt = sr.dt;
        const R kd = (sr.flags & 1) ? H.gamma * (R(1) + H.s_loc * (I.rho * H.rho0_inv - R(1))) : R(0);
        const R h = R(0.5) * dt * H.invM1;
        for (int d = 0; d < 3; ++d) {
            const R fe = -kd * I.v[d];
            add_velocity<R>(I, d, h * (I.f[d] + fe));
        }
        for (int d = 0; d < 3; ++d) {
            const R dx = dt * I.v[d];
            I.x[d] += (double)dx;
            S->rel[d] += dx;
            S->Aold[d] = I.A[d];
        }
        S->shift = (sr.flags & 4) ? 1 : 0;
        if (S->shift) {
            for (int d = 0; d < 3; ++d) I.A[d] = sr.A[d];
            set_frame<R>(P, S);
        }
        S->dt = dt;
    }
    __syncthreads();
    const R dt = S->dt, hdt = R(0.5) * S->dt;
    const int shift = S->shift;
    for (int i = threadIdx.x; i < P.na; i += blockDim.x) {
        V4<R> p = W.pos[i], v = W.vel[i], f = W.frc[i];
        if (is_active(p)) {   // (kick and drift precede the window move, as in the forward step)
            const R k = hdt * H.invM2[species_of(p)];
            v.x += k * f.x;
            v.y += k * f.y;
            v.z += k * f.z;
            p.x += dt * v.x;
            p.y += dt * v.y;
            p.z += dt * v.z;
        }
        if (shift) reanchor_atom<R>(P, H, S->ion.key, i, S->Aold, S->ion.A, p, v, f);
        W.pos[i] = p;
        W.vel[i] = v;
        if (shift) W.frc[i] = f;
    }
    Partial<R> q = {R(0), R(0), R(0), R(0), R(0), R(0), 0, 0};
    force_phase<R, TT, true>(P, H, W, hdt, q, false);
    reduce_partials<R, TT>(W, q);
    __syncthreads();
    if (threadIdx.x == 0) {
        R red[REED_NRED];
        gather_partials<R, TT>(W, red);
        IonState<R>& I = S->ion;
        for (int d = 0; d < 3; ++d) I.f[d] = red[d];
        I.rho = red[3];
        I.vmax2 = red[4];
        const R kd = (sr.flags & 2) ? H.gamma * (R(1) + H.s_loc * (I.rho * H.rho0_inv - R(1))) : R(0);
        const R h = R(0.5) * sr.dt * H.invM1;
        for (int d = 0; d < 3; ++d) {
            const R fe = -kd * I.v[d];
            add_velocity<R>(I, d, h * (I.f[d] + fe));
        }
        I.t += (double)sr.dt;
        I.steps += 1;
    }
    __syncthreads();
}

// Reverse pass over the truncated segment of the track that just stopped.
// Writes dz_T/dtheta into g[8] (thread 0).  All threads call it.
template <typename R, int TT>
__device__ void adjoint_track(const DevParams& P, const HotParams<R>& H, Win<R, TT>& W, AdjScratch<R, TT>& A,
                              double g[REED_NTHETA])
{
    TrackShared<R>* S = W.S;
    const long long T = S->ion.steps;
    const long long seg = P.adj_seg, every = P.adj_every;
    const long long s0 = T > seg ? every * ((T - seg) / every) : 0;
    // seed: the final depth
    for (int i = threadIdx.x; i < P.na; i += blockDim.x) {
        V4<R> z = {R(0), R(0), R(0), R(0)};
        W.xbar[i] = z;
        W.vbar[i] = z;
    }
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            S->xbi[d] = R(0);
            S->vbi[d] = R(0);
        }
        S->xbi[2] = R(1);
        for (int k = 0; k < REED_NTHETA; ++k) S->gth[k] = 0.0;
    }
    __syncthreads();
    const R g0 = H.gamma0, rho0i = H.rho0_inv;
    for (long long bs = s0 + every * ((T - 1 - s0) / every); bs >= s0; bs -= every) {
        const long long be = min(bs + every, T);
        // restore the checkpoint and re-run the block, keeping every state
        load_state<R, TT>(P, W, A.ring + (size_t)((bs / every) % P.adj_nck) * A.entry);
        __syncthreads();
        if (threadIdx.x == 0) set_frame<R>(P, S);
        __syncthreads();
        save_state<R, TT>(P, W, A.block);
        __syncthreads();
        for (long long s = bs; s < be; ++s) {
            replay_step<R, TT>(P, H, W, A.steps[s % REED_STEP_RING]);
            save_state<R, TT>(P, W, A.block + (size_t)(s + 1 - bs) * A.entry);
            __syncthreads();
        }
        // reverse through the block
        for (long long s = be - 1; s >= bs; --s) {
            const StepRec<R> sr = A.steps[s % REED_STEP_RING];
            const unsigned char* r0 = A.block + (size_t)(s - bs) * A.entry;
            const unsigned char* r1 = r0 + A.entry;
            const IonState<R>& I0 = *reinterpret_cast<const IonState<R>*>(r0);
            const IonState<R>& I1 = *reinterpret_cast<const IonState<R>*>(r1);
            const R dt = sr.dt, h = R(0.5) * sr.dt;
            // (a) cells created by this step's window move owe nothing to earlier states
            if (sr.flags & 4) {
                for (int i = threadIdx.x; i < P.na; i += blockDim.x)
                    if (slot_replaced(P, i, I0.A, I1.A)) {
                        V4<R> z = {R(0), R(0), R(0), R(0)};
                        W.xbar[i] = z;
                        W.vbar[i] = z;
                    }
            }
            // ion quantities of the second half kick
            if (threadIdx.x == 0) {
                const R k1 = (sr.flags & 1) ? H.gamma * (R(1) + H.s_loc * (I0.rho * rho0i - R(1))) : R(0);
                const R hm = h * H.invM1;
                R vh[3];
                for (int d = 0; d < 3; ++d) vh[d] = I0.v[d] + hm * (I0.f[d] - k1 * I0.v[d]);
                R vub = R(0);
                for (int d = 0; d < 3; ++d) {
                    S->ubi[d] = hm * S->vbi[d];
                    S->vh[d] = vh[d];
                    vub += vh[d] * S->ubi[d];
                }
                S->vub = vub;
                for (int d = 0; d < 3; ++d) S->irel[d] = R(I1.x[d] - (double)I1.A[d] * P.a);
            }
            __syncthreads();
            // (b) transposed Jacobian of the second kick at x'
            const R crho = H.gamma * H.s_loc * rho0i;
            {
                AdjPartial<R> q = {{R(0), R(0), R(0)}, {R(0), R(0), R(0), R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
                adj_pass<R, TT>(P, H, W, state_pos<R, TT>(r1), S->irel, h, S->ubi, (sr.flags & 2) ? S->vub : R(0),
                                crho, q);
                adj_reduce<R, TT>(W, q);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                R sum[12];
                adj_gather<R, TT>(W, sum);
                const R on = (sr.flags & 2) ? R(1) : R(0);
                const R k2 = on * H.gamma * (R(1) + H.s_loc * (I1.rho * rho0i - R(1)));
                for (int d = 0; d < 3; ++d) S->xbi[d] += sum[d] + on * S->vub * crho * sum[9 + d];
                for (int k = 0; k < 6; ++k) S->gth[2 + k] += (double)sum[3 + k];
                S->gth[0] -= (double)(on * g0 * (R(1) + H.s_loc * (I1.rho * rho0i - R(1))) * S->vub);
                S->gth[1] -= (double)(on * H.gamma / (H.gamma0 > R(0) ? H.gamma0 : R(1)) * g0 *
                                      (I1.rho * rho0i - R(1)) * S->vub);
                // v_bar at the half step, then (c): x' = x + dt v_h
                for (int d = 0; d < 3; ++d) {
                    S->vbi[d] -= k2 * S->ubi[d];
                    S->vbi[d] += dt * S->xbi[d];
                }
                const R k1 = (sr.flags & 1) ? H.gamma * (R(1) + H.s_loc * (I0.rho * rho0i - R(1))) : R(0);
                const R hm = h * H.invM1;
                R vub = R(0);
                for (int d = 0; d < 3; ++d) {
                    S->ubi[d] = hm * S->vbi[d];
                    vub += I0.v[d] * S->ubi[d];
                }
                S->vub = vub;
                S->k1 = k1;
                for (int d = 0; d < 3; ++d) S->irel[d] = R(I0.x[d] - (double)I0.A[d] * P.a);
            }
            __syncthreads();
            // (c) for the atoms, then (d) transposed Jacobian of the first kick at x
            for (int j = threadIdx.x; j < P.na; j += blockDim.x) {
                V4<R> vb = W.vbar[j];
                const V4<R> xb = W.xbar[j];
                vb.x += dt * xb.x;
                vb.y += dt * xb.y;
                vb.z += dt * xb.z;
                W.vbar[j] = vb;
            }
            __syncthreads();
            {
                AdjPartial<R> q = {{R(0), R(0), R(0)}, {R(0), R(0), R(0), R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
                adj_pass<R, TT>(P, H, W, state_pos<R, TT>(r0), S->irel, h, S->ubi, (sr.flags & 1) ? S->vub : R(0),
                                crho, q);
                adj_reduce<R, TT>(W, q);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                R sum[12];
                adj_gather<R, TT>(W, sum);
                const R on = (sr.flags & 1) ? R(1) : R(0);
                for (int d = 0; d < 3; ++d) S->xbi[d] += sum[d] + on * S->vub * crho * sum[9 + d];
                for (int k = 0; k < 6; ++k) S->gth[2 + k] += (double)sum[3 + k];
                S->gth[0] -= (double)(on * g0 * (R(1) + H.s_loc * (I0.rho * rho0i - R(1))) * S->vub);
                S->gth[1] -= (double)(on * H.gamma / (H.gamma0 > R(0) ? H.gamma0 : R(1)) * g0 *
                                      (I0.rho * rho0i - R(1)) * S->vub);
                for (int d = 0; d < 3; ++d) S->vbi[d] -= S->k1 * S->ubi[d];
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < REED_NTHETA; ++k) g[k] = S->gth[k];
}
