// The two kernels of one TLSPH step (Algorithm 1) and their diagnostics.
//
// Pass 1 (k_gradient + k_stress; one thread per particle, SELL-32 neighbour slices):
//   F_i = I + B_i Ahat_i,  B_i = sum_j V_j w_ij (u_j - u_i) (X_j - X_i)^T
// which is eq. deformGradTLSPH with the corrected gradient L_i gradW_ij =
// w_ij Ahat_i (X_j - X_i); soft particles (s_i <= s_l) take F = I
// (eq. defGrad_phase).  Then the stress (NH / J2), the history functional,
// and the per-particle matrices pass 2 needs:
//   Q_i = P_i Ahat_i,  Vm_i = J_i F_i^-T Ahat_i.
// Pass 2 (same layout):
//   a_i = (1/rho_i) [Q_i sum_j V_j w d + sum_j V_j w Q_j d]   (eq. MomentumEqTLSPH, symmetric form)
//       - Vm_i sum_j m_j pi_ij w d                            (eq. artViscCoef, Pv = -J pi F^-T)
//   lap s_i = -2 Ahat_i : sum_j (s_i - s_j) V_j w d d^T / r^2  (eq. phasefieldLapLacian)
// plus body and boundary forces, the phase-field acceleration
// (eq. phasefieldddot), the Algorithm 1 update, and the per-specimen maxima of
// |v| and |a| for the next step size; the last block to finish advances the
// specimen clocks (eq. dt_criterion).
#pragma once
#include "common.cuh"
#include "expr_eval.cuh"
#include "lattice.cuh"
#include "mlp.cuh"
#include "mlp_tc.cuh"

namespace tl {

// Value a boundary condition prescribes for component k of particle i (slot = the condition's place in
// the particle's group, f = its ramp factor at the time in question, >= 0): the ramped constant, or
// the value its expression took at the start of the step.  False when the expression skips it.
template <typename T>
__device__ __forceinline__ bool dev_bc_value(const StepArgs<T> &a, const BCDev &bc, int i, int slot, int phase,
                                             int k, double f, double &val) {
    if (bc.expr[k] >= 0) {
        const int q = 2 * a.expos[i] + phase;
        if ((a.exskip[q] >> (3 * slot + k)) & 1u) return false;
        val = a.exval[q * 12 + 3 * slot + k];
        return true;
    }
    val = f * bc.value[k];
    return true;
}

template <typename T, int DIM> __device__ __forceinline__ void load_ahat(const T *Ahat, int n, int i, T A[3][3]) {
    if (DIM == 3) {
        A[0][0] = Ahat[i];
        A[1][1] = Ahat[n + i];
        A[2][2] = Ahat[2 * n + i];
        A[0][1] = A[1][0] = Ahat[3 * n + i];
        A[0][2] = A[2][0] = Ahat[4 * n + i];
        A[1][2] = A[2][1] = Ahat[5 * n + i];
    } else {
        A[0][0] = Ahat[i];
        A[1][1] = Ahat[n + i];
        A[0][1] = A[1][0] = Ahat[3 * n + i];
    }
}

template <typename T> __device__ __forceinline__ bool finite_t(T x) { return isfinite(x); }

// Visit the neighbours j of particle i in ascending sorted index, calling pair(j, on).  Stencil
// layout (a.nsten > 0): the warp's 32 consecutive rows walk the stencil differences together
// and row i takes the entries its mask keeps, so the k-th reads of the warp are consecutive
// particles (one table per specimen when each specimen has its own row pitch; a warp that
// spans two specimens reads two tables).  The differences come in runs of consecutive values (one row of a lattice
// stencil each), so the k-th entry of a run reads at a fixed offset from the run's base.  An
// entry the mask drops comes as pair(i + D, false), reading another particle or the zero halo
// around the gathered arrays: the body runs without a branch (the unrolled run issues its
// loads together) and must add exact zeros.  With SKIP, an entry that no row of the warp keeps
// is skipped (a warp vote), which saves its loads at the faces of a block.  Without RUNS the
// entries are walked one by one (UNROLL at a time across runs, each reading its difference).
// SELL-32 layout otherwise: entry k of row i at slice_off[i / 32] + 32 k + i % 32.
// Debug builds (TLSPH_DEBUG) check every neighbour index before it is used: a stencil slot may point into
// the zero halo around the gathered arrays, an active neighbour and a CSR entry must be a particle.  A bad
// index sets a flag (reported by the step as a status) and the access is skipped; nothing traps.
template <typename T> __device__ __forceinline__ bool neighbour_ok(const StepArgs<T> &a, int j, bool on) {
#ifdef TLSPH_DEBUG
    const bool in_particles = j >= 0 && j < a.n;
    const bool ok = a.nsten > 0 ? (j >= -a.halo && j < a.n + a.halo && (!on || in_particles)) : in_particles;
    if (!ok) atomicAdd(&a.flags[kFlagBounds], 1);
    return ok;
#else
    (void)a;
    (void)j;
    (void)on;
    return true;
#endif
}

template <int UNROLL = 4, bool SKIP = false, bool RUNS = true, typename T, typename Pair>
__device__ __forceinline__ void for_each_neighbour(const StepArgs<T> &a, int i, Pair &&pair) {
    // the row's stencil table: its specimen's, when each specimen has its own
    const int tab = a.nsten > 0 && a.sten_groups > 1 ? a.spec[i] * kMaxStencil : 0;
    if (!RUNS && a.nsten > 0) {
        for (int s0 = 0; s0 < a.nsten; s0 += 32) {
            const unsigned m = __ldg(a.nmask + (int64_t)(s0 >> 5) * a.n + i);
            const int lim = min(32, a.nsten - s0);
            const int *off = a.soff + tab + s0;
#pragma unroll UNROLL
            for (int b = 0; b < lim; b++) {
                const bool on = (m >> b) & 1u;
                if (SKIP && !__any_sync(__activemask(), on)) continue;
                const int j = i + __ldg(off + b);
                if (neighbour_ok(a, j, on)) pair(j, on);
            }
        }
    } else if (a.nsten > 0) {
        const int nw = (a.nsten + 31) >> 5;
        unsigned mw[4];
#pragma unroll
        for (int q = 0; q < 4; q++) mw[q] = q < nw ? __ldg(a.nmask + (int64_t)q * a.n + i) : 0u;
        for (int r = 0; r < a.nruns; r++) {
            const int2 rr = __ldg(a.runs + tab + r);
            const int s0 = rr.y & 255, len = rr.y >> 8;
            const int w0 = s0 >> 5;
            const unsigned lo = w0 == 0 ? mw[0] : w0 == 1 ? mw[1] : w0 == 2 ? mw[2] : mw[3];
            const unsigned hi = w0 == 0 ? mw[1] : w0 == 1 ? mw[2] : w0 == 2 ? mw[3] : 0u;
            const unsigned bits = __funnelshift_r(lo, hi, s0 & 31);
            const int io = i + rr.x;
#pragma unroll
            for (int k = 0; k < kMaxRun; k++) {
                if (k < len) {
                    const bool on = (bits >> k) & 1u;
                    if (SKIP && !__any_sync(__activemask(), on)) continue;
                    if (neighbour_ok(a, io + k, on)) pair(io + k, on);
                }
            }
        }
    } else {
        const int64_t base = a.slice_off[i >> 5] + (i & 31);
        const int len = a.row_len[i];
        const int *cp = a.col + base;
#pragma unroll UNROLL
        for (int k = 0; k < len; k++) {
            const int j = __ldg(cp + 32 * k);
            if (neighbour_ok(a, j, true)) pair(j, true);
        }
    }
}

// |X_j - X_i| for the kernel weight: r2 rsqrt(r2) in FP32 (one special-function op: the approximate
// reciprocal square root with subnormals flushed, which r2 of two distinct particles never is), sqrt in
// FP64.  r2 = 0 (a dropped entry reading the zero halo) gives NaN, which the pair bodies select away.
__device__ __forceinline__ float pair_dist(float r2) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
    return r2 * r;
}
__device__ __forceinline__ double pair_dist(double r2) { return sqrt(r2); }
// x / y of the viscosity and Laplacian terms: the approximate division (subnormals flushed) in FP32, IEEE
// division in FP64.
__device__ __forceinline__ float pair_div(float x, float y) {
    float q;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(q) : "f"(x), "f"(y));
    return q;
}
__device__ __forceinline__ double pair_div(double x, double y) { return x / y; }

// |X_j - X_i|^2 of a pair and the Wendland C2 factor t = max(1 - r / (2h), 0) (w = t^3).
template <typename T, int DIM> __device__ __forceinline__ T pair_r2(const T d[DIM]) {
    T r2 = d[0] * d[0];
    r2 = t_fma(d[1], d[1], r2);
    if (DIM == 3) r2 = t_fma(d[DIM - 1], d[DIM - 1], r2);
    return r2;
}
template <typename T> __device__ __forceinline__ T pair_t(T r2, T inv2h) {
    return t_max(t_fma(-pair_dist(r2), inv2h, T(1)), T(0));
}
// The same without the clamp at zero, for the step's pair bodies: a kept pair has r0 < R, and an
// entry the mask drops has its weight selected to zero after the cube, so the clamp adds nothing.
template <typename T> __device__ __forceinline__ T pair_t_kept(T r2, T inv2h) {
    return t_fma(-pair_dist(r2), inv2h, T(1));
}

// Prefetch the SELL-32 slice of row i to L2 (no index stream in the stencil layout).
template <typename T> __device__ __forceinline__ void prefetch_rows(const StepArgs<T> &a, int i) {
    if (a.nsten == 0) prefetch_slice(a.col, a.slice_off, i);
}

// ---------------------------------------------------------------- pass 1a: deformation gradient
// G_i = F_i - I = (sum_j V_j w_ij (u_j - u_i) (X_j - X_i)^T) Ahat_i, and in the same walk the two other
// sums over the neighbours of the state at the step's start, which share the pair's distance, weight
// and displacement difference:
//   the artificial viscosity (VISC): s3_i = sum_j m_j w g (beta2 h g - beta1 c0) (X_j - X_i), over the
//   pairs in relative compression, (v_j - v_i).(x_j - x_i) < 0 with x = X + u, where
//   g = (v_j - v_i).(X_j - X_i) / (r^2 + eps).  Times h / rho_i this is sum_j m_j pi_ij w (X_j - X_i)
//   (eq. artViscCoef), which the stress pass turns into the viscous acceleration J F^-T Ahat s3 h / rho_i;
//   the phase-field Laplacian (FRAC): lap_i = -2 Ahat_i : sum_j (s_i - s_j) V_j w d d^T / r^2
//   (eq. phasefieldLapLacian).
// Written as pieces (own state, neighbour record, pair term, closing product), which keeps the loop
// body's live state explicit.
template <typename T, int DIM> struct GradOwn {
    V4<T> xi, ui, vsi;
    bool frac;
    T cvis, b2h;  // beta1 c0 and beta2 h of the particle's material
    T B[DIM][DIM];
    T s3[DIM], Tl[DIM == 3 ? 6 : 3];
};
template <typename T> struct GradRec {
    V4<T> xj, uj, vsj;
};
template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void grad_begin(const StepArgs<T> &a, int i, GradOwn<T, DIM> &o) {
    o.xi = a.X0V[i];
    o.ui = a.ug_cur[i];
    o.vsi = V4<T>{T(0), T(0), T(0), T(1)};
    if (VISC || FRAC) o.vsi = a.vs_cur[i];
    o.frac = false;
    o.cvis = o.b2h = T(0);
    if (VISC || FRAC) {
        const MatT<T> &m = a.mats[a.mid[i]];
        o.frac = FRAC && m.fracture;
        o.cvis = m.beta1 * m.c0;
        o.b2h = m.beta2 * a.h;
    }
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        o.s3[p] = T(0);
#pragma unroll
        for (int q = 0; q < DIM; q++) o.B[p][q] = T(0);
    }
#pragma unroll
    for (int p = 0; p < (DIM == 3 ? 6 : 3); p++) o.Tl[p] = T(0);
}
template <typename T, bool FRAC, bool VISC> __device__ __forceinline__ GradRec<T> grad_load(const StepArgs<T> &a, int j) {
    GradRec<T> r;
    r.xj = ldg4(a.X0V + j);
    r.uj = ldg4(a.ug_cur + j);
    r.vsj = V4<T>{T(0), T(0), T(0), T(0)};
    if (VISC || FRAC) r.vsj = ldg4(a.vs_cur + j);
    return r;
}
template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void grad_pair(const StepArgs<T> &a, GradOwn<T, DIM> &o, const GradRec<T> &r, bool on) {
    T d[DIM], du[DIM];
    d[0] = r.xj.x - o.xi.x;
    d[1] = r.xj.y - o.xi.y;
    du[0] = r.uj.x - o.ui.x;
    du[1] = r.uj.y - o.ui.y;
    if (DIM == 3) {
        d[DIM - 1] = r.xj.z - o.xi.z;
        du[DIM - 1] = r.uj.z - o.ui.z;
    }
    const T r2 = pair_r2<T, DIM>(d);
    const T t = pair_t_kept(r2, a.inv2h);
    const T w = t * t * t;
    const T Vj = DIM == 3 ? r.xj.w : r.xj.z;
    const T aw = on ? w * Vj : T(0);
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        const T c = aw * du[p];
#pragma unroll
        for (int q = 0; q < DIM; q++) o.B[p][q] = t_fma(c, d[q], o.B[p][q]);
    }
    if (VISC) {
        const V4<T> &vsi = o.vsi, &vsj = r.vsj;
        const T mj = DIM == 3 ? r.uj.w : r.xj.w;  // reference mass m0_j
        T dv[DIM];
        dv[0] = vsj.x - vsi.x;
        dv[1] = vsj.y - vsi.y;
        if (DIM == 3) dv[DIM - 1] = vsj.z - vsi.z;
        // (v_j - v_i).(X_j - X_i), then + (v_j - v_i).(u_j - u_i) for the current separation
        T vX = dv[0] * d[0];
        vX = t_fma(dv[1], d[1], vX);
        if (DIM == 3) vX = t_fma(dv[DIM - 1], d[DIM - 1], vX);
        T vx = t_fma(dv[0], du[0], vX);
        vx = t_fma(dv[1], du[1], vx);
        if (DIM == 3) vx = t_fma(dv[DIM - 1], du[DIM - 1], vx);
        if (DIM == 3) {
            // computed for every pair and kept for pairs in relative compression (the others add exact
            // zeros), so the pair body has no branch (measured faster in 3D; the 2D pass keeps the branch)
            const T g = pair_div(vX, r2 + a.visc_eps);
            const T c = on && vx < T(0) ? mj * w * g * t_fma(o.b2h, g, -o.cvis) : T(0);
#pragma unroll
            for (int p = 0; p < DIM; p++) o.s3[p] = t_fma(c, d[p], o.s3[p]);
        } else if (on && vx < T(0)) {  // pair in relative compression
            const T g = pair_div(vX, r2 + a.visc_eps);
            const T c = mj * w * g * t_fma(o.b2h, g, -o.cvis);
#pragma unroll
            for (int p = 0; p < DIM; p++) o.s3[p] = t_fma(c, d[p], o.s3[p]);
        }
    }
    if (FRAC && o.frac) {
        T *Tl = o.Tl;
        const T c = on ? pair_div((o.vsi.w - r.vsj.w) * aw, r2) : T(0);  // fast division in FP32, as the viscosity
        const T c0 = c * d[0], c1 = c * d[1];
        Tl[0] = t_fma(c0, d[0], Tl[0]);
        Tl[1] = t_fma(c1, d[1], Tl[1]);
        if (DIM == 3) {
            Tl[2] = t_fma(c * d[2], d[2], Tl[2]);
            Tl[3] = t_fma(c0, d[1], Tl[3]);
            Tl[4] = t_fma(c0, d[2], Tl[4]);
            Tl[5] = t_fma(c1, d[2], Tl[5]);
        } else {
            Tl[2] = t_fma(c0, d[1], Tl[2]);
        }
    }
}
// G = B Ahat, and the closing of the other two sums: the viscosity sum as it is (s3), the Laplacian
// lap = -2 Ahat : Tl (0 without phase field).
template <typename T, int DIM, bool FRAC>
__device__ __forceinline__ void grad_finish(const StepArgs<T> &a, int i, const GradOwn<T, DIM> &o, T Gm[DIM][DIM],
                                            T &lap) {
    T A[3][3];
    load_ahat<T, DIM>(a.Ahat, a.n, i, A);
#pragma unroll
    for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) {
            T s = o.B[p][0] * A[0][q];
#pragma unroll
            for (int r = 1; r < DIM; r++) s = t_fma(o.B[p][r], A[r][q], s);
            Gm[p][q] = s;
        }
    lap = T(0);
    if (FRAC && o.frac) {
        const T *Tl = o.Tl;
        T AT;
        if (DIM == 3)
            AT = A[0][0] * Tl[0] + A[1][1] * Tl[1] + A[2][2] * Tl[2] +
                 T(2) * (A[0][1] * Tl[3] + A[0][2] * Tl[4] + A[1][2] * Tl[5]);
        else
            AT = A[0][0] * Tl[0] + A[1][1] * Tl[1] + T(2) * A[0][1] * Tl[2];
        lap = T(-2) * AT;
    }
}
// F - I to G; the viscosity sum to S3 and the Laplacian to LAP for the stress pass and pass 2.
template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void grad_store(const StepArgs<T> &a, int i, const GradOwn<T, DIM> &o, const T Gm[DIM][DIM],
                                           T lap) {
#pragma unroll
    for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) a.G[(p * DIM + q) * a.n + i] = Gm[p][q];
    if (VISC)
#pragma unroll
        for (int p = 0; p < DIM; p++) a.S3[p * a.n + i] = o.s3[p];
    if (FRAC) a.LAP[i] = lap;
}

template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void dev_gradient(const StepArgs<T> &a, int i, GradOwn<T, DIM> &o, T Gm[DIM][DIM], T &lap) {
    grad_begin<T, DIM, FRAC, VISC>(a, i, o);
    for_each_neighbour<4, false, false>(a, i, [&](const int j, const bool on) {
        grad_pair<T, DIM, FRAC, VISC>(a, o, grad_load<T, FRAC, VISC>(a, j), on);
    });
    grad_finish<T, DIM, FRAC>(a, i, o, Gm, lap);
}

template <typename T, int DIM, bool FRAC, bool VISC, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) k_gradient(StepArgs<T> a) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= a.n) return;
    prefetch_rows(a, i);
    GradOwn<T, DIM> o;
    T Gm[DIM][DIM], lap;
    dev_gradient<T, DIM, FRAC, VISC>(a, i, o, Gm, lap);
    grad_store<T, DIM, FRAC, VISC>(a, i, o, Gm, lap);
}

// First moment of the corrected kernel over the particle's volume, sum_j V_j w_ij (X_j - X_i) / V_i: it
// depends on the reference configuration only, so the setup computes it once for pass 2 (which holds
// Q_i V_i, so that Q_i sum_j V_j w d = (V_i Q_i) S1_i).
template <typename T, int DIM> __global__ void k_first_moment(StepArgs<T> a, V4<T> *S1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const V4<T> xi = a.X0V[i];
    T s1[3] = {T(0), T(0), T(0)};
    for_each_neighbour(a, i, [&](const int j, const bool on) {
        const V4<T> xj = ldg4(a.X0V + j);
        T d[DIM];
        d[0] = xj.x - xi.x;
        d[1] = xj.y - xi.y;
        if (DIM == 3) d[DIM - 1] = xj.z - xi.z;
        const T t = pair_t(pair_r2<T, DIM>(d), a.inv2h);
        const T w = on ? t * t * t : T(0);
        const T Vj = DIM == 3 ? xj.w : xj.z;
        const T aw = w * Vj;
#pragma unroll
        for (int p = 0; p < DIM; p++) s1[p] = t_fma(aw, d[p], s1[p]);
    });
    const T Vi = DIM == 3 ? xi.w : xi.z;
    S1[i] = V4<T>{s1[0] / Vi, s1[1] / Vi, s1[2] / Vi, T(0)};
}

// ---------------------------------------------------------------- pass 1b: stress
template <typename T, int DIM>
__device__ __forceinline__ void dev_write_qvm(const StepArgs<T> &a, int i, const M3<T> &F, const M3<T> &P, T J, T irho,
                                              const T *s3v);

// Soft particles (eq. defGrad_phase), NH / J2 stress, history functional, and what pass 2 takes of
// the particle: Q_i = P_i Ahat_i and the viscous acceleration.  s3v: the particle's viscosity sum when
// the caller holds it, else null (read from S3).
template <typename T, int DIM, bool FRAC, bool DIAG>
__device__ __forceinline__ void dev_stress(const StepArgs<T> &a, int i, const T Gm[DIM][DIM], const T *s3v = nullptr) {
    const int n = a.n;
    M3<T> G = m3_zero<T>();
#pragma unroll
    for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) G(p, q) = Gm[p][q];
    const MatT<T> m = a.mats[a.mid[i]];
    T s = T(1);
    const bool frac = FRAC && m.fracture;
    if (frac) {
        s = a.vs_cur[i].w;
        if (s <= m.s_lim) G = m3_zero<T>();
    }
    const Kin<T> kin = kinematics(G);
    M3<T> S;
    T psi = T(0);
    if (m.model == 3) {
        T K6[6], K6o[6], epo, dg;
#pragma unroll
        for (int q = 0; q < 6; q++) K6[q] = a.K[q * n + i];
        const T ep = a.ep[i];
        const int st = j2_update(kin, K6, ep, m, K6o, epo, S, dg);
        if (DIAG) {
            psi = j2_energy(kin, K6o, m);
        } else {
            if (dg > T(0)) {
#pragma unroll
                for (int q = 0; q < 6; q++) a.K[q * n + i] = K6o[q];
                a.ep[i] = epo;
            }
            if (st) atomicAdd(&a.flags[kFlagNoconv], 1);
        }
    } else {
        T pp, pm;
        if (m.model == 1) svk_stress<T, DIM>(kin, s, m, S, pp, pm);
        else nh_stress(kin, s, m, S, pp, pm);
        psi = s * s * pp + pm;
        if (!DIAG && frac && pp > a.H[i]) a.H[i] = pp;  // eq. irreversibility
    }
    // P = F S
    M3<T> F = G;
    F.a[0] += T(1);
    F.a[4] += T(1);
    F.a[8] += T(1);
    const M3<T> P = mul(F, S);
    if (DIAG) {
#pragma unroll
        for (int q = 0; q < 9; q++) {
            a.Fout[q * n + i] = F.a[q];
            a.Pout[q * n + i] = P.a[q];
        }
        a.psi_out[i] = psi;
        return;
    }
    dev_write_qvm<T, DIM>(a, i, F, P, T(1) + kin.Jm1, T(1) / m.rho, s3v);
}

// What pass 2 takes of particle i: V_i Q_i with Q_i = P_i Ahat_i (3D: q00 q01 q02 q10 | q11 q12 q20 q21 in
// Qa, Qb, and q22 in the fourth place of XQ = (x, y, z, q22) beside the particle's reference position, so
// that pass 2 gathers three float4 records per neighbour; 2D: Qa) and, in a step with viscosity (Av set),
// the viscous acceleration
// Av_i = Vm_i s3_i h / rho_i with Vm_i = J_i F_i^-T Ahat_i (in-plane block), the viscosity sum s3_i of
// pass 1a closed with the particle's own matrices.
template <typename T, int DIM>
__device__ __forceinline__ void dev_write_qvm_fi(const StepArgs<T> &a, int i, const M3<T> &Fi, const M3<T> &P, T J,
                                                 T irho, const T *s3v);
template <typename T, int DIM>
__device__ __forceinline__ void dev_write_qvm(const StepArgs<T> &a, int i, const M3<T> &F, const M3<T> &P, T J, T irho,
                                              const T *s3v) {
    M3<T> Fi;
    inverse(F, Fi);
    dev_write_qvm_fi<T, DIM>(a, i, Fi, P, J, irho, s3v);
}
// The same, given F^-1.
template <typename T, int DIM>
__device__ __forceinline__ void dev_write_qvm_fi(const StepArgs<T> &a, int i, const M3<T> &Fi, const M3<T> &P, T J,
                                                 T irho, const T *s3v) {
    const int n = a.n;
    T A[3][3];
    load_ahat<T, DIM>(a.Ahat, n, i, A);
    T Qm[DIM][DIM], Vm[DIM][DIM];
    bool ok = true;
#pragma unroll
    for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) {
            T s1 = T(0), s2 = T(0);
#pragma unroll
            for (int r = 0; r < DIM; r++) {
                s1 += P(p, r) * A[r][q];
                s2 += Fi(r, p) * A[r][q];
            }
            Qm[p][q] = s1;
            Vm[p][q] = J * s2;
            ok = ok && finite_t(s1) && finite_t(s2);
        }
    if (!ok) atomicAdd(&a.flags[kFlagNonfinite], 1);
    const V4<T> xi = a.X0V[i];
    const T Vi = DIM == 3 ? xi.w : xi.z;
    if (DIM == 3) {
        a.Qa[i] = V4<T>{Vi * Qm[0][0], Vi * Qm[0][1], Vi * Qm[0][DIM - 1], Vi * Qm[1][0]};
        a.Qb[i] = V4<T>{Vi * Qm[1][1], Vi * Qm[1][DIM - 1], Vi * Qm[DIM - 1][0], Vi * Qm[DIM - 1][1]};
        a.XQ[i] = V4<T>{xi.x, xi.y, xi.z, Vi * Qm[DIM - 1][DIM - 1]};
    } else {
        a.Qa[i] = V4<T>{Vi * Qm[0][0], Vi * Qm[0][1], Vi * Qm[1][0], Vi * Qm[1][1]};
    }
    if (a.Av) {
        T s3[DIM];
#pragma unroll
        for (int q = 0; q < DIM; q++) s3[q] = (s3v ? s3v[q] : a.S3[q * n + i]) * (a.h * irho);
#pragma unroll
        for (int p = 0; p < DIM; p++) {
            T v = T(0);
#pragma unroll
            for (int q = 0; q < DIM; q++) v = t_fma(Vm[p][q], s3[q], v);
            a.Av[p * n + i] = v;
        }
    }
}

// FP32: eight blocks of 128 threads per SM (64 registers; the J2 return map's rare plastic branch spills a
// little), measured 11% faster on the 1M-particle J2 block than the unbounded 91 registers
#ifndef TLSPH_STRESS_MINB
#define TLSPH_STRESS_MINB 8
#endif
template <typename T, int DIM, bool FRAC, bool DIAG, int BS>
__global__ void __launch_bounds__(BS, sizeof(T) == 4 ? TLSPH_STRESS_MINB * 128 / BS : 1) k_stress(StepArgs<T> a) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= a.n) return;
    T Gm[DIM][DIM];
#pragma unroll
    for (int p = 0; p < DIM; p++)
#pragma unroll
        for (int q = 0; q < DIM; q++) Gm[p][q] = a.G[(p * DIM + q) * a.n + i];
    dev_stress<T, DIM, FRAC, DIAG>(a, i, Gm);
}

// ---------------------------------------------------------------- pass 2
// Pass 2 in pieces: the particle's own state and sums, the neighbour record, the pair term and the
// closing update (the loop's live state is the own state; the compiler keeps fewer values across it
// than with one function body).
template <typename T, int DIM> struct P2Own {
    V4<T> xi;
    T s2[DIM];
};
// the neighbour's records: position (3D with q22 beside it), V Q with Q = P Ahat
template <typename T> struct P2Rec {
    V4<T> xj, q0, q1;
};
template <typename T, int DIM>
__device__ __forceinline__ void p2_begin(const StepArgs<T> &a, int i, P2Own<T, DIM> &o) {
    o.xi = a.X0V[i];
#pragma unroll
    for (int p = 0; p < DIM; p++) o.s2[p] = T(0);
}
template <typename T, int DIM> __device__ __forceinline__ P2Rec<T> p2_load(const StepArgs<T> &a, int j) {
    P2Rec<T> r;
    r.xj = ldg4((DIM == 3 ? a.XQ : a.X0V) + j);
    r.q0 = ldg4(a.Qa + j);
    if (DIM == 3) r.q1 = ldg4(a.Qb + j);
    return r;
}
// One pair of pass 2: s2 += w (V_j Q_j) (X_j - X_i).
template <typename T, int DIM>
__device__ __forceinline__ void p2_pair(const StepArgs<T> &a, P2Own<T, DIM> &o, const P2Rec<T> &r, bool on) {
    const V4<T> &xi = o.xi, &xj = r.xj;
    T d[DIM];
    d[0] = xj.x - xi.x;
    d[1] = xj.y - xi.y;
    if (DIM == 3) d[DIM - 1] = xj.z - xi.z;
    const T t = pair_t_kept(pair_r2<T, DIM>(d), a.inv2h);
    const T aw = on ? t * t * t : T(0);
    T Qd[DIM];
    if (DIM == 3) {
        const V4<T> &q0 = r.q0, &q1 = r.q1;
        const T q2 = xj.w;
        Qd[0] = t_fma(q0.z, d[DIM - 1], t_fma(q0.y, d[1], q0.x * d[0]));
        Qd[1] = t_fma(q1.y, d[DIM - 1], t_fma(q1.x, d[1], q0.w * d[0]));
        Qd[DIM - 1] = t_fma(q2, d[DIM - 1], t_fma(q1.w, d[1], q1.z * d[0]));
    } else {
        const V4<T> &q0 = r.q0;
        Qd[0] = t_fma(q0.y, d[1], q0.x * d[0]);
        Qd[1] = t_fma(q0.w, d[1], q0.z * d[0]);
    }
#pragma unroll
    for (int p = 0; p < DIM; p++) o.s2[p] = t_fma(aw, Qd[p], o.s2[p]);
}
template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void p2_finish(const StepArgs<T> &a, int i, const P2Own<T, DIM> &o, T &vmag, T &amag) {
    const int n = a.n;
    const int sp = a.spec[i];
    const V4<T> &xi = o.xi;
    const V4<T> vsi = a.vs_cur[i];
    const MatT<T> m = a.mats[a.mid[i]];
    const bool frac = FRAC && m.fracture;
    const T irho = T(1) / m.rho;
    const T *s2 = o.s2;
    T s1[DIM];
    {
        const V4<T> m1 = a.S1[i];  // sum_j V_j w d / V_i, fixed in the reference configuration
        s1[0] = m1.x;
        s1[1] = m1.y;
        if (DIM == 3) s1[DIM - 1] = m1.z;
    }
    // own matrices
    T Qi[DIM][DIM];
    if (DIM == 3) {
        const V4<T> q0 = a.Qa[i], q1 = a.Qb[i];
        Qi[0][0] = q0.x; Qi[0][1] = q0.y; Qi[0][DIM - 1] = q0.z;
        Qi[1][0] = q0.w; Qi[1][1] = q1.x; Qi[1][DIM - 1] = q1.y;
        Qi[DIM - 1][0] = q1.z; Qi[DIM - 1][1] = q1.w; Qi[DIM - 1][DIM - 1] = a.XQ[i].w;
    } else {
        const V4<T> q0 = a.Qa[i];
        Qi[0][0] = q0.x; Qi[0][1] = q0.y; Qi[1][0] = q0.z; Qi[1][1] = q0.w;
    }
    T acc[3] = {T(0), T(0), T(0)};
    T acc_in[3] = {T(0), T(0), T(0)};  // the acceleration of the interactions (stress, viscosity, contact)
    double aext[3] = {0.0, 0.0, 0.0};  // and of the external forces (gravity, force conditions)
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        T f = s2[p];
#pragma unroll
        for (int q = 0; q < DIM; q++) f = t_fma(Qi[p][q], s1[q], f);
        acc[p] = f * irho;
        if (VISC) acc[p] -= a.Av[p * n + i];  // viscous acceleration of the stress pass
        acc_in[p] = acc[p] + (a.accc ? a.accc[p * n + i] : T(0));
        acc[p] += a.grav[p];
        aext[p] = (double)a.grav[p];
        if (a.accc) acc[p] += a.accc[p * n + i];
    }
    // forces act at t_n (Algorithm 1) or t_{n+1/2} (Algorithm 2); velocity BCs hold at t_{n+1}
    const double dt = a.dt[sp], t_1 = a.t[sp] + dt, t_n = a.t[sp] + (a.leap ? 0.5 * dt : 0.0);
    const int g = a.bcgrp[i];
    const T mass = DIM == 3 ? m.rho * xi.w : xi.w;
    double vset[3];
    int vmask = 0;
    if (g) {
        for (int b = 0; b < kMaxBcPerParticle; b++) {
            const int id = a.grp_bcs[4 * g + b];
            if (id < 0) break;
            const BCDev bc = a.bcs[id];
            if (bc.kind == 4) continue;  // phase-field bound: applied with the update of s below
            if (bc.kind == 0) {  // velocity: value at t_{n+1}
                const double f = bc_factor(bc, t_1);
                if (f < 0.0) continue;
                for (int p = 0; p < DIM; p++) {
                    double val;
                    if ((bc.comp_mask & (1 << p)) && dev_bc_value(a, bc, i, b, 0, p, f, val)) {
                        vset[p] = val;
                        vmask |= 1 << p;
                    }
                }
            } else {  // forces at t_n
                const double f = bc_factor(bc, t_n);
                if (f < 0.0) continue;
                for (int p = 0; p < DIM; p++) {
                    double val;
                    if (!(bc.comp_mask & (1 << p)) || !dev_bc_value(a, bc, i, b, 0, p, f, val)) continue;
                    const double ae = bc.kind == 1 ? val * bc.area / (double)mass
                                                   : (bc.kind == 2 ? val : val * bc.inv_count / (double)mass);
                    acc[p] += (T)ae;
                    aext[p] += ae;
                }
            }
        }
    }
    // phase field (eq. phasefieldddot)
    T s_new = FRAC ? vsi.w : T(1);
    if (frac) {
        const T lap = a.LAP[i];  // Laplacian of pass 1a
        const T Hh = a.H[i], si = vsi.w, sd = a.sdot[i];
        const T e0 = m.eps0, c2e = m.c0 * m.c0 / (T(2) * e0);
        // eq. phasefieldddot with its local terms at the new time level:
        // sdot_{n+1} = (sdot_n + dt r_n) / (1 + dt gamma + dt^2 k)
        const T r = c2e * (T(2) * e0 * lap + (T(1) - si) / (T(2) * e0) - T(2) * si * Hh / m.Gc);
        const T kk = c2e * (T(1) / (T(2) * e0) + T(2) * Hh / m.Gc);
        const T gam = m.c0 / e0 * t_sqrt(T(4) * e0 * Hh / m.Gc + T(1));
        const T dts = (T)dt;
        const T sd_new = (sd + dts * r) / (T(1) + dts * gam + dts * dts * kk);
        a.sdot[i] = sd_new;
        // s_{n+1} = s_n + dt sdot_{n+1} (Algorithm 1), s_{n+1/2} + dt/2 sdot_{n+1} (Algorithm 2)
        s_new = t_min(T(1), t_max(T(0), si + (T)(a.leap ? 0.5 * dt : dt) * sd_new));
        // <restrictphi> (Sec. 3.3): a phase-field bound covering the particle keeps s_{n+1} >= its value at t_{n+1}
        for (int b = 0; g && b < kMaxBcPerParticle; b++) {
            const int id = a.grp_bcs[4 * g + b];
            if (id < 0) break;
            const BCDev bc = a.bcs[id];
            if (bc.kind != 4 || !(bc.comp_mask & 1)) continue;
            const double f = bc_factor(bc, t_1);
            double val;
            // an expression's value is kept in [0, 1]
            if (f >= 0.0 && dev_bc_value(a, bc, i, b, 0, 0, f, val)) s_new = t_max(s_new, (T)fmin(fmax(val, 0.0), 1.0));
        }
    }
    // update: v_{n+1} = v_n + dt a; u_{n+1} = u_n + dt v_{n+1} (Algorithm 1) or
    // u_{n+1/2} + dt/2 v_{n+1} (Algorithm 2, u64 holding u_{n+1/2})
    const V4<T> vo = a.leap ? a.v_own[i] : vsi;
    T vn[3] = {vo.x, vo.y, vo.z};
    const T vo_c[3] = {vo.x, vo.y, vo.z};
    const T dtT = (T)dt;
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        vn[p] = vn[p] + dtT * acc[p];
        if (vmask & (1 << p)) vn[p] = (T)vset[p];
    }
    double un[3];
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        un[p] = a.u64[p * n + i] + (a.leap ? 0.5 * dt : dt) * (double)vn[p];
        a.u64[p * n + i] = un[p];
    }
    // work of the external forces along the step's displacement increment u_{n+1} - u_n (Algorithm 1:
    // dt v_{n+1}; Algorithm 2: dt (v_n + v_{n+1}) / 2): gravity and force conditions, and on a component a
    // velocity condition holds the reaction m (v_{n+1} - v_n) / dt - m a_interactions
    if (g || a.grav[0] != T(0) || a.grav[1] != T(0) || a.grav[2] != T(0)) {
        double wk = 0.0;
#pragma unroll
        for (int p = 0; p < DIM; p++) {
            const double fe = (vmask & (1 << p)) ? (double)mass * (((double)vn[p] - (double)vo_c[p]) / dt - (double)acc_in[p])
                                                 : (double)mass * aext[p];
            const double du = a.leap ? 0.5 * dt * ((double)vo_c[p] + (double)vn[p]) : dt * (double)vn[p];
            wk += fe * du;
        }
        a.wext[i] += wk;
    }
    a.ug_next[i] = V4<T>{(T)un[0], (T)un[1], DIM == 3 ? (T)un[DIM - 1] : T(0), DIM == 3 ? mass : T(0)};
    a.vs_next[i] = V4<T>{vn[0], vn[1], DIM == 3 ? vn[DIM - 1] : T(0), s_new};
    if (a.acc_out)
#pragma unroll
        for (int p = 0; p < DIM; p++) a.acc_out[p * n + i] = acc[p];
    T vv = T(0), aa = T(0);
#pragma unroll
    for (int p = 0; p < DIM; p++) {
        vv += vn[p] * vn[p];
        aa += acc[p] * acc[p];
    }
    vmag = t_sqrt(vv);
    amag = t_sqrt(aa);
    if (!(finite_t(vmag) && finite_t(amag))) atomicAdd(&a.flags[kFlagNonfinite], 1);
}

template <typename T, int DIM, bool FRAC, bool VISC>
__device__ __forceinline__ void dev_pass2(const StepArgs<T> &a, int i, T &vmag, T &amag) {
    P2Own<T, DIM> o;
    p2_begin<T, DIM>(a, i, o);
    // entry by entry, four (3D) or two (2D) at a time across runs: measured faster than the unrolled runs
    // and than other depths (crack-branching plate: 0.139 ms at two, 0.145 at four, 0.148 at eight)
    for_each_neighbour<DIM == 3 ? 4 : 2, false, false>(a, i, [&](const int j, const bool on) {
        p2_pair<T, DIM>(a, o, p2_load<T, DIM>(a, j), on);
    });
    p2_finish<T, DIM, FRAC, VISC>(a, i, o, vmag, amag);
}

// Velocity boundary conditions of particle i at time t: the constrained components of v take the
// prescribed values (expression values of the given phase).
template <typename T, int DIM>
__device__ __forceinline__ void dev_velocity_bcs(const StepArgs<T> &a, int i, double t, T v[3], int phase) {
    const int g = a.bcgrp[i];
    if (!g) return;
    for (int b = 0; b < kMaxBcPerParticle; b++) {
        const int id = a.grp_bcs[4 * g + b];
        if (id < 0) break;
        const BCDev bc = a.bcs[id];
        if (bc.kind != 0) continue;
        const double f = bc_factor(bc, t);
        if (f < 0.0) continue;
        for (int p = 0; p < DIM; p++) {
            double val;
            if ((bc.comp_mask & (1 << p)) && dev_bc_value(a, bc, i, b, phase, p, f, val)) v[p] = (T)val;
        }
    }
}

// Algorithm 2, predictor: u_{n+1/2} = u_n + dt/2 v_n (FP64 accumulator and its FP32 copy),
// v_{n+1/2} = v_n + dt/2 a_{n-1/2} with the velocity BCs at t_{n+1/2}, s_{n+1/2} = s_n + dt/2 sdot_n
// (kept in [0, 1]).  The half level goes to ug_half / vs_half, which the step's other kernels read.
template <typename T, int DIM, bool FRAC, int BS>
__global__ void __launch_bounds__(BS) k_predict(StepArgs<T> a) {
    const int i = blockIdx.x * BS + threadIdx.x;
    if (i >= a.n) return;
    const int n = a.n;
    const int sp = a.spec[i];
    const double dt = a.dt[sp], th = a.t[sp] + 0.5 * dt;
    const V4<T> v = a.v_own[i];
    const T vv[3] = {v.x, v.y, v.z};
    T uf[3] = {T(0), T(0), T(0)}, vh[3] = {v.x, v.y, v.z};
    for (int p = 0; p < DIM; p++) {
        const double uh = a.u64[p * n + i] + 0.5 * dt * (double)vv[p];
        a.u64[p * n + i] = uh;
        uf[p] = (T)uh;
        vh[p] = vv[p] + (T)(0.5 * dt) * a.acc_out[p * n + i];
    }
    dev_velocity_bcs<T, DIM>(a, i, th, vh, 1);
    T sh = v.w;
    if (FRAC && a.mats[a.mid[i]].fracture) {
        sh = t_min(T(1), t_max(T(0), v.w + (T)(0.5 * dt) * a.sdot[i]));
        // <restrictphi>: a phase-field bound holds at the half level too, with its value at t_{n+1/2}
        const int g = a.bcgrp[i];
        for (int b = 0; g && b < kMaxBcPerParticle; b++) {
            const int id = a.grp_bcs[4 * g + b];
            if (id < 0) break;
            const BCDev bc = a.bcs[id];
            if (bc.kind != 4 || !(bc.comp_mask & 1)) continue;
            const double f = bc_factor(bc, th);
            double val;
            if (f >= 0.0 && dev_bc_value(a, bc, i, b, 1, 0, f, val)) sh = t_max(sh, (T)fmin(fmax(val, 0.0), 1.0));
        }
    }
    a.ug_half[i] = V4<T>{uf[0], uf[1], DIM == 3 ? uf[DIM - 1] : T(0), DIM == 3 ? a.ug_next[i].w : T(0)};
    a.vs_half[i] = V4<T>{vh[0], vh[1], DIM == 3 ? vh[DIM - 1] : T(0), sh};
}

// Per-specimen maxima of |v_{n+1}| and |a_n| of one block (one atomic per block when the
// block holds a single specimen).
template <typename T, int BS>
__device__ __forceinline__ void dev_block_maxima(const StepArgs<T> &a, bool active, int sp, T vmag, T amag) {
    __shared__ int s_sp;
    __shared__ double s_v[BS / 32], s_a[BS / 32];
    if (threadIdx.x == 0) s_sp = sp;
    __syncthreads();
    const bool uniform = __syncthreads_and(!active || sp == s_sp);
    if (uniform) {
        double v, ac;
        if constexpr (sizeof(T) == 4) {
            // non-negative floats order like their bit patterns; one integer reduction per warp each (a NaN
            // counts as 0, as fmax drops it).  The maxima equal those of the same values in double.
            const unsigned vb = __reduce_max_sync(0xffffffffu, isnan(vmag) ? 0u : __float_as_uint((float)vmag));
            const unsigned ab = __reduce_max_sync(0xffffffffu, isnan(amag) ? 0u : __float_as_uint((float)amag));
            v = (double)__uint_as_float(vb);
            ac = (double)__uint_as_float(ab);
        } else {
            v = (double)vmag;
            ac = (double)amag;
            for (int o = 16; o > 0; o >>= 1) {
                v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
                ac = fmax(ac, __shfl_xor_sync(0xffffffffu, ac, o));
            }
        }
        if ((threadIdx.x & 31) == 0) {
            s_v[threadIdx.x >> 5] = v;
            s_a[threadIdx.x >> 5] = ac;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < BS / 32; q++) {
                v = fmax(v, s_v[q]);
                ac = fmax(ac, s_a[q]);
            }
            atomicMax(&a.vmax_bits[s_sp], (unsigned long long)__double_as_longlong(v));
            atomicMax(&a.amax_bits[s_sp], (unsigned long long)__double_as_longlong(ac));
        }
    } else if (active) {
        atomicMax(&a.vmax_bits[sp], (unsigned long long)__double_as_longlong((double)vmag));
        atomicMax(&a.amax_bits[sp], (unsigned long long)__double_as_longlong((double)amag));
    }
    __syncthreads();
}

// Advance every specimen's clock by its step and pick the next step size (eq. dt_criterion),
// after all of the step's maxima are in; run by the threads of one block.
template <typename T> __device__ __forceinline__ void dev_finalize(const StepArgs<T> &a) {
    {
        for (int q = threadIdx.x; q < a.nspec; q += blockDim.x) {
            const double dts = a.dt[q];
            a.t[q] = a.t[q] + dts;
            const double vm = __longlong_as_double((long long)atomicExch(&a.vmax_bits[q], 0ull));
            const double am = __longlong_as_double((long long)atomicExch(&a.amax_bits[q], 0ull));
            a.last_vmax[q] = vm;
            a.last_amax[q] = am;
            if (a.dt_mode == 1) {
                const double dtv = a.hd / (a.cmax[q] + vm);
                const double dta = am > 0.0 ? sqrt(a.hd / am) : INFINITY;
                a.dt[q] = a.cfl * (dtv < dta ? dtv : dta);
            }
        }
    }
}

template <typename T, int DIM, bool FRAC, bool VISC, int BS>
__global__ void __launch_bounds__(BS, 896 / BS) k_pass2(StepArgs<T> a) {
    __shared__ bool s_last;
    const int i = blockIdx.x * BS + threadIdx.x;
    const bool active = i < a.n;
    T vmag = T(0), amag = T(0);
    int sp = 0;
    if (active) {
        prefetch_rows(a, i);
        sp = a.spec[i];
        dev_pass2<T, DIM, FRAC, VISC>(a, i, vmag, amag);
    }
    dev_block_maxima<T, BS>(a, active, sp, vmag, amag);
    // the last block to finish advances the clocks and picks the next step size
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        dev_finalize(a);
        if (threadIdx.x == 0) *a.done = 0u;
    }
}

// ---------------------------------------------------------------- lattice kernels (3D, FP32)
// The two neighbour passes walking the ball of lattice.cuh instead of a difference table: the same
// pair bodies (grad_pair, p2_pair) in the same order per row, P rows per thread.  Debug builds check
// every record index against the zero halo and every kept entry against the particle range.
template <typename T> __device__ __forceinline__ bool lat_index_ok(const StepArgs<T> &a, int j) {
#ifdef TLSPH_DEBUG
    const bool ok = j >= -a.halo && j < a.n + a.halo;
    if (!ok) atomicAdd(&a.flags[kFlagBounds], 1);
    return ok;
#else
    (void)a;
    (void)j;
    return true;
#endif
}
// Blocks per SM the lattice kernels are compiled for (register budget): pass 1 with one or two rows per
// thread (two rows: in paired FP32 without phase field), pass 2 with one, two or four.
#ifndef TLSPH_LAT_GRAD_MINB
#define TLSPH_LAT_GRAD_MINB 6
#endif
#ifndef TLSPH_LAT_GRAD_PK_MINB  // pass 1 with two rows in paired FP32 (96 registers)
#define TLSPH_LAT_GRAD_PK_MINB 5
#endif
#ifndef TLSPH_LAT_P2_MINB
#define TLSPH_LAT_P2_MINB 6
#endif
#ifndef TLSPH_LAT_P4_MINB
#define TLSPH_LAT_P4_MINB 5
#endif
template <typename T, bool FRAC, bool VISC, int P> struct GradLatWalk {
    const StepArgs<T> &a;
    int NX, NXNY;
    GradOwn<T, 3> o[P];
    __device__ __forceinline__ GradRec<T> load(int j) const {
        if (!lat_index_ok(a, j)) j = a.n;  // debug builds: read a zero record instead
        return grad_load<T, FRAC, VISC>(a, j);
    }
    __device__ __forceinline__ void pair(int p, const GradRec<T> &r, int j, bool on) {
        if (neighbour_ok(a, j, on)) grad_pair<T, 3, FRAC, VISC>(a, o[p], r, on);
    }
};
// Pass 1 for two rows in paired FP32 (fma.rn.f32x2 and its add and multiply, one instruction for the
// same operation of both rows): lane 0 is row i0, lane 1 row i0 + NX.  Each lane repeats grad_pair's
// operations in its order and rounding (a - b as a + (-b), fma(-r, 1/2h, 1) as fma(r, -1/2h, 1), both
// exact rewritings), so the two rows get the bit patterns the scalar body gives them.  Without phase
// field only.
__device__ __forceinline__ float2 f2_bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <bool VISC> struct GradOwnPk {
    float2 nx[3], nu[3], nv[3];  // -X_i, -u_i, -v_i of the two rows
    float2 b2h, ncvis;           // beta2 h and -beta1 c0 of the rows' materials
    float2 B[3][3], s3[3];
};
template <bool VISC> struct GradLatWalkPk {
    const StepArgs<float> &a;
    int NX, NXNY;
    GradOwnPk<VISC> o;
    __device__ __forceinline__ GradRec<float> load(int j) const {
        if (!lat_index_ok(a, j)) j = a.n;
        return grad_load<float, false, VISC>(a, j);
    }
    __device__ __forceinline__ void pair2(const GradRec<float> &r, int j, bool on0, bool on1) {
        if (!neighbour_ok(a, j, on0 || on1)) return;
        float2 d[3], du[3];
        d[0] = f2_add(f2_bc(r.xj.x), o.nx[0]);
        d[1] = f2_add(f2_bc(r.xj.y), o.nx[1]);
        du[0] = f2_add(f2_bc(r.uj.x), o.nu[0]);
        du[1] = f2_add(f2_bc(r.uj.y), o.nu[1]);
        d[2] = f2_add(f2_bc(r.xj.z), o.nx[2]);
        du[2] = f2_add(f2_bc(r.uj.z), o.nu[2]);
        float2 r2 = f2_mul(d[0], d[0]);
        r2 = f2_fma(d[1], d[1], r2);
        r2 = f2_fma(d[2], d[2], r2);
        float2 rs;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.x) : "f"(r2.x));
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.y) : "f"(r2.y));
        const float2 t = f2_fma(f2_mul(r2, rs), f2_bc(-a.inv2h), f2_bc(1.0f));
        const float2 w = f2_mul(f2_mul(t, t), t);
        float2 aw = f2_mul(w, f2_bc(r.xj.w));
        aw.x = on0 ? aw.x : 0.0f;
        aw.y = on1 ? aw.y : 0.0f;
#pragma unroll
        for (int p = 0; p < 3; p++) {
            const float2 c = f2_mul(aw, du[p]);
#pragma unroll
            for (int q = 0; q < 3; q++) o.B[p][q] = f2_fma(c, d[q], o.B[p][q]);
        }
        if (VISC) {
            float2 dv[3];
            dv[0] = f2_add(f2_bc(r.vsj.x), o.nv[0]);
            dv[1] = f2_add(f2_bc(r.vsj.y), o.nv[1]);
            dv[2] = f2_add(f2_bc(r.vsj.z), o.nv[2]);
            float2 vX = f2_mul(dv[0], d[0]);
            vX = f2_fma(dv[1], d[1], vX);
            vX = f2_fma(dv[2], d[2], vX);
            float2 vx = f2_fma(dv[0], du[0], vX);
            vx = f2_fma(dv[1], du[1], vx);
            vx = f2_fma(dv[2], du[2], vx);
            const float2 den = f2_add(r2, f2_bc(a.visc_eps));
            float2 g;
            asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(g.x) : "f"(vX.x), "f"(den.x));
            asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(g.y) : "f"(vX.y), "f"(den.y));
            float2 c = f2_mul(f2_mul(f2_mul(f2_bc(r.uj.w), w), g), f2_fma(o.b2h, g, o.ncvis));
            c.x = on0 && vx.x < 0.0f ? c.x : 0.0f;
            c.y = on1 && vx.y < 0.0f ? c.y : 0.0f;
#pragma unroll
            for (int p = 0; p < 3; p++) o.s3[p] = f2_fma(c, d[p], o.s3[p]);
        }
    }
};
// Rows i0 and i0 + NX (active flags act) of the paired pass 1: set up, walk, and the rows' F - I and sums
// to memory as k_gradient_lat stores them.
template <bool VISC>
__device__ __forceinline__ void grad_lat_pk(const StepArgs<float> &a, int i0, const bool act[2]) {
    const int NX = a.lat_nx;
    GradLatWalkPk<VISC> w{a, NX, a.lat_nxny};
    GradOwn<float, 3> so[2];
#pragma unroll
    for (int p = 0; p < 2; p++) grad_begin<float, 3, false, VISC>(a, act[p] ? i0 + p * NX : i0, so[p]);
    w.o.nx[0] = make_float2(-so[0].xi.x, -so[1].xi.x);
    w.o.nx[1] = make_float2(-so[0].xi.y, -so[1].xi.y);
    w.o.nx[2] = make_float2(-so[0].xi.z, -so[1].xi.z);
    w.o.nu[0] = make_float2(-so[0].ui.x, -so[1].ui.x);
    w.o.nu[1] = make_float2(-so[0].ui.y, -so[1].ui.y);
    w.o.nu[2] = make_float2(-so[0].ui.z, -so[1].ui.z);
    w.o.nv[0] = make_float2(-so[0].vsi.x, -so[1].vsi.x);
    w.o.nv[1] = make_float2(-so[0].vsi.y, -so[1].vsi.y);
    w.o.nv[2] = make_float2(-so[0].vsi.z, -so[1].vsi.z);
    w.o.b2h = make_float2(so[0].b2h, so[1].b2h);
    w.o.ncvis = make_float2(-so[0].cvis, -so[1].cvis);
#pragma unroll
    for (int p = 0; p < 3; p++) {
        w.o.s3[p] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 3; q++) w.o.B[p][q] = make_float2(0.0f, 0.0f);
    }
    lat_walk_pk(w, a.lmask, a.n, i0, act);
#pragma unroll
    for (int p = 0; p < 3; p++) {
        so[0].s3[p] = w.o.s3[p].x;
        so[1].s3[p] = w.o.s3[p].y;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            so[0].B[p][q] = w.o.B[p][q].x;
            so[1].B[p][q] = w.o.B[p][q].y;
        }
    }
#pragma unroll
    for (int p = 0; p < 2; p++) {
        if (!act[p]) continue;
        const int i = i0 + p * NX;
        float Gm[3][3], lap;
        grad_finish<float, 3, false>(a, i, so[p], Gm, lap);
        grad_store<float, 3, false, VISC>(a, i, so[p], Gm, lap);
    }
}

// Pass 1 on the lattice: F - I and the viscosity and Laplacian sums of P rows per thread, then (FUSE)
// their stress and what pass 2 takes of them in the same thread, or (!FUSE) F - I and the sums to
// memory for a separate stress pass.
template <typename T, bool FRAC, bool VISC, bool FUSE, int P, int BS>
__global__ void __launch_bounds__(BS, FUSE ? 5 : (P == 1 ? 8 : (FRAC ? TLSPH_LAT_GRAD_MINB : TLSPH_LAT_GRAD_PK_MINB)))
    k_gradient_lat(StepArgs<T> a) {
    const int NX = a.lat_nx;
    bool owns;
    const int i0 = lat_block_row<P, BS>(blockIdx.x, threadIdx.x, NX, a.lat_cw, owns);
    if (!owns || i0 >= a.n) return;
    if constexpr (P == 2 && !FRAC && !FUSE && sizeof(T) == 4) {  // two rows in paired FP32
        const bool act2[2] = {true, i0 + NX < a.n};
        grad_lat_pk<VISC>(a, i0, act2);
        return;
    }
    GradLatWalk<T, FRAC, VISC, P> w{a, NX, a.lat_nxny};
    bool act[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        act[p] = i0 + p * NX < a.n;
        grad_begin<T, 3, FRAC, VISC>(a, act[p] ? i0 + p * NX : i0, w.o[p]);
    }
    lat_walk<P>(w, a.lmask, a.n, i0, act);
#pragma unroll
    for (int p = 0; p < P; p++) {
        if (!act[p]) continue;
        const int i = i0 + p * NX;
        T Gm[3][3], lap;
        grad_finish<T, 3, FRAC>(a, i, w.o[p], Gm, lap);
        if (FUSE) {
            if (FRAC) a.LAP[i] = lap;
            dev_stress<T, 3, FRAC, false>(a, i, Gm, w.o[p].s3);
        } else {
            grad_store<T, 3, FRAC, VISC>(a, i, w.o[p], Gm, lap);
        }
    }
}

template <typename T, int P> struct P2LatWalk {
    const StepArgs<T> &a;
    int NX, NXNY;
    P2Own<T, 3> o[P];
    __device__ __forceinline__ P2Rec<T> load(int j) const {
        if (!lat_index_ok(a, j)) j = a.n;
        return p2_load<T, 3>(a, j);
    }
    __device__ __forceinline__ void pair(int p, const P2Rec<T> &r, int j, bool on) {
        if (neighbour_ok(a, j, on)) p2_pair<T, 3>(a, o[p], r, on);
    }
};
// Pass 2 on the lattice: forces, damage, conditions and the update of P rows per thread; the last block
// advances the clocks (as k_pass2).
template <typename T, bool FRAC, bool VISC, int P, int BS>
__global__ void __launch_bounds__(BS, P == 1 ? 8 : (P == 2 ? TLSPH_LAT_P2_MINB : TLSPH_LAT_P4_MINB)) k_pass2_lat(StepArgs<T> a) {
    __shared__ bool s_last;
    const int NX = a.lat_nx;
    bool owns;
    const int i0 = lat_block_row<P, BS>(blockIdx.x, threadIdx.x, NX, a.lat_cw, owns);
    bool act[P];
    T vmag[P], amag[P];
    int sp[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        act[p] = owns && i0 + p * NX < a.n;
        vmag[p] = amag[p] = T(0);
        sp[p] = 0;
    }
    if (act[0]) {
        P2LatWalk<T, P> w{a, NX, a.lat_nxny};
#pragma unroll
        for (int p = 0; p < P; p++) p2_begin<T, 3>(a, act[p] ? i0 + p * NX : i0, w.o[p]);
        lat_walk<P>(w, a.lmask, a.n, i0, act);
#pragma unroll
        for (int p = 0; p < P; p++) {
            if (!act[p]) continue;
            const int i = i0 + p * NX;
            sp[p] = a.spec[i];
            p2_finish<T, 3, FRAC, VISC>(a, i, w.o[p], vmag[p], amag[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; p++) dev_block_maxima<T, BS>(a, act[p], sp[p], vmag[p], amag[p]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        dev_finalize(a);
        if (threadIdx.x == 0) *a.done = 0u;
    }
}

// ---------------------------------------------------------------- force pass streaming along z
// Pass 2 on the lattice with a column of planes per thread: thread (q, c) takes the rows
// i = z NXNY + c of planes z = q zc .. q zc + zc - 1 (c < NXNY: the place in a plane).  It walks the
// planes zp = q zc - 3 .. q zc + zc + 2 once and keeps the sums of the seven rows that plane zp serves,
// z = zp + 3 - k in slot k (entry dz = k - 3 of the ball), in registers.  A neighbour record
// zp NXNY + c + dy NX + dx is loaded once and added to every slot whose ball holds (dx, dy, dz): 29
// records per plane for 122 pairs, against one record per pair for one row per thread.  After plane zp
// the row of slot 6 has all its entries; its sum is parked in G and the slots move up by one.  The rows
// are updated (p2_finish) after the walk.
//
// Each row still receives its entries in ascending difference (planes ascending, then rows dy and dx
// ascending within a plane), so the step is bit-identical to the other walks.
template <typename T> struct ZsState {
    P2Own<T, 3> o[7];
    unsigned am;  // bit k: slot k holds a row of this thread's planes
};
template <int AY, int DX, int DZ, typename T>
__device__ __forceinline__ void zs_dz(const StepArgs<T> &a, ZsState<T> &s, const P2Rec<T> &r, int j, const unsigned (&lm)[7]) {
    constexpr int M = lat_ext(DX, AY);
    if constexpr (DZ <= M) {
        if constexpr (!(DX == 0 && AY == 0 && DZ == 0)) {
            constexpr int k = DZ + 3;
            if (s.am & (1u << k)) {
                const bool on = ((lm[k] >> (DX + lat_ext(AY, DZ))) & 1u) != 0u;
                if (neighbour_ok(a, j, on)) p2_pair<T, 3>(a, s.o[k], r, on);
            }
        }
        zs_dz<AY, DX, DZ + 1>(a, s, r, j, lm);
    }
}
template <int AY, int DX, typename T>
__device__ __forceinline__ void zs_dx(const StepArgs<T> &a, ZsState<T> &s, int rb, const unsigned (&lm)[7]) {
    constexpr int E = lat_ext(AY, 0);
    if constexpr (DX <= E) {
        int j = rb + DX;
        if (!lat_index_ok(a, j)) j = a.n;
        const P2Rec<T> r = p2_load<T, 3>(a, j);
        zs_dz<AY, DX, -lat_ext(DX, AY)>(a, s, r, rb + DX, lm);
        zs_dx<AY, DX + 1>(a, s, rb, lm);
    }
}
// Row dy = +-AY of plane zp.  lm[k] holds slot k's layer word moved so that bit 0 is the first entry of
// this row; it moves on past the row for the next one.
template <int AY, typename T>
__device__ __forceinline__ void zs_row(const StepArgs<T> &a, ZsState<T> &s, int rb, int dy, unsigned (&lm)[7]) {
    zs_dx<AY, -lat_ext(AY, 0)>(a, s, rb, lm);
#pragma unroll
    for (int k = 0; k < 7; k++) lm[k] >>= c_lat_rows.width[k][dy + 3];
}
#ifndef TLSPH_ZS_MINB
#define TLSPH_ZS_MINB 5
#endif
template <typename T, bool FRAC, bool VISC, int BS>
__global__ void __launch_bounds__(BS, TLSPH_ZS_MINB) k_pass2_zs(StepArgs<T> a) {
    __shared__ bool s_last;
    const int NX = a.lat_nx, NXNY = a.lat_nxny, zc = a.lat_zc;
    const int64_t t = (int64_t)blockIdx.x * BS + threadIdx.x;
    const int q = (int)(t / NXNY), c = (int)(t - (int64_t)q * NXNY);
    const int nz = (int)((a.n + NXNY - 1) / NXNY);
    const int zb = q * zc, ze = min(zb + zc, nz);
    T vmax = T(0), amax = T(0);
    int sp = 0;
    bool any = false;
    if (zb < nz) {
        ZsState<T> s;
        s.am = 0u;
#pragma unroll
        for (int k = 0; k < 7; k++) {
            s.o[k].xi = V4<T>{T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int p = 0; p < 3; p++) s.o[k].s2[p] = T(0);
        }
#pragma unroll 1
        for (int zp = zb - 3; zp < ze + 3; zp++) {
            // slot 0 takes the row z = zp + 3, whose first entries (dz = -3) lie in plane zp
            {
                const int zn = zp + 3;
                const int64_t in = (int64_t)zn * NXNY + c;
                const bool act = zn >= zb && zn < ze && in < a.n;
                s.am = (s.am << 1) & 0x7fu;
                if (act) {
                    s.am |= 1u;
                    const V4<T> x = a.X0V[in];
                    s.o[0].xi = V4<T>{x.x, x.y, x.z, T(0)};
                }
#pragma unroll
                for (int p = 0; p < 3; p++) s.o[0].s2[p] = T(0);
            }
            if (zp >= 0 && zp < nz && s.am != 0u) {
                unsigned lm[7];
#pragma unroll
                for (int k = 0; k < 7; k++)
                    lm[k] = (s.am >> k) & 1u ? __ldg(a.lmask + (int64_t)k * a.n + (int64_t)(zp + 3 - k) * NXNY + c) : 0u;
                const int pb = zp * NXNY + c;
#pragma unroll 1
                for (int dy = -3; dy <= 3; dy++) {
                    const int rb = pb + dy * NX;
                    switch (dy < 0 ? -dy : dy) {
                    case 0: zs_row<0>(a, s, rb, dy, lm); break;
                    case 1: zs_row<1>(a, s, rb, dy, lm); break;
                    case 2: zs_row<2>(a, s, rb, dy, lm); break;
                    default: zs_row<3>(a, s, rb, dy, lm); break;
                    }
                }
            }
            // slot 6 (z = zp - 3) has its last entries (dz = +3): its sum goes to the first three arrays of
            // G (F - I, which the stress pass has consumed), to be finished after the walk
            if (s.am & 0x40u) {
                const int i = (zp - 3) * NXNY + c;
#pragma unroll
                for (int p = 0; p < 3; p++) a.G[p * a.n + i] = s.o[6].s2[p];
            }
#pragma unroll
            for (int k = 6; k > 0; k--) s.o[k] = s.o[k - 1];
        }
        // the update of the thread's rows, with the registers of the walk free again
#pragma unroll 1
        for (int z = zb; z < ze; z++) {
            const int i = z * NXNY + c;
            if (i >= a.n) break;
            P2Own<T, 3> f;
            f.xi = a.X0V[i];
#pragma unroll
            for (int p = 0; p < 3; p++) f.s2[p] = a.G[p * a.n + i];
            T vmag, amag;
            p2_finish<T, 3, FRAC, VISC>(a, i, f, vmag, amag);
            sp = a.spec[i];
            any = true;
            vmax = fmax(vmax, vmag);
            amax = fmax(amax, amag);
        }
    }
    dev_block_maxima<T, BS>(a, any, sp, vmax, amax);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        dev_finalize(a);
        if (threadIdx.x == 0) *a.done = 0u;
    }
}

// ---------------------------------------------------------------- persistent step loop
// Bounded grid barrier of a cooperative launch: every block arrives once per phase; a
// block that waits longer than limit_cycles (about a second) flags kFlagTimeout and all
// blocks leave the kernel at their next barrier.
struct GridBarrier {
    unsigned int *count;
    unsigned int *gen;
    unsigned int expected;
    long long limit_cycles;
};

template <typename T> __device__ __forceinline__ bool grid_sync(const GridBarrier &b, int *flags) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = b.gen;
        volatile int *vflag = flags + kFlagTimeout;
        int ok = *vflag == 0;
        if (ok) {
            const unsigned int g0 = *vgen;
            __threadfence();
            const unsigned int arrived = atomicAdd(b.count, 1u) + 1u;
            if (arrived == b.expected) {
                atomicExch(b.count, 0u);
                __threadfence();
                atomicAdd(b.gen, 1u);
            } else {
                const long long t0 = clock64();
                while (*vgen == g0) {
                    if (*vflag != 0 || clock64() - t0 > b.limit_cycles) {
                        atomicAdd(flags + kFlagTimeout, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// nsteps steps in one cooperative launch: phase A (gradient + stress per particle, no
// neighbour dependency between them), barrier, phase B (force, damage, update), barrier.
// Block 0 advances the clocks of the previous step while phase A runs.
// FP32: eight blocks of 128 threads per SM (64 registers).  The kernel holds the neighbour walks and the
// J2 update in one body; left free it took 100-144 registers, and its latency-bound walks ran at a third
// fewer warps than the separate kernels (512-specimen batch: 1.73 against 1.08 ms per step at 64).
#ifndef TLSPH_PERSIST_MINB
#define TLSPH_PERSIST_MINB 8
#endif
template <typename T, int DIM, bool FRAC, bool VISC, int BS>
__global__ void __launch_bounds__(BS, sizeof(T) == 4 ? TLSPH_PERSIST_MINB * 128 / BS : 1) k_persistent(StepArgs<T> a, int nsteps,
                                                                                                   GridBarrier bar) {
    const int n = a.n;
    const int stride = gridDim.x * BS;
    for (int step = 0; step < nsteps; step++) {
        for (int base = blockIdx.x * BS; base < n; base += stride) {
            const int i = base + threadIdx.x;
            if (i < n) {
                prefetch_rows(a, i);
                GradOwn<T, DIM> o;
                T Gm[DIM][DIM], lap;
                dev_gradient<T, DIM, FRAC, VISC>(a, i, o, Gm, lap);
                if (FRAC) a.LAP[i] = lap;
                dev_stress<T, DIM, FRAC, false>(a, i, Gm, o.s3);
            }
        }
        if (step > 0 && blockIdx.x == 0) dev_finalize(a);
        if (!grid_sync<T>(bar, a.flags)) return;
        for (int base = blockIdx.x * BS; base < n; base += stride) {
            const int i = base + threadIdx.x;
            const bool active = i < n;
            T vmag = T(0), amag = T(0);
            int sp = 0;
            if (active) {
                prefetch_rows(a, i);
                sp = a.spec[i];
                dev_pass2<T, DIM, FRAC, VISC>(a, i, vmag, amag);
            }
            dev_block_maxima<T, BS>(a, active, sp, vmag, amag);
        }
        // ping-pong: the new displacement and velocity become current
        const V4<T> *u0 = a.ug_cur, *v0 = a.vs_cur;
        a.ug_cur = a.ug_next;
        a.vs_cur = a.vs_next;
        a.ug_next = const_cast<V4<T> *>(u0);
        a.vs_next = const_cast<V4<T> *>(v0);
        if (!grid_sync<T>(bar, a.flags)) return;
    }
    if (nsteps > 0 && blockIdx.x == 0) dev_finalize(a);
}

// ---------------------------------------------------------------- learned constitutive surrogate
// Features of a J2 material point (rows of 16): x = (F row-major 9, b_e^tr xx yy zz xy xz yz,
// eps_p^n) with the trial elastic left Cauchy-Green tensor b_e^tr = F C_p^-1 F^T, and targets
// y = (P - P^tr 9, b_e^{n+1} - b_e^tr 6, eps_p^{n+1} - eps_p^n) of the exact return map, where
// P^tr = F S(C_p^-1 of the last step) is the elastic predictor (closed form in x: P^tr = tau F^-T,
// tau = mu dev(J^-2/3 b_e^tr) + kappa/2 (J^2 - 1) I).  Stress and state enter as the plastic
// corrections, which vanish in elastic steps and stay small in plastic ones, so that the
// network's relative error neither reaches the elastic response nor accumulates in the state.
__device__ __forceinline__ void sym_to6(const M3<float> &b, float *o) {
    o[0] = b.a[0];
    o[1] = b.a[4];
    o[2] = b.a[8];
    o[3] = b.a[1];
    o[4] = b.a[2];
    o[5] = b.a[5];
}
template <typename T> __device__ __forceinline__ M3<T> left_cg(const M3<T> &F, const T K6[6]) {
    M3<T> Cp;  // C_p^-1 = I + K
    Cp.a[0] = T(1) + K6[0]; Cp.a[4] = T(1) + K6[1]; Cp.a[8] = T(1) + K6[2];
    Cp.a[1] = Cp.a[3] = K6[3];
    Cp.a[2] = Cp.a[6] = K6[4];
    Cp.a[5] = Cp.a[7] = K6[5];
    return mul(mul(F, Cp), transpose(F));
}

// Return-map samples of the current state (after k_gradient): every J2 particle whose hash
// falls in 1 / stride_el (elastic step) or 1 / stride_pl (plastic step).  WRITE = false marks
// the kept particles (flag[i] = 0 / 1); WRITE = true writes them at row offset[i] (the
// exclusive scan of the flags), in particle order.
template <typename T, int DIM, bool WRITE>
__global__ void k_j2_samples(StepArgs<T> a, int stride_el, int stride_pl, unsigned salt, int64_t *flag,
                             const int64_t *offset, float *x, float *y, float *pnorm, int64_t cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int n = a.n;
    const MatT<T> m = a.mats[a.mid[i]];
    if (m.model != 3) {
        if (!WRITE) flag[i] = 0;
        return;
    }
    M3<T> G = m3_zero<T>();
    for (int p = 0; p < DIM; p++)
        for (int q = 0; q < DIM; q++) G(p, q) = a.G[(p * DIM + q) * n + i];
    const Kin<T> kin = kinematics(G);
    T K6[6], K6o[6], epo, dg;
    for (int q = 0; q < 6; q++) K6[q] = a.K[q * n + i];
    const T ep = a.ep[i];
    M3<T> S;
    j2_update(kin, K6, ep, m, K6o, epo, S, dg);
    const unsigned h = (unsigned)i * 2654435761u ^ (salt * 2246822519u + 0x9e3779b9u);
    const unsigned stride = dg > T(0) ? (unsigned)stride_pl : (unsigned)stride_el;
    const bool keep = ((h >> 7) % stride) == 0u;
    if (!WRITE) {
        flag[i] = keep ? 1 : 0;
        return;
    }
    if (!keep || offset[i] >= cap) return;
    M3<T> F = G;
    F.a[0] += T(1);
    F.a[4] += T(1);
    F.a[8] += T(1);
    const M3<T> P = mul(F, S);
    // elastic predictor: the stress of the trial state (C_p^-1 of the last step)
    const M3<T> Ptr = mul(F, j2_stress(kin, j2_trial(kin, K6, ep, m).dev, m));
    const M3<T> btr = left_cg(F, K6), bnew = left_cg(F, K6o);
    float *xr = x + 16 * offset[i], *yr = y + 16 * offset[i];
    M3<float> bf, bd;
    T pn = T(0);
    for (int q = 0; q < 9; q++) {
        xr[q] = (float)F.a[q];
        yr[q] = (float)(P.a[q] - Ptr.a[q]);
        bf.a[q] = (float)btr.a[q];
        bd.a[q] = (float)(bnew.a[q] - btr.a[q]);
        pn += P.a[q] * P.a[q];
    }
    if (pnorm) pnorm[offset[i]] = (float)t_sqrt(pn);
    sym_to6(bf, xr + 9);
    sym_to6(bd, yr + 9);
    xr[15] = (float)ep;
    yr[15] = (float)(epo - ep);
}

// Features of the surrogate for particle i (FP32): xn = normalised (F, b_e^tr, eps_p) when i is a
// J2 particle without phase field that the network serves (inside the envelope and, with scope 1,
// with a yielding trial state); returns whether it does.  Counts the J2 particles it leaves to the
// exact update (n_out: outside the envelope, n_el: elastic trial state under scope 1).
template <int DIM, bool FRAC>
__device__ __forceinline__ bool sur_features(const StepArgs<float> &a, const SurrogateDev &s, int i, const M3<float> &G,
                                             float xn[16], int &n_out, int &n_el) {
    const int n = a.n;
    const MatT<float> m = a.mats[a.mid[i]];
    if (m.model != 3 || (FRAC && m.fracture)) return false;
    float K6[6];
    for (int q = 0; q < 6; q++) K6[q] = a.K[q * n + i];
    const float ep = a.ep[i];
    if (s.scope == 1 && !(j2_trial(kinematics(G), K6, ep, m).f > 0.0f)) {
        n_el++;
        return false;
    }
    M3<float> F = G;
    F.a[0] += 1.0f;
    F.a[4] += 1.0f;
    F.a[8] += 1.0f;
    const M3<float> btr = left_cg(F, K6);
    float xr[16];
    for (int q = 0; q < 9; q++) xr[q] = F.a[q];
    sym_to6(btr, xr + 9);
    xr[15] = ep;
    bool use = s.enabled != 0;
    for (int c = 0; c < 16; c++) {
        xn[c] = __fdividef(xr[c] - s.in_mean[c], s.in_std[c]);
        use = use && xn[c] >= s.env_lo[c] && xn[c] <= s.env_hi[c];
    }
    if (!use) n_out++;
    return use;
}

// Apply the network's outputs yn (normalised) to particle i: P = elastic predictor + correction,
// C_p^-1 += F^-1 db F^-T with det C_p^-1 = 1 (eq. Fp_iso_proj), eps_p += max(0, increment), and
// the pass-2 matrices.  The outputs are kept only if the new C_p^-1 is symmetric positive definite
// (leading minors of I + K positive) and the stress finite; otherwise nothing is written and the
// function returns false, so that the exact update serves the particle (a metric that is not
// positive definite would leave later return maps without a bracket).
template <int DIM, bool FRAC>
__device__ __forceinline__ bool sur_apply(const StepArgs<float> &a, const SurrogateDev &s, int i, const M3<float> &G,
                                          const float yn[16]) {
    const int n = a.n;
    float yr[16];
    for (int c = 0; c < 16; c++) yr[c] = yn[c] * s.out_std[c] + s.out_mean[c];
    const MatT<float> m = a.mats[a.mid[i]];
    float K6[6];
    for (int q = 0; q < 6; q++) K6[q] = a.K[q * n + i];
    const Kin<float> kin = kinematics(G);
    M3<float> F = G;
    F.a[0] += 1.0f;
    F.a[4] += 1.0f;
    F.a[8] += 1.0f;
    M3<float> P = mul(F, j2_stress(kin, j2_trial(kin, K6, a.ep[i], m).dev, m)), db;
    for (int q = 0; q < 9; q++) P.a[q] += yr[q];
    db.a[0] = yr[9]; db.a[4] = yr[10]; db.a[8] = yr[11];
    db.a[1] = db.a[3] = yr[12];
    db.a[2] = db.a[6] = yr[13];
    db.a[5] = db.a[7] = yr[14];
    if (DIM == 2) {  // plane strain: keep the in-plane block structure
        P.a[2] = P.a[5] = P.a[6] = P.a[7] = 0.0f;
        db.a[2] = db.a[6] = db.a[5] = db.a[7] = 0.0f;
    }
    // b_e^{n+1} = b_e^tr + db with b_e^tr = F C_p^-1 F^T, so C_p^-1 grows by F^-1 db F^-T (added to
    // C_p^-1 - I directly: no cancellation), then det C_p^-1 = 1 as in eq. Fp_iso_proj
    M3<float> Fi;
    inverse(F, Fi);
    const M3<float> dK = sym_part(mul(mul(Fi, db), transpose(Fi)));
    M3<float> Kn;
    Kn.a[0] = K6[0]; Kn.a[4] = K6[1]; Kn.a[8] = K6[2];
    Kn.a[1] = Kn.a[3] = K6[3];
    Kn.a[2] = Kn.a[6] = K6[4];
    Kn.a[5] = Kn.a[7] = K6[5];
    for (int q = 0; q < 9; q++) Kn.a[q] += dK.a[q];
    const float dm1 = det_eye_plus_m1(Kn);
    {
        const float a00 = 1.0f + Kn.a[0], a11 = 1.0f + Kn.a[4];
        bool ok = isfinite(dm1) && dm1 > -1.0f && a00 > 0.0f && a00 * a11 - Kn.a[1] * Kn.a[1] > 0.0f;
        for (int q = 0; q < 9; q++) ok = ok && isfinite(P.a[q]) && isfinite(Kn.a[q]);
        if (!ok) return false;
    }
    const float fm1 = expm1f(-log1pf(dm1) / 3.0f);
    for (int q = 0; q < 9; q++) Kn.a[q] = Kn.a[q] * (1.0f + fm1);
    a.K[0 * n + i] = Kn.a[0] + fm1;
    a.K[1 * n + i] = Kn.a[4] + fm1;
    a.K[2 * n + i] = Kn.a[8] + fm1;
    a.K[3 * n + i] = Kn.a[1];
    a.K[4 * n + i] = Kn.a[2];
    a.K[5 * n + i] = Kn.a[5];
    a.ep[i] = a.ep[i] + fmaxf(yr[15], 0.0f);  // irreversible
    dev_write_qvm_fi<float, DIM>(a, i, Fi, P, 1.0f + kin.Jm1, 1.0f / m.rho, nullptr);
    return true;
}

// The surrogate inputs of the tile of 128 particles starting at particle base (G, C_p^-1 - I, eps_p and
// material ids) into L2 by the TMA unit while the current tile runs through the network: thread r of the
// tile's threads issues one bulk prefetch for one array, over the whole 16-byte units of the tile's slice
// (aligned, and inside the array).  A hint only: nothing depends on it.
template <int DIM>
__device__ __forceinline__ void sur_prefetch_tile(const StepArgs<float> &a, int base, int r) {
    const int n = a.n;
    if (base >= n) return;
    const int cnt = min(128, n - base);
    const int na = DIM * DIM + 6;
    const char *lo = nullptr, *hi = nullptr;
    if (r < na) {
        const float *arr = r < DIM * DIM ? a.G + (int64_t)r * n : a.K + (int64_t)(r - DIM * DIM) * n;
        lo = reinterpret_cast<const char *>(arr + base);
        hi = reinterpret_cast<const char *>(arr + base + cnt);
    } else if (r == na) {
        lo = reinterpret_cast<const char *>(a.ep + base);
        hi = reinterpret_cast<const char *>(a.ep + base + cnt);
    } else if (r == na + 1) {
        lo = reinterpret_cast<const char *>(a.mid + base);
        hi = reinterpret_cast<const char *>(a.mid + base + cnt);
    } else {
        return;
    }
    const uintptr_t a0 = (reinterpret_cast<uintptr_t>(lo) + 15) & ~(uintptr_t)15;
    const uintptr_t a1 = reinterpret_cast<uintptr_t>(hi) & ~(uintptr_t)15;
    if (a1 > a0) prefetch_l2_bulk(reinterpret_cast<const void *>(a0), (uint32_t)(a1 - a0));
}

// Append row i (when need) to the list of rows left to the exact update: one atomic per warp.  All 32
// lanes of the warp call it.
__device__ __forceinline__ void sur_list_push(int *list, unsigned *nlist, bool need, int i) {
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m == 0u) return;
    const unsigned lane = threadIdx.x & 31u;
    unsigned base = 0u;
    if (lane == 0u) base = atomicAdd(nlist, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (need) list[base + (unsigned)__popc(m & ((1u << lane) - 1u))] = i;
}

__device__ __forceinline__ void sur_count(unsigned long long *counters, int n_mlp, int n_out, int n_el) {
    for (int o = 16; o > 0; o >>= 1) {
        n_mlp += __shfl_xor_sync(0xffffffffu, n_mlp, o);
        n_out += __shfl_xor_sync(0xffffffffu, n_out, o);
        n_el += __shfl_xor_sync(0xffffffffu, n_el, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counters[0], (unsigned long long)n_mlp);
        atomicAdd(&counters[1], (unsigned long long)n_out);
        atomicAdd(&counters[2], (unsigned long long)n_el);
    }
}

// Pass 1b with the surrogate (FP32), warp-level tensor cores: every block loads the network into
// shared memory once and walks tiles of 128 particles.  A J2 particle (without phase field) whose
// normalised features lie inside the training envelope takes the plastic corrections of P and of
// its state from the network (BF16 mma.sync, FP32 accumulation) on top of the closed-form
// elastic predictor; with scope 1 only particles whose trial state yields do.  Every other
// particle goes to the list exact (nexact rows) for k_stress_exact, which runs next.  A tile in which no
// particle uses the network skips the forward pass.
// counters: [0] network, [1] J2 outside the envelope, [2] elastic trial states (scope 1).
template <int DIM, bool FRAC>
__global__ void __launch_bounds__(128, 2) k_stress_sur(StepArgs<float> a, SurrogateDev s, int *exact, unsigned *nexact,
                                                       unsigned long long *counters) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    mlp_load_params(sm, s);
    __syncthreads();
    const int n = a.n, ntiles = (n + 127) / 128;
    int n_mlp = 0, n_out = 0, n_el = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * 128 + threadIdx.x;
        const bool active = i < n;
        sur_prefetch_tile<DIM>(a, (tile + gridDim.x) * 128, threadIdx.x);
        bool use = false;
        float xn[16];
        M3<float> G = m3_zero<float>();
        if (active) {
            for (int p = 0; p < DIM; p++)
                for (int q = 0; q < DIM; q++) G(p, q) = a.G[(p * DIM + q) * n + i];
            use = sur_features<DIM, FRAC>(a, s, i, G, xn, n_out, n_el);
        }
        bool need = active && !use;
        for (int c = 0; c < 16; c++) sm.X[threadIdx.x][c] = __float2bfloat16_rn(use ? xn[c] : 0.0f);
        if (__syncthreads_or(use)) {  // block-uniform
            mlp_forward_block(sm);
            if (use) {
                if (sur_apply<DIM, FRAC>(a, s, i, G, sm.Y[threadIdx.x])) {
                    n_mlp++;
                } else {  // rejected output: the exact update serves the particle
                    need = true;
                    n_out++;
                }
            }
        }
        sur_list_push(exact, nexact, need, i);
        __syncthreads();
    }
    sur_count(counters, n_mlp, n_out, n_el);
}

// The same pass on the 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM; see
// mlp_tc.cuh): CTAs of 4 groups x 128 threads, each group persistent over tiles of 128
// particles.  A wait on the tensor cores that runs out sets kFlagTimeout and ends the group's
// work (its remaining particles keep their old state).
template <int DIM, bool FRAC>
__global__ void __launch_bounds__(128 * kTcGroups, 1) k_stress_sur_tc(StepArgs<float> a, SurrogateDev s, int *exact,
                                                                     unsigned *nexact, unsigned long long *counters) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpTcSmem &sm = *reinterpret_cast<MlpTcSmem *>(smraw);
    mlp_tc_setup(sm, s);
    const int g = threadIdx.x >> 7, r = threadIdx.x & 127;
    unsigned phase = 0;
    bool pending = false;
    const int n = a.n, ntiles = (n + 127) / 128;
    int n_mlp = 0, n_out = 0, n_el = 0;
    for (int tile = blockIdx.x * kTcGroups + g; tile < ntiles; tile += gridDim.x * kTcGroups) {
        const int i = tile * 128 + r;
        const bool active = i < n;
        sur_prefetch_tile<DIM>(a, (tile + gridDim.x * kTcGroups) * 128, r);
        bool use = false;
        float xn[16];
        M3<float> G = m3_zero<float>();
        if (active) {
            for (int p = 0; p < DIM; p++)
                for (int q = 0; q < DIM; q++) G(p, q) = a.G[(p * DIM + q) * n + i];
            use = sur_features<DIM, FRAC>(a, s, i, G, xn, n_out, n_el);
        }
        bool need = active && !use;
        if (!use)
            for (int c = 0; c < 16; c++) xn[c] = 0.0f;
        mlp_tc_put_row(sm, g, r, xn);
        if (group_or(g, use)) {  // group-uniform
            float yn[16];
            if (!mlp_tc_tile(sm, g, r, phase, yn)) {
                if (r == 0) atomicAdd(&a.flags[kFlagTimeout], 1);
                pending = true;
                break;
            }
            if (use) {
                if (sur_apply<DIM, FRAC>(a, s, i, G, yn)) {
                    n_mlp++;
                } else {  // rejected output: the exact update serves the particle
                    need = true;
                    n_out++;
                }
            }
        }
        sur_list_push(exact, nexact, need, i);
    }
    mlp_tc_finish(sm, g, phase, pending);
    sur_count(counters, n_mlp, n_out, n_el);
}

// The exact constitutive update of the particles the network pass left to it: the nexact rows of the
// list exact, in the order the network pass appended them (each particle's update is its own, so the
// order does not change a result).  Consecutive threads take consecutive list entries, so a warp's lanes
// all work however few and scattered the rows are.
template <int DIM, bool FRAC, int BS>
__global__ void __launch_bounds__(BS) k_stress_exact(StepArgs<float> a, const int *exact, const unsigned *nexact) {
    const unsigned cnt = *nexact;
    for (unsigned k = blockIdx.x * BS + threadIdx.x; k < cnt; k += gridDim.x * BS) {
        const int i = exact[k];
        float Gm[DIM][DIM];
#pragma unroll
        for (int p = 0; p < DIM; p++)
#pragma unroll
            for (int q = 0; q < DIM; q++) Gm[p][q] = a.G[(p * DIM + q) * a.n + i];
        dev_stress<float, DIM, FRAC, false>(a, i, Gm);
    }
}

// ---------------------------------------------------------------- diagnostics
// grad s and the energy densities of the current state (FP64 sums).
template <typename T, int DIM, bool FRAC>
__global__ void __launch_bounds__(128) k_energy(StepArgs<T> a, double *out) {
    __shared__ double red[5][4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e[5] = {0, 0, 0, 0, 0};
    if (i < a.n) {
        const int n = a.n;
        const MatT<T> m = a.mats[a.mid[i]];
        const V4<T> xi = a.X0V[i];
        const V4<T> vsi = a.vs_cur[i];
        const double V = DIM == 3 ? (double)xi.w : (double)xi.z;
        const double vv = (double)vsi.x * vsi.x + (double)vsi.y * vsi.y + (double)vsi.z * vsi.z;
        e[0] = 0.5 * (double)m.rho * V * vv;
        e[1] = V * (double)a.psi_out[i];
        e[4] = a.wext[i];
        if (m.model == 3) {
            const double ep = a.ep[i];
            e[3] = V * ((double)m.sy0 * ep + 0.5 * (double)m.Hh * ep * ep);
        }
        if (FRAC && m.fracture) {
            const int64_t base = a.slice_off[i >> 5] + (i & 31);
            const int len = a.row_len[i];
            double gs[3] = {0, 0, 0};
            for (int k = 0; k < len; k++) {
                const int j = a.col[base + 32 * k];
                const V4<T> xj = a.X0V[j];
                double d[3] = {(double)(xj.x - xi.x), (double)(xj.y - xi.y), DIM == 3 ? (double)(xj.z - xi.z) : 0.0};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double t = fmax(1.0 - r * (double)a.inv2h, 0.0);
                double Vj = DIM == 3 ? (double)xj.w : (double)xj.z;
                double c = Vj * t * t * t * ((double)a.vs_cur[j].w - (double)vsi.w);
                for (int p = 0; p < 3; p++) gs[p] += c * d[p];
            }
            T A[3][3];
            load_ahat<T, DIM>(a.Ahat, n, i, A);
            double g2 = 0.0;
            for (int p = 0; p < DIM; p++) {
                double gp = 0.0;
                for (int q = 0; q < DIM; q++) gp += (double)A[p][q] * gs[q];
                g2 += gp * gp;
            }
            const double om = 1.0 - (double)vsi.w;
            e[2] = V * (double)m.Gc * (om * om / (4.0 * (double)m.eps0) + (double)m.eps0 * g2);
        }
    }
    for (int q = 0; q < 5; q++)
        for (int o = 16; o > 0; o >>= 1) e[q] += __shfl_xor_sync(0xffffffffu, e[q], o);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 5; q++) red[q][threadIdx.x >> 5] = e[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; q++) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[q][w];
            atomicAdd(&out[q], s);
        }
}

// ---------------------------------------------------------------- gathers to / from the caller's order
// out[perm[k] * nc + c] = src_c[k] for c < nc, sources given as nc strided arrays of T.
template <typename S>
__global__ void k_to_caller(int64_t n, int nc, const S *src, int64_t cstride, const int *perm, double *out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    for (int c = 0; c < nc; c++) out[p * nc + c] = (double)src[c * cstride + k];
}
template <typename S>
__global__ void k_from_caller(int64_t n, int nc, const double *in, const int *perm, S *dst, int64_t cstride) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    for (int c = 0; c < nc; c++) dst[c * cstride + k] = (S)in[p * nc + c];
}
// V4 records (vs, ug): component c of record k
template <typename T>
__global__ void k_v4_to_caller(int64_t n, int nc, int c0, const V4<T> *src, const int *perm, double *out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    const T *r = reinterpret_cast<const T *>(src + k);
    for (int c = 0; c < nc; c++) out[p * nc + c] = (double)r[c0 + c];
}
template <typename T>
__global__ void k_v4_from_caller(int64_t n, int nc, int c0, const double *in, const int *perm, V4<T> *dst) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    T *r = reinterpret_cast<T *>(dst + k);
    for (int c = 0; c < nc; c++) r[c0 + c] = (T)in[p * nc + c];
}
// current position X0 + u (FP64) to the caller
__global__ void k_x_to_caller(int64_t n, int dim, const double *X0d, const double *u64, const int *perm, double *out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    for (int c = 0; c < dim; c++) out[p * dim + c] = X0d[c * n + k] + u64[c * n + k];
}
// u64 (FP64) -> gathered copy ug
template <typename T> __global__ void k_refresh_ug(int64_t n, int dim, const double *u64, V4<T> *ug) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    ug[k] = V4<T>{(T)u64[k], (T)u64[n + k], dim == 3 ? (T)u64[2 * n + k] : T(0), ug[k].w};
}
// C_p^-1 = I + K (9 components) to the caller
template <typename T> __global__ void k_cpinv_to_caller(int64_t n, const T *K, const int *perm, double *out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
    for (int c = 0; c < 9; c++) out[p * 9 + c] = (double)K[map[c] * n + k] + ((c % 4) == 0 ? 1.0 : 0.0);
}
template <typename T> __global__ void k_cpinv_from_caller(int64_t n, const double *in, const int *perm, T *K) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t p = perm[k];
    const int src[6] = {0, 4, 8, 1, 2, 5};
    for (int q = 0; q < 6; q++) K[q * n + k] = (T)(in[p * 9 + src[q]] - ((src[q] % 4) == 0 ? 1.0 : 0.0));
}
// caller CSR: row lengths in caller order, then rows mapped to caller ids and sorted
__global__ void k_rowlen_caller(int64_t n, const int *row_len, const int *perm, int64_t *len_out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) len_out[perm[k]] = row_len[k];
}
__global__ void k_rows_caller(int64_t n, const int64_t *row_ptr, const int *col, const int *perm, const int64_t *rp_out,
                              int *col_out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t b = row_ptr[k], e = row_ptr[k + 1], o = rp_out[perm[k]];
    for (int64_t q = 0; q < e - b; q++) col_out[o + q] = perm[col[b + q]];
    for (int64_t x = 1; x < e - b; x++) {  // insertion sort: rows are short
        int v = col_out[o + x];
        int64_t y = x - 1;
        while (y >= 0 && col_out[o + y] > v) {
            col_out[o + y + 1] = col_out[o + y];
            y--;
        }
        col_out[o + y + 1] = v;
    }
}

// ---- user-defined expressions (Sec. 3.3)

// Built-in variables of particle i at time t: x0 y0 z0 x y z ux uy uz t dt dx (FP64 reference positions
// and displacement).
template <typename T, int DIM>
__device__ __forceinline__ void ex_vars(const StepArgs<T> &a, const double *X0d, int i, double t, double dt,
                                        double dx, double v[kExVars]) {
    const int n = a.n;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const double x0 = q < DIM ? X0d[q * n + i] : 0.0;
        const double u = q < DIM ? a.u64[q * n + i] : 0.0;
        v[q] = x0;
        v[3 + q] = x0 + u;
        v[6 + q] = u;
    }
    v[9] = t;
    v[10] = dt;
    v[11] = dx;
}

// Evaluates the expressions of the boundary conditions of the listed particles for the coming step,
// with the state at its start: velocity values at t_{n+1} (and, for Algorithm 2, at t_{n+1/2} for the
// predictor, phase 1), force values at the time of the forces.  One thread per listed particle.
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_expr_bcs(StepArgs<T> a, const int *exlist, int m, const double *X0d,
                                                  const ExInstr *code, const double *K, const ExProg *progs,
                                                  double dx, double *exval, uint16_t *exskip) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const int i = exlist[p];
    const int g = a.bcgrp[i];
    const int sp = a.spec[i];
    const double t = a.t[sp], dt = a.dt[sp];
    double v[kExVars];
    ex_vars<T, DIM>(a, X0d, i, t, dt, dx, v);
    uint32_t skip0 = 0, skip1 = 0;
    for (int b = 0; b < kMaxBcPerParticle && g; b++) {
        const int id = a.grp_bcs[4 * g + b];
        if (id < 0) break;
        const BCDev bc = a.bcs[id];
        for (int k = 0; k < DIM; k++) {
            const int e = bc.expr[k];
            if (e < 0 || !(bc.comp_mask & (1 << k))) continue;
            const ExProg pr = progs[e];
            const int nph = ((bc.kind == 0 || bc.kind == 4) && a.leap) ? 2 : 1;
            for (int ph = 0; ph < nph; ph++) {
                double off;
                if (bc.kind == 0 || bc.kind == 4) off = ph == 0 ? dt : 0.5 * dt;  // the new level t_{n+1}
                else off = a.leap ? 0.5 * dt : 0.0;
                v[9] = t + off;
                bool sk;
                const double val = ex_run(code + pr.code, pr.ncode, K + pr.consts, v, sk);
                exval[(2 * p + ph) * 12 + 3 * b + k] = val;
                if (sk) (ph == 0 ? skip0 : skip1) |= 1u << (3 * b + k);
            }
        }
    }
    exskip[2 * p] = (uint16_t)skip0;
    exskip[2 * p + 1] = (uint16_t)skip1;
}

// Sets components of the displacement (field 0) or velocity (field 1) of every particle to expressions
// evaluated now (time t_n of its specimen); a skipped value or a component without an expression (-1)
// is left alone.  The FP32 copy of the displacement follows.
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_expr_field(StepArgs<T> a, const double *X0d, const ExInstr *code,
                                                    const double *K, const ExProg *progs, int3 ids, double dx,
                                                    int field, V4<T> *ug, V4<T> *vs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int n = a.n;
    const int sp = a.spec[i];
    double v[kExVars];
    ex_vars<T, DIM>(a, X0d, i, a.t[sp], a.dt[sp], dx, v);
    const int id[3] = {ids.x, ids.y, ids.z};
    double val[3];
    bool set[3] = {false, false, false};
    for (int k = 0; k < DIM; k++) {
        if (id[k] < 0) continue;
        const ExProg pr = progs[id[k]];
        bool sk;
        val[k] = ex_run(code + pr.code, pr.ncode, K + pr.consts, v, sk);
        set[k] = !sk;
    }
    if (field == 0) {
        V4<T> r = ug[i];
        T *rc = &r.x;
        for (int k = 0; k < DIM; k++)
            if (set[k]) {
                a.u64[k * n + i] = val[k];
                rc[k] = (T)val[k];
            }
        ug[i] = r;
    } else {
        V4<T> r = vs[i];
        T *rc = &r.x;
        for (int k = 0; k < DIM; k++)
            if (set[k]) rc[k] = (T)val[k];
        vs[i] = r;
    }
}

}  // namespace tl
