/*
 * FP64 CPU oracle for the total-Lagrangian SPH (TLSPH) solid step of
 * "SoliDualSPHysics" (arXiv 2602.15149).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library and the timed CPU baseline.  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline leg may load it.  It shares no code, header
 * or constant with the CUDA path.
 *
 * Everything is plain FP64 and written in the paper's order and notation:
 *   - reference configuration: neighbours by the predicate r0^2 < R^2,
 *     correction tensor L_i (Sec. 2.4, corrected kernel gradient),
 *   - deformation gradient F_i (Sec. 2.4, eq. deformGradTLSPH; soft
 *     particles eq. defGrad_phase),
 *   - neo-Hookean stress with the J-split (Sec. 2.3.2) and finite-strain J2
 *     plasticity stored as F_p with exponential-map return (Sec. 2.3.3),
 *   - symmetric momentum sum with artificial viscosity (Sec. 2.4,
 *     eq. MomentumEqTLSPH, eq. artViscCoef),
 *   - hyperbolic phase field (Sec. 2.2, eq. phasefieldddot, SPH Laplacian
 *     eq. phasefieldLapLacian),
 *   - Algorithm 1 (symplectic Euler) or Algorithm 2 (leapfrog) time update
 *     with velocity / force boundary conditions (Sec. 2.5, Sec. 3.3.2), and
 *     the time-step bound eq. dt_criterion.
 *
 * Readings of the paper where it is silent or inconsistent are marked
 * "reading:" below.  Compile with -ffp-contract=off so that no fused
 * multiply-add changes the reference-configuration predicates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_OOM -3
#define ORC_ERR_SINGULAR -4
#define ORC_ERR_NONFINITE -5
#define ORC_ERR_STATE -8

#define ORC_MODEL_SVK 1
#define ORC_MODEL_NH 2
#define ORC_MODEL_J2 3

#define ORC_BC_VEL 0
#define ORC_BC_TRACTION 1
#define ORC_BC_ACCEL 2
#define ORC_BC_POINTFORCE 3
#define ORC_BC_PHASE_BOUND 4 /* <restrictphi> (Sec. 3.3): s >= value at t_{n+1}, component 0 */

#define ORC_DT_FIXED 0
#define ORC_DT_ADAPTIVE 1
#define ORC_DT_CFL_STATIC 2

#define ORC_MAX_BC 256
#define ORC_MAX_NOTCH 512

typedef struct {
    int dim;            /* 2 (plane strain, x-y plane, F_zz = 1) or 3 */
    double h;           /* smoothing length */
    double support;     /* R = support * h (Wendland C2: 2) */
    double cfl;         /* C_CFL of eq. dt_criterion */
    int dt_mode;        /* ORC_DT_* */
    double fixed_dt;    /* used when dt_mode == ORC_DT_FIXED */
    double gravity[3];  /* body force per unit mass f_0 */
    int visc_literal;   /* 0: Pv = -J pi F^-T (dissipative reading), 1: literal +J pi F^-1 */
    int lap_uncorrected;/* 0: Laplacian uses the corrected gradient, 1: raw kernel gradient */
    int integrator;     /* 1 (or 0): Algorithm 1, symplectic Euler; 2: Algorithm 2, leapfrog */
    int pf_explicit;    /* 0: the phase field's local terms at the new time level (reading); 1: the printed
                         * explicit update sdot_{n+1} = sdot_n + dt sddot_n of Algorithm 1 */
} orc_params;

typedef struct {
    int model;          /* ORC_MODEL_SVK, ORC_MODEL_NH or ORC_MODEL_J2 */
    double rho, E, nu;
    double sigma_y0, H_hard;
    double beta1, beta2;
    int fracture;
    double Gc, eps0, s_lim;
} orc_material;

typedef struct {
    int kind, comp_mask;
    double value[3];
    double t_start, t_end, ramp, area;
    uint8_t *mask;
    int64_t count;
    /* user-defined expressions (Sec. 3.3): per-particle prescribed values (n x 3) and skip flags set
     * before each step by the caller; [0] for the step's value, [1] for the leapfrog predictor */
    double *exval[2];
    uint8_t *exskip[2];
} orc_bc;

typedef struct orc_ctx {
    orc_params p;
    int nmat;
    orc_material *mat;
    int64_t n;
    int nspec;
    double *X0, *vol, *u, *v, *acc, *s, *sdot, *sdd, *Hh, *Fp, *ep;
    double *lap, *pf_b, *pf_k, *pf_g;  /* phase-field terms of the current step */
    double *aext;                /* acceleration of the external forces of the current step (n x 3) */
    double *wext;                /* work of the external forces on each particle since the reference setup */
    int32_t *mid, *spec;
    double *F, *P, *L;           /* per-particle 3x3 (L: in-plane block) */
    int32_t *status;             /* per-particle return-map status */
    int nbc;
    orc_bc bc[ORC_MAX_BC];
    int nnotch;
    double notch[ORC_MAX_NOTCH][12];
    int64_t *row_ptr;
    int32_t *col;
    int64_t *perm;               /* cell-sorted order (reference setup) */
    double cell_size, xmin[3];
    int64_t ncell[3];
    double *t, *dt, *vmax, *amax, *cmax; /* per specimen */
    int64_t step;
    int64_t noconv;
    int built;
    /* contact between bodies (the specimens): on/off, potential multiplier, contact distance,
     * restitution per specimen, contact accelerations of the current step */
    int contact;
    double kc, dc;
    double *rest;
    double *kfric;  /* per body <kfric>, or NULL (no friction) */
    double *accc;
} orc_ctx;

/* ------------------------------------------------------------------ */
/* small dense 3x3 helpers (row-major a[3*r+c])                        */
/* ------------------------------------------------------------------ */
static void m_eye(double *a) { memset(a, 0, 9 * sizeof(double)); a[0] = a[4] = a[8] = 1.0; }
static void m_mul(const double *a, const double *b, double *c) {
    double t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = s;
        }
    memcpy(c, t, sizeof t);
}
static void m_tr(const double *a, double *b) {
    double t[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) t[3 * i + j] = a[3 * j + i];
    memcpy(b, t, sizeof t);
}
static double m_det(const double *a) {
    return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
           a[2] * (a[3] * a[7] - a[4] * a[6]);
}
static int m_inv(const double *a, double *b) {
    double d = m_det(a);
    if (!(d != 0.0) || !isfinite(d)) return -1;
    double t[9];
    t[0] = (a[4] * a[8] - a[5] * a[7]) / d;
    t[1] = (a[2] * a[7] - a[1] * a[8]) / d;
    t[2] = (a[1] * a[5] - a[2] * a[4]) / d;
    t[3] = (a[5] * a[6] - a[3] * a[8]) / d;
    t[4] = (a[0] * a[8] - a[2] * a[6]) / d;
    t[5] = (a[2] * a[3] - a[0] * a[5]) / d;
    t[6] = (a[3] * a[7] - a[4] * a[6]) / d;
    t[7] = (a[1] * a[6] - a[0] * a[7]) / d;
    t[8] = (a[0] * a[4] - a[1] * a[3]) / d;
    memcpy(b, t, sizeof t);
    return 0;
}
static double m_trace(const double *a) { return a[0] + a[4] + a[8]; }
static double m_ddot(const double *a, const double *b) {
    double s = 0.0;
    for (int k = 0; k < 9; k++) s += a[k] * b[k];
    return s;
}
static void m_scale(double *a, double s) { for (int k = 0; k < 9; k++) a[k] *= s; }
static void m_dev(const double *a, double *d) {
    double m = m_trace(a) / 3.0;
    for (int k = 0; k < 9; k++) d[k] = a[k];
    d[0] -= m; d[4] -= m; d[8] -= m;
}

/* Matrix exponential by scaling and squaring of a Taylor series (Sec. 2.3.3,
 * "scaling-and-squaring Taylor scheme").  reading: scale by 2^-k until the
 * Frobenius norm is at most 1/8, Taylor order 12, square k times. */
void orc_expm(const double *A, double *E) {
    double nrm = sqrt(m_ddot(A, A));
    int k = 0;
    while (nrm > 0.125 && k < 60) { nrm *= 0.5; k++; }
    double B[9];
    for (int i = 0; i < 9; i++) B[i] = ldexp(A[i], -k);
    double term[9], sum[9];
    m_eye(term);
    m_eye(sum);
    for (int m = 1; m <= 12; m++) {
        m_mul(term, B, term);
        m_scale(term, 1.0 / (double)m);
        for (int i = 0; i < 9; i++) sum[i] += term[i];
    }
    for (int i = 0; i < k; i++) m_mul(sum, sum, sum);
    memcpy(E, sum, 9 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* Wendland C2 kernel (Kernel=2 of the appendices):                    */
/* W(q) = alpha_D (1 - q/2)^4 (2q + 1), q = r/h in [0, 2].             */
/* ------------------------------------------------------------------ */
static double wendland_alpha(int dim, double h) {
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}
void orc_wendland(int dim, double h, double r, double *W, double *dWdr) {
    double q = r / h, a = wendland_alpha(dim, h);
    if (q >= 2.0) { *W = 0.0; *dWdr = 0.0; return; }
    double t = 1.0 - 0.5 * q;
    *W = a * t * t * t * t * (2.0 * q + 1.0);
    /* d/dr: (a/h) d/dq[(1-q/2)^4 (2q+1)] = (a/h)(-5 q (1-q/2)^3) */
    *dWdr = (a / h) * (-5.0 * q * t * t * t);
}

/* Gradient with respect to X_i of W(|X_i - X_j|): (dW/dr) (X_i - X_j)/r. */
static void kernel_grad(const orc_ctx *c, const double *r0, double r, double *g) {
    double W, dW;
    orc_wendland(c->p.dim, c->p.h, r, &W, &dW);
    for (int k = 0; k < 3; k++) g[k] = dW * r0[k] / r;
}

/* ------------------------------------------------------------------ */
/* material constants                                                  */
/* ------------------------------------------------------------------ */
static void lame(const orc_material *m, double *lam, double *mu, double *kap) {
    *lam = m->E * m->nu / ((1.0 + m->nu) * (1.0 - 2.0 * m->nu));
    *mu = m->E / (2.0 * (1.0 + m->nu));
    *kap = *lam + 2.0 * (*mu) / 3.0; /* Sec. 2.2: kappa = lambda + 2 mu / 3 */
}
/* Sec. 2.2 / eq. speedofsound: c = sqrt((kappa + 4 mu / 3) / rho0). */
double orc_sound_speed(const orc_material *m) {
    double lam, mu, kap;
    lame(m, &lam, &mu, &kap);
    return sqrt((kap + 4.0 * mu / 3.0) / m->rho);
}

/* ------------------------------------------------------------------ */
/* Neo-Hookean stress with the J-split (Sec. 2.3.2).                   */
/* reading: the printed stress is written with b^-1; S = 2 dpsi/dC     */
/* gives C^-1, which is what is used here (it is the form that is      */
/* frame-indifferent and equals the derivative of the stated energy). */
/* ------------------------------------------------------------------ */
int orc_nh_stress(const double *F, double s, const orc_material *m, double *S, double *psi_plus,
                  double *psi_minus) {
    double lam, mu, kap;
    lame(m, &lam, &mu, &kap);
    double Ft[9], C[9], Ci[9];
    m_tr(F, Ft);
    m_mul(Ft, F, C);
    double J = m_det(F);
    if (!(J > 0.0) || m_inv(C, Ci) != 0) return ORC_ERR_NONFINITE;
    double trC = m_trace(C);
    double Jm23 = pow(J, -2.0 / 3.0);
    double Svol[9], Siso[9], I[9];
    m_eye(I);
    for (int k = 0; k < 9; k++) {
        Svol[k] = 0.5 * kap * (J * J - 1.0) * Ci[k];
        Siso[k] = mu * Jm23 * (I[k] - trC / 3.0 * Ci[k]);
    }
    double U = 0.5 * kap * (0.5 * (J * J - 1.0) - log(J)); /* eq. UjNeoHok */
    double psibar = 0.5 * mu * (Jm23 * trC - 3.0);         /* eq. ksiNeoHok, tr b = tr C */
    double s2 = s * s;
    if (J >= 1.0) { /* eq. ksipNH / ksinNH, J >= 1 */
        for (int k = 0; k < 9; k++) S[k] = s2 * (Svol[k] + Siso[k]);
        *psi_plus = U + psibar;
        *psi_minus = 0.0;
    } else {
        for (int k = 0; k < 9; k++) S[k] = Svol[k] + s2 * Siso[k];
        *psi_plus = psibar;
        *psi_minus = U;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Symmetric eigen-decomposition by cyclic Jacobi rotations (FP64):    */
/* A = Q diag(w) Q^T, eigenvectors as the columns of Q (row-major).    */
/* ------------------------------------------------------------------ */
void orc_sym_eig3(const double *A, double *w, double *Q) {
    double a[9];
    memcpy(a, A, sizeof a);
    a[1] = a[3] = 0.5 * (A[1] + A[3]);
    a[2] = a[6] = 0.5 * (A[2] + A[6]);
    a[5] = a[7] = 0.5 * (A[5] + A[7]);
    m_eye(Q);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
        double dia = a[0] * a[0] + a[4] * a[4] + a[8] * a[8];
        if (off == 0.0 || off <= 1e-40 * dia) break;
        static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int r = 0; r < 3; r++) {
            int p = P[r][0], q = P[r][1];
            double apq = a[3 * p + q];
            if (apq == 0.0) continue;
            /* the rotation J(p, q, theta) that zeroes a_pq: tan(2 theta) = 2 a_pq / (a_qq - a_pp) */
            double theta = (a[3 * q + q] - a[3 * p + p]) / (2.0 * apq);
            double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
            double J[9];
            m_eye(J);
            J[3 * p + p] = cs;
            J[3 * q + q] = cs;
            J[3 * p + q] = sn;
            J[3 * q + p] = -sn;
            double Jt[9], tmp[9];
            m_tr(J, Jt);
            m_mul(Jt, a, tmp);
            m_mul(tmp, J, a); /* a <- J^T a J */
            a[3 * p + q] = a[3 * q + p] = 0.0;
            m_mul(Q, J, tmp); /* Q <- Q J */
            memcpy(Q, tmp, sizeof tmp);
        }
    }
    for (int k = 0; k < 3; k++) w[k] = a[4 * k];
}

/* ------------------------------------------------------------------ */
/* St. Venant-Kirchhoff stress with the spectral split of the          */
/* Green-Lagrange strain (Sec. 2.3.1, eq. elasEnergyP, elasEnergyN,    */
/* GLstratinP, GLstratinN, 2PK_SVK1, 2PK_SVK2):                         */
/*   E = (F^T F - I) / 2 = Q diag(lambda_a) Q^T,                        */
/*   E+- = Q diag({lambda_a}+-) Q^T,                                     */
/*   psi+- = lambda/2 {tr E}+-^2 + mu tr(E+- E+-),                       */
/*   S+- = lambda {tr E}+- I + 2 mu E+-,   S = s^2 S+ + S-.              */
/* ------------------------------------------------------------------ */
int orc_svk_stress(const double *F, double s, const orc_material *m, double *S, double *psi_plus,
                   double *psi_minus) {
    double lam, mu, kap;
    lame(m, &lam, &mu, &kap);
    double Ft[9], C[9], E[9], w[3], Q[9];
    m_tr(F, Ft);
    m_mul(Ft, F, C);
    for (int k = 0; k < 9; k++) E[k] = 0.5 * (C[k] - (k % 4 == 0 ? 1.0 : 0.0));
    orc_sym_eig3(E, w, Q);
    double Ep[9] = {0}, Em[9] = {0};
    double sp2 = 0.0, sm2 = 0.0;
    for (int a = 0; a < 3; a++) {
        double lp = w[a] > 0.0 ? w[a] : 0.0, lm = w[a] < 0.0 ? w[a] : 0.0;
        sp2 += lp * lp;
        sm2 += lm * lm;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double qq = Q[3 * i + a] * Q[3 * j + a];
                Ep[3 * i + j] += lp * qq;
                Em[3 * i + j] += lm * qq;
            }
    }
    double trE = m_trace(E);
    double trp = trE > 0.0 ? trE : 0.0, trm = trE < 0.0 ? trE : 0.0;
    *psi_plus = 0.5 * lam * trp * trp + mu * sp2;
    *psi_minus = 0.5 * lam * trm * trm + mu * sm2;
    double s2 = s * s;
    for (int k = 0; k < 9; k++) {
        double id = (k % 4 == 0) ? 1.0 : 0.0;
        S[k] = s2 * (lam * trp * id + 2.0 * mu * Ep[k]) + (lam * trm * id + 2.0 * mu * Em[k]);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Finite-strain J2 plasticity, F_p stored (Sec. 2.3.3).               */
/* ------------------------------------------------------------------ */
static double j2_sigma_eq(const double *Ce, double J, double mu) {
    /* M_dev = mu dev(J^-2/3 C_e), sigma_eq = sqrt(3/2 M_dev : M_dev) */
    double Cb[9], Md[9];
    for (int k = 0; k < 9; k++) Cb[k] = pow(J, -2.0 / 3.0) * Ce[k];
    m_dev(Cb, Md);
    m_scale(Md, mu);
    return sqrt(1.5 * m_ddot(Md, Md));
}
/* C_e = F_p^-T C F_p^-1 */
static int j2_Ce(const double *Fp, const double *C, double *Ce) {
    double Fpi[9], FpiT[9];
    if (m_inv(Fp, Fpi) != 0) return -1;
    m_tr(Fpi, FpiT);
    m_mul(FpiT, C, Ce);
    m_mul(Ce, Fpi, Ce);
    return 0;
}
/* candidate F_p(dgamma) = det(F*)^-1/3 F*, F* = exp(dgamma N) F_p^n (eq. expmap, eq. Fp_iso_proj) */
static void j2_Fp_candidate(const double *N, const double *Fpn, double dg, double *Fp) {
    double A[9], E[9];
    for (int k = 0; k < 9; k++) A[k] = dg * N[k];
    orc_expm(A, E);
    m_mul(E, Fpn, Fp);
    double d = m_det(Fp);
    m_scale(Fp, pow(d, -1.0 / 3.0));
}
/* residual of eq. J2_residual */
static double j2_residual(const double *N, const double *Fpn, const double *C, double J, double mu,
                          double sy0, double Hh, double epn, double dg) {
    double Fp[9], Ce[9];
    j2_Fp_candidate(N, Fpn, dg, Fp);
    if (j2_Ce(Fp, C, Ce) != 0) return NAN;
    return j2_sigma_eq(Ce, J, mu) - (sy0 + Hh * (epn + dg));
}

/*
 * One return-mapping update.  Inputs F (3x3), F_p^n, eps_p^n.  Outputs
 * F_p^{n+1}, eps_p^{n+1}, S, the increment dgamma and the iteration count.
 * Returns 0, or 1 if the bracket or the Illinois iteration did not converge.
 * reading (tolerances, not given in the paper): bracket epsilon
 * 1e-12 sigma_y/mu, at most 60 doublings, stop at |r| <= 1e-10 sigma_y0 or
 * |R - L| <= 1e-14 R, at most 100 Illinois iterations.
 * reading (the bracket): r(dgamma) of eq. J2_residual falls from r(0) = f > 0
 * to about -sigma_y where the frozen flow has removed the deviatoric stress and
 * rises again beyond, so it has a root below that minimum.  A doubling step that
 * lands past the minimum with r still positive (r rose) has stepped over the
 * negative interval; a golden-section search for the minimum of r between the
 * last two points then stops at the first point with r <= 0 (and the doubling
 * goes on if it finds none: near r = 0 rounding alone can make r rise).
 */
int orc_j2_update(const double *F, const double *Fpn, double epn, const orc_material *m, double *Fp_out,
                  double *ep_out, double *S, double *dgamma, int *iters) {
    double lam, mu, kap;
    lame(m, &lam, &mu, &kap);
    double Hh = m->H_hard, sy0 = m->sigma_y0;
    double Ft[9], C[9], Ci[9];
    m_tr(F, Ft);
    m_mul(Ft, F, C);
    double J = m_det(F);
    int status = 0;
    *iters = 0;
    *dgamma = 0.0;
    if (!(J > 0.0) || m_inv(C, Ci) != 0) return -1;
    /* trial state: F_p frozen */
    double Ce[9], Cb[9], Md[9];
    if (j2_Ce(Fpn, C, Ce) != 0) return -1;
    for (int k = 0; k < 9; k++) Cb[k] = pow(J, -2.0 / 3.0) * Ce[k];
    m_dev(Cb, Md);
    m_scale(Md, mu);
    double sig_tr = sqrt(1.5 * m_ddot(Md, Md));
    double syn = sy0 + Hh * epn;
    double f = sig_tr - syn;
    double Fp[9];
    memcpy(Fp, Fpn, sizeof Fp);
    double dg = 0.0;
    if (f > 0.0) {
        double N[9];
        for (int k = 0; k < 9; k++) N[k] = 1.5 / sig_tr * Md[k]; /* trial flow direction */
        double L = 0.0, rL = f;
        double eps_b = 1e-12 * syn / mu;
        double R = (sig_tr - syn) / (3.0 * mu + Hh);
        if (R < eps_b) R = eps_b;
        double rR = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, R);
        double Rp = 0.0; /* the point before R (r(0) = f > 0) */
        int nd = 0;
        while (rR > 0.0 && nd < 60) { /* double the upper end until r(R) <= 0 */
            double Rn = 2.0 * R;
            double rn = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, Rn);
            nd++;
            if (rn > 0.0 && rn >= rR) {
                /* past the minimum of r without a sign change: golden-section search on [Rp, Rn] */
                const double g = 0.6180339887498949;
                double a = Rp, b = Rn;
                double c1 = b - g * (b - a), d1 = a + g * (b - a);
                double rc = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, c1);
                double rd = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, d1);
                int found = 0;
                for (int k = 0; k < 80 && !found; k++) {
                    if (rc <= 0.0) { R = c1; rR = rc; found = 1; break; }
                    if (rd <= 0.0) { R = d1; rR = rd; found = 1; break; }
                    if (rc < rd) {
                        b = d1; d1 = c1; rd = rc;
                        c1 = b - g * (b - a);
                        rc = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, c1);
                    } else {
                        a = c1; c1 = d1; rc = rd;
                        d1 = a + g * (b - a);
                        rd = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, d1);
                    }
                }
                if (found) break;
                /* no point below zero (r rose only by rounding near r = 0): keep doubling */
            }
            Rp = R;
            R = Rn;
            rR = rn;
        }
        if (!(rR <= 0.0)) status = 1;
        double x = R, rx = rR;
        if (rR != 0.0 && status == 0) {
            int it;
            for (it = 0; it < 100; it++) {
                x = R - rR * (R - L) / (rR - rL); /* false-position step */
                rx = j2_residual(N, Fpn, C, J, mu, sy0, Hh, epn, x);
                if (fabs(rx) <= 1e-10 * sy0 || fabs(R - L) <= 1e-14 * fabs(R)) break;
                if ((rx < 0.0 && rR > 0.0) || (rx > 0.0 && rR < 0.0)) {
                    L = R; /* bracket flips: old R becomes the other end */
                    rL = rR;
                } else {
                    rL = 0.5 * rL; /* Illinois: halve the stale end's residual */
                }
                R = x;
                rR = rx;
            }
            *iters = it + 1;
            if (it == 100) status = 1;
        }
        dg = x;
        j2_Fp_candidate(N, Fpn, dg, Fp); /* F_p^{n+1} */
    }
    /* stress assembly: S = F_p^-1 [C_e^-1 M_dev] F_p^-T + kappa/2 (J^2 - 1) C^-1 */
    double Fpi[9], FpiT[9], Cei[9], Se[9], Siso[9];
    j2_Ce(Fp, C, Ce);
    for (int k = 0; k < 9; k++) Cb[k] = pow(J, -2.0 / 3.0) * Ce[k];
    m_dev(Cb, Md);
    m_scale(Md, mu);
    m_inv(Ce, Cei);
    m_mul(Cei, Md, Se);
    m_inv(Fp, Fpi);
    m_tr(Fpi, FpiT);
    m_mul(Fpi, Se, Siso);
    m_mul(Siso, FpiT, Siso);
    for (int k = 0; k < 9; k++) S[k] = Siso[k] + 0.5 * kap * (J * J - 1.0) * Ci[k];
    memcpy(Fp_out, Fp, sizeof Fp);
    *ep_out = epn + dg;
    *dgamma = dg;
    return status;
}

/* strain energy of the J2 model: psi_vol(J) + psi_iso(Cbar_e) (Sec. 2.3.3) */
static double j2_energy(const double *F, const double *Fp, const orc_material *m) {
    double lam, mu, kap;
    lame(m, &lam, &mu, &kap);
    double Ft[9], C[9], Ce[9];
    m_tr(F, Ft);
    m_mul(Ft, F, C);
    double J = m_det(F);
    if (j2_Ce(Fp, C, Ce) != 0 || !(J > 0.0)) return NAN;
    return 0.25 * kap * (J * J - 1.0 - 2.0 * log(J)) + 0.5 * mu * (pow(J, -2.0 / 3.0) * m_trace(Ce) - 3.0);
}

/* ------------------------------------------------------------------ */
/* context                                                             */
/* ------------------------------------------------------------------ */
static void *xcalloc(size_t n, size_t sz) { return n ? calloc(n, sz) : calloc(1, sz); }

orc_ctx *orc_create(const orc_params *p) {
    if (!p || (p->dim != 2 && p->dim != 3) || !(p->h > 0.0) || !(p->support > 0.0) || p->integrator < 0 ||
        p->integrator > 2)
        return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    return c;
}

static void free_particles(orc_ctx *c) {
    free(c->rest); free(c->accc); free(c->kfric);
    free(c->X0); free(c->vol); free(c->u); free(c->v); free(c->acc); free(c->s); free(c->sdot);
    free(c->aext); free(c->wext);
    free(c->sdd); free(c->lap); free(c->pf_b); free(c->pf_k); free(c->pf_g); free(c->Hh); free(c->Fp); free(c->ep); free(c->mid); free(c->spec); free(c->F);
    free(c->P); free(c->L); free(c->status); free(c->row_ptr); free(c->col); free(c->perm);
    free(c->t); free(c->dt); free(c->vmax); free(c->amax); free(c->cmax);
    for (int b = 0; b < c->nbc; b++) {
        free(c->bc[b].mask);
        for (int ph = 0; ph < 2; ph++) {
            free(c->bc[b].exval[ph]);
            free(c->bc[b].exskip[ph]);
        }
    }
    c->nbc = 0;
}

void orc_destroy(orc_ctx *c) {
    if (!c) return;
    free_particles(c);
    free(c->mat);
    free(c);
}

int orc_set_materials(orc_ctx *c, int n, const orc_material *m) {
    if (!c || n <= 0 || !m) return ORC_ERR_ARG;
    for (int i = 0; i < n; i++) {
        if (!(m[i].E > 0.0) || !(m[i].nu > -1.0 && m[i].nu < 0.5) || !(m[i].rho > 0.0)) return ORC_ERR_ARG;
        if (m[i].model != ORC_MODEL_SVK && m[i].model != ORC_MODEL_NH && m[i].model != ORC_MODEL_J2) return ORC_ERR_ARG;
    }
    free(c->mat);
    c->mat = (orc_material *)malloc(sizeof(orc_material) * n);
    memcpy(c->mat, m, sizeof(orc_material) * n);
    /* Sec. 3.3.1: fracture is disabled when J2 plasticity is selected */
    for (int i = 0; i < n; i++)
        if (c->mat[i].model == ORC_MODEL_J2) c->mat[i].fracture = 0;
    c->nmat = n;
    return ORC_OK;
}

int orc_create_particles(orc_ctx *c, int64_t n, const double *X0, const double *vol, const double *v0,
                         const int32_t *material_id, const int32_t *specimen_id) {
    if (!c || n <= 0 || !X0 || !vol || !material_id || c->nmat <= 0) return ORC_ERR_ARG;
    free_particles(c);
    int d = c->p.dim;
    c->n = n;
    c->X0 = xcalloc(n * 3, sizeof(double));
    c->vol = xcalloc(n, sizeof(double));
    c->u = xcalloc(n * 3, sizeof(double));
    c->v = xcalloc(n * 3, sizeof(double));
    c->acc = xcalloc(n * 3, sizeof(double));
    c->aext = xcalloc(n * 3, sizeof(double));
    c->wext = xcalloc(n, sizeof(double));
    c->s = xcalloc(n, sizeof(double));
    c->sdot = xcalloc(n, sizeof(double));
    c->sdd = xcalloc(n, sizeof(double));
    c->lap = xcalloc(n, sizeof(double));
    c->pf_b = xcalloc(n, sizeof(double));
    c->pf_k = xcalloc(n, sizeof(double));
    c->pf_g = xcalloc(n, sizeof(double));
    c->Hh = xcalloc(n, sizeof(double));
    c->Fp = xcalloc(n * 9, sizeof(double));
    c->ep = xcalloc(n, sizeof(double));
    c->mid = xcalloc(n, sizeof(int32_t));
    c->spec = xcalloc(n, sizeof(int32_t));
    c->F = xcalloc(n * 9, sizeof(double));
    c->P = xcalloc(n * 9, sizeof(double));
    c->L = xcalloc(n * 9, sizeof(double));
    c->status = xcalloc(n, sizeof(int32_t));
    if (!c->X0 || !c->Fp || !c->L) return ORC_ERR_OOM;
    int nspec = 1;
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < d; k++) c->X0[3 * i + k] = X0[d * i + k];
        c->vol[i] = vol[i];
        if (v0)
            for (int k = 0; k < d; k++) c->v[3 * i + k] = v0[d * i + k];
        if (material_id[i] < 0 || material_id[i] >= c->nmat || !(vol[i] > 0.0)) return ORC_ERR_ARG;
        c->mid[i] = material_id[i];
        c->spec[i] = specimen_id ? specimen_id[i] : 0;
        if (c->spec[i] < 0) return ORC_ERR_ARG;
        if (c->spec[i] + 1 > nspec) nspec = c->spec[i] + 1;
        c->s[i] = 1.0; /* intact material, s = 1 (Sec. 2.2) */
        m_eye(&c->Fp[9 * i]);
    }
    c->nspec = nspec;
    c->t = xcalloc(nspec, sizeof(double));
    c->dt = xcalloc(nspec, sizeof(double));
    c->vmax = xcalloc(nspec, sizeof(double));
    c->amax = xcalloc(nspec, sizeof(double));
    c->cmax = xcalloc(nspec, sizeof(double));
    c->built = 0;
    c->step = 0;
    c->noconv = 0;
    return ORC_OK;
}

int orc_add_bc(orc_ctx *c, const uint8_t *mask, int kind, int comp_mask, const double *value, double t_start,
               double t_end, double ramp, double area) {
    if (!c || !mask || !value || c->n <= 0 || c->nbc >= ORC_MAX_BC || kind < 0 || kind > 4) return ORC_ERR_ARG;
    /* a phase-field bound acts on s (component 0) with a value in [0, 1] */
    if (kind == ORC_BC_PHASE_BOUND && (!(comp_mask & 1) || !(value[0] >= 0.0 && value[0] <= 1.0)))
        return ORC_ERR_ARG;
    orc_bc *b = &c->bc[c->nbc];
    memset(b, 0, sizeof *b);
    b->kind = kind;
    b->comp_mask = comp_mask;
    memcpy(b->value, value, 3 * sizeof(double));
    b->t_start = t_start;
    b->t_end = t_end;
    b->ramp = ramp;
    b->area = area;
    b->mask = (uint8_t *)malloc(c->n);
    memcpy(b->mask, mask, c->n);
    b->count = 0;
    for (int64_t i = 0; i < c->n; i++) b->count += mask[i] ? 1 : 0;
    c->nbc++;
    return ORC_OK;
}

/* Per-particle values of a boundary condition given by expressions (caller order, n x 3, and a skip
 * flag per value); phase 0 is used by the step's update, phase 1 by the Algorithm 2 predictor. */
int orc_set_bc_values(orc_ctx *c, int b, int phase, const double *val, const uint8_t *skip) {
    if (!c || b < 0 || b >= c->nbc || phase < 0 || phase > 1 || !val || !skip) return ORC_ERR_ARG;
    orc_bc *bc = &c->bc[b];
    if (!bc->exval[phase]) {
        bc->exval[phase] = (double *)malloc(sizeof(double) * 3 * c->n);
        bc->exskip[phase] = (uint8_t *)malloc(3 * c->n);
    }
    memcpy(bc->exval[phase], val, sizeof(double) * 3 * c->n);
    memcpy(bc->exskip[phase], skip, 3 * c->n);
    return ORC_OK;
}

int orc_add_notch(orc_ctx *c, const double *quad) {
    if (!c || !quad || c->nnotch >= ORC_MAX_NOTCH) return ORC_ERR_ARG;
    for (int k = 0; k < 12; k++)
        if (!isfinite(quad[k])) return ORC_ERR_ARG;
    memcpy(c->notch[c->nnotch], quad, 12 * sizeof(double));
    c->nnotch++;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* reference configuration: neighbours, notch cut, cell sort           */
/* ------------------------------------------------------------------ */
/* r0^2 summed in the fixed order ((dx dx + dy dy) + dz dz), no FMA. */
static double ref_r2(const orc_ctx *c, int64_t i, int64_t j) {
    const double *a = &c->X0[3 * i], *b = &c->X0[3 * j];
    double dx = b[0] - a[0], dy = b[1] - a[1], r2 = dx * dx + dy * dy;
    if (c->p.dim == 3) {
        double dz = b[2] - a[2];
        r2 = r2 + dz * dz;
    }
    return r2;
}

/* 2D orientation of p w.r.t. the directed line a->b */
static double orient2(const double *a, const double *b, const double *p) {
    double t1 = (b[0] - a[0]) * (p[1] - a[1]);
    double t2 = (b[1] - a[1]) * (p[0] - a[0]);
    return t1 - t2;
}
/* 3D orientation: det[b - a, c - a, d - a] */
static double orient3(const double *a, const double *b, const double *c, const double *d) {
    double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
    double vx = c[0] - a[0], vy = c[1] - a[1], vz = c[2] - a[2];
    double wx = d[0] - a[0], wy = d[1] - a[1], wz = d[2] - a[2];
    double c1 = vy * wz - vz * wy;
    double c2 = vz * wx - vx * wz;
    double c3 = vx * wy - vy * wx;
    return (ux * c1 + uy * c2) + uz * c3;
}
static int opposite(double a, double b) { return (a > 0.0 && b < 0.0) || (a < 0.0 && b > 0.0); }

/* Sec. 3.3.1 (pre-existing notch).  reading: a bond i-j is removed when the
 * reference segment X_i X_j crosses the notch strictly inside it, by a
 * relative margin of 1e-9 (a crossing on the notch's rim, e.g. exactly at
 * its tip, keeps the bond).  2D uses the segment p1-p2 (x, y); 3D uses the
 * planar convex quad p1..p4. */
#define NOTCH_MARGIN 1e-9
static int notch_cuts(const orc_ctx *c, const double *P, const double *Q) {
    for (int k = 0; k < c->nnotch; k++) {
        const double *q = c->notch[k];
        if (c->p.dim == 2) {
            double A[2] = {q[0], q[1]}, B[2] = {q[3], q[4]};
            if (!opposite(orient2(A, B, P), orient2(A, B, Q))) continue;
            double o3 = orient2(P, Q, A), o4 = orient2(P, Q, B);
            if (!opposite(o3, o4)) continue;
            double t = o3 / (o3 - o4); /* crossing point along the notch, in (0, 1) */
            if (t > NOTCH_MARGIN && t < 1.0 - NOTCH_MARGIN) return 1;
        } else {
            const double *p1 = q, *p2 = q + 3, *p3 = q + 6, *p4 = q + 9;
            if (!opposite(orient3(p1, p2, p3, P), orient3(p1, p2, p3, Q))) continue;
            double e1 = orient3(P, Q, p1, p2), e2 = orient3(P, Q, p2, p3);
            double e3 = orient3(P, Q, p3, p4), e4 = orient3(P, Q, p4, p1);
            int pos = e1 > 0.0 && e2 > 0.0 && e3 > 0.0 && e4 > 0.0;
            int neg = e1 < 0.0 && e2 < 0.0 && e3 < 0.0 && e4 < 0.0;
            if (!pos && !neg) continue;
            double sum = ((e1 + e2) + e3) + e4;
            if (e1 / sum > NOTCH_MARGIN && e2 / sum > NOTCH_MARGIN && e3 / sum > NOTCH_MARGIN &&
                e4 / sum > NOTCH_MARGIN)
                return 1;
        }
    }
    return 0;
}

static int is_neighbour(const orc_ctx *c, int64_t i, int64_t j, double R2) {
    if (i == j || c->spec[i] != c->spec[j]) return 0;
    if (!(ref_r2(c, i, j) < R2)) return 0;
    /* the segment is always taken from the lower to the higher id, so the
     * relation stays symmetric whatever the rounding */
    int64_t a = i < j ? i : j, b = i < j ? j : i;
    if (c->nnotch && notch_cuts(c, &c->X0[3 * a], &c->X0[3 * b])) return 0;
    return 1;
}

typedef struct { int64_t key, id; } keyid;
static int cmp_keyid(const void *a, const void *b) {
    const keyid *x = (const keyid *)a, *y = (const keyid *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* Cells of size R/3 centred on the planes X = Xmin + k R/3, cell coordinate
 * floor((X - Xmin) / (R/3) + 1/2).  A pair with r0 < R is at most 3 cells
 * apart per axis; the search covers 4 to absorb the rounding of the cell
 * coordinate.  reading (the paper only says that particles are sorted by
 * cell): cells this fine hold about one particle of a lattice of spacing R/3,
 * so the cell-sorted order is the lattice order. */
#define CELL_RANGE 4
static void cell_setup(orc_ctx *c) {
    double R = c->p.support * c->p.h;
    c->cell_size = R / 3.0;
    for (int k = 0; k < 3; k++) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = 0; i < c->n; i++) {
            double x = c->X0[3 * i + k];
            if (x < mn) mn = x;
            if (x > mx) mx = x;
        }
        if (k >= c->p.dim) { mn = 0.0; mx = 0.0; }
        c->xmin[k] = mn;
        c->ncell[k] = (int64_t)floor((mx - mn) / c->cell_size + 0.5) + 1;
    }
}
static void cell_of(const orc_ctx *c, int64_t i, int64_t *cc) {
    for (int k = 0; k < 3; k++)
        cc[k] = k < c->p.dim ? (int64_t)floor((c->X0[3 * i + k] - c->xmin[k]) / c->cell_size + 0.5) : 0;
}
static int64_t cell_key(const orc_ctx *c, int64_t spec, const int64_t *cc) {
    return ((spec * c->ncell[2] + cc[2]) * c->ncell[1] + cc[1]) * c->ncell[0] + cc[0];
}

/* method 0: brute force O(N^2); method 1: cell list.  Rows are in the
 * caller's order, each row ascending by neighbour id. */
int orc_build_neighbours(orc_ctx *c, int method) {
    if (!c || c->n <= 0) return ORC_ERR_STATE;
    int64_t n = c->n;
    double R = c->p.support * c->p.h, R2 = R * R;
    cell_setup(c);
    /* cell-sorted permutation: stable sort by (cell key, id) */
    keyid *ki = (keyid *)malloc(sizeof(keyid) * n);
    for (int64_t i = 0; i < n; i++) {
        int64_t cc[3];
        cell_of(c, i, cc);
        ki[i].key = cell_key(c, c->spec[i], cc);
        ki[i].id = i;
    }
    qsort(ki, n, sizeof(keyid), cmp_keyid);
    free(c->perm);
    c->perm = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; i++) c->perm[i] = ki[i].id;

    int64_t *cnt = (int64_t *)calloc(n + 1, sizeof(int64_t));
    int32_t **rows = (int32_t **)calloc(n, sizeof(int32_t *));
    /* per-cell ranges of the sorted order, for the cell method */
    int64_t nk = ki[n - 1].key + 1;
    int64_t *cstart = NULL, *cend = NULL;
    if (method == 1) {
        cstart = (int64_t *)malloc(sizeof(int64_t) * nk);
        cend = (int64_t *)malloc(sizeof(int64_t) * nk);
        for (int64_t k = 0; k < nk; k++) cstart[k] = cend[k] = 0;
        for (int64_t s = 0; s < n; s++) {
            if (s == 0 || ki[s].key != ki[s - 1].key) cstart[ki[s].key] = s;
            cend[ki[s].key] = s + 1;
        }
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t cap = 64, m = 0;
        int32_t *row = (int32_t *)malloc(sizeof(int32_t) * cap);
        if (method == 0) {
            for (int64_t j = 0; j < n; j++) {
                if (!is_neighbour(c, i, j, R2)) continue;
                if (m == cap) { cap *= 2; row = (int32_t *)realloc(row, sizeof(int32_t) * cap); }
                row[m++] = (int32_t)j;
            }
        } else {
            int64_t cc[3];
            cell_of(c, i, cc);
            int dz0 = c->p.dim == 3 ? -CELL_RANGE : 0, dz1 = c->p.dim == 3 ? CELL_RANGE : 0;
            for (int dz = dz0; dz <= dz1; dz++)
                for (int dy = -CELL_RANGE; dy <= CELL_RANGE; dy++)
                    for (int dx = -CELL_RANGE; dx <= CELL_RANGE; dx++) {
                        int64_t q[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                        if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= c->ncell[0] || q[1] >= c->ncell[1] ||
                            q[2] >= c->ncell[2])
                            continue;
                        int64_t key = cell_key(c, c->spec[i], q);
                        if (key >= nk) continue;
                        for (int64_t s = cstart[key]; s < cend[key]; s++) {
                            int64_t j = ki[s].id;
                            if (!is_neighbour(c, i, j, R2)) continue;
                            if (m == cap) { cap *= 2; row = (int32_t *)realloc(row, sizeof(int32_t) * cap); }
                            row[m++] = (int32_t)j;
                        }
                    }
            /* ascending by id (insertion sort: rows are short) */
            for (int64_t a = 1; a < m; a++) {
                int32_t x = row[a];
                int64_t b = a - 1;
                while (b >= 0 && row[b] > x) { row[b + 1] = row[b]; b--; }
                row[b + 1] = x;
            }
        }
        rows[i] = row;
        cnt[i] = m;
    }
    free(cstart);
    free(cend);
    free(ki);
    free(c->row_ptr);
    free(c->col);
    c->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    c->row_ptr[0] = 0;
    for (int64_t i = 0; i < n; i++) c->row_ptr[i + 1] = c->row_ptr[i] + cnt[i];
    c->col = (int32_t *)malloc(sizeof(int32_t) * (c->row_ptr[n] ? c->row_ptr[n] : 1));
    for (int64_t i = 0; i < n; i++) {
        memcpy(&c->col[c->row_ptr[i]], rows[i], sizeof(int32_t) * cnt[i]);
        free(rows[i]);
    }
    free(rows);
    free(cnt);

    /* two particles of one specimen at the same reference position are an input error */
    for (int64_t i = 0; i < n; i++)
        for (int64_t q = c->row_ptr[i]; q < c->row_ptr[i + 1]; q++)
            if (ref_r2(c, i, c->col[q]) == 0.0) return ORC_ERR_ARG;

    /* correction tensor L_i = -(sum_j gradW_ij (x) r0_ij V0j)^-1 (Sec. 2.4) */
    int d = c->p.dim;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < n; i++) {
        double M[9] = {0};
        for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; e++) {
            int64_t j = c->col[e];
            double r0[3] = {0, 0, 0}, g[3];
            for (int k = 0; k < d; k++) r0[k] = c->X0[3 * i + k] - c->X0[3 * j + k];
            double r = sqrt(ref_r2(c, i, j));
            kernel_grad(c, r0, r, g);
            for (int a = 0; a < d; a++)
                for (int b = 0; b < d; b++) M[3 * a + b] += g[a] * r0[b] * c->vol[j];
        }
        double *L = &c->L[9 * i];
        memset(L, 0, 9 * sizeof(double));
        if (d == 2) {
            double det = M[0] * M[4] - M[1] * M[3];
            double scale = fabs(M[0]) + fabs(M[4]);
            if (!(fabs(det) > 1e-12 * scale * scale)) { bad++; continue; }
            L[0] = -M[4] / det;
            L[1] = M[1] / det;
            L[3] = M[3] / det;
            L[4] = -M[0] / det;
        } else {
            double Mi[9];
            double scale = fabs(M[0]) + fabs(M[4]) + fabs(M[8]);
            double det = m_det(M);
            if (!(fabs(det) > 1e-12 * scale * scale * scale) || m_inv(M, Mi) != 0) { bad++; continue; }
            for (int k = 0; k < 9; k++) L[k] = -Mi[k];
        }
    }
    if (bad) return ORC_ERR_SINGULAR;
    /* time-step constants per specimen */
    for (int s = 0; s < c->nspec; s++) c->cmax[s] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double cs = orc_sound_speed(&c->mat[c->mid[i]]);
        if (cs > c->cmax[c->spec[i]]) c->cmax[c->spec[i]] = cs;
    }
    if (c->contact) { /* bodies in contact share one clock: the largest sound speed of all */
        double cm = 0.0;
        for (int s = 0; s < c->nspec; s++) cm = c->cmax[s] > cm ? c->cmax[s] : cm;
        for (int s = 0; s < c->nspec; s++) c->cmax[s] = cm;
    }
    for (int s = 0; s < c->nspec; s++) {
        c->t[s] = 0.0;
        c->vmax[s] = 0.0;
        c->amax[s] = 0.0;
    }
    for (int64_t i = 0; i < n; i++) {
        double vv = 0.0;
        for (int k = 0; k < 3; k++) vv += c->v[3 * i + k] * c->v[3 * i + k];
        vv = sqrt(vv);
        if (vv > c->vmax[c->spec[i]]) c->vmax[c->spec[i]] = vv;
    }
    c->built = 1;
    return ORC_OK;
}

int64_t orc_nnz(const orc_ctx *c) { return (c && c->row_ptr) ? c->row_ptr[c->n] : -1; }

int orc_neighbours(const orc_ctx *c, int64_t *row_ptr, int32_t *col, int64_t cap) {
    if (!c || !c->row_ptr) return ORC_ERR_STATE;
    if (cap < c->row_ptr[c->n]) return ORC_ERR_ARG;
    memcpy(row_ptr, c->row_ptr, sizeof(int64_t) * (c->n + 1));
    memcpy(col, c->col, sizeof(int32_t) * c->row_ptr[c->n]);
    return ORC_OK;
}

int orc_perm(const orc_ctx *c, int64_t *perm) {
    if (!c || !c->perm) return ORC_ERR_STATE;
    memcpy(perm, c->perm, sizeof(int64_t) * c->n);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* per-step pieces                                                     */
/* ------------------------------------------------------------------ */
/* corrected gradient Ltilde = L_i . gradW_ij (in-plane components) */
static void corrected_grad(const orc_ctx *c, int64_t i, int64_t j, double *gt, double *graw, double *r0,
                           double *r) {
    int d = c->p.dim;
    r0[0] = r0[1] = r0[2] = 0.0;
    for (int k = 0; k < d; k++) r0[k] = c->X0[3 * i + k] - c->X0[3 * j + k];
    *r = sqrt(ref_r2(c, i, j));
    kernel_grad(c, r0, *r, graw);
    const double *L = &c->L[9 * i];
    for (int a = 0; a < 3; a++) {
        gt[a] = 0.0;
        if (a < d)
            for (int b = 0; b < d; b++) gt[a] += L[3 * a + b] * graw[b];
    }
}

static int is_fracture(const orc_ctx *c, int64_t i) {
    const orc_material *m = &c->mat[c->mid[i]];
    return m->fracture && m->model != ORC_MODEL_J2;
}

/* eq. deformGradTLSPH with V0j in place of m0j / rho0i (identical for a
 * single body; reading: V0j keeps first-order consistency at material
 * interfaces), soft-particle rule eq. defGrad_phase. */
static void deformation_gradient(const orc_ctx *c, const double *u, int64_t i, double *F) {
    int d = c->p.dim;
    m_eye(F);
    if (is_fracture(c, i) && c->s[i] <= c->mat[c->mid[i]].s_lim) return;
    for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; e++) {
        int64_t j = c->col[e];
        double gt[3], g[3], r0[3], r;
        corrected_grad(c, i, j, gt, g, r0, &r);
        for (int k = 0; k < d; k++)
            for (int q = 0; q < d; q++) F[3 * k + q] += c->vol[j] * (u[3 * j + k] - u[3 * i + k]) * gt[q];
    }
}

/* Evaluate F, the stress P, and (commit != 0) the state update of particle i. */
static void constitutive(orc_ctx *c, int64_t i, const double *F, int commit, double *P, double *psi,
                         double *Fp_new, double *ep_new) {
    const orc_material *m = &c->mat[c->mid[i]];
    double S[9];
    c->status[i] = 0;
    if (m->model == ORC_MODEL_NH || m->model == ORC_MODEL_SVK) {
        double s = is_fracture(c, i) ? c->s[i] : 1.0; /* degradation with s_n (Algorithm 1) */
        double pp, pm;
        int st = m->model == ORC_MODEL_NH ? orc_nh_stress(F, s, m, S, &pp, &pm) : orc_svk_stress(F, s, m, S, &pp, &pm);
        if (st != 0) {
            for (int k = 0; k < 9; k++) P[k] = NAN;
            c->status[i] = 2;
            return;
        }
        if (psi) *psi = s * s * pp + pm; /* eq. energy_density */
        if (commit && is_fracture(c, i) && pp > c->Hh[i]) c->Hh[i] = pp; /* eq. irreversibility */
    } else {
        double dg;
        int it;
        int st = orc_j2_update(F, &c->Fp[9 * i], c->ep[i], m, Fp_new, ep_new, S, &dg, &it);
        if (st != 0) c->status[i] = st < 0 ? 2 : 1;
        if (psi) *psi = j2_energy(F, Fp_new, m);
    }
    m_mul(F, S, P); /* P = F S */
}

static double bc_factor(const orc_bc *b, double t) {
    if (t < b->t_start) return -1.0;
    if (b->t_end >= 0.0 && t > b->t_end) return -1.0;
    if (b->ramp > 0.0) {
        double f = (t - b->t_start) / b->ramp;
        return f < 1.0 ? f : 1.0;
    }
    return 1.0;
}

/* ------------------------------------------------------------------ */
/* Contact between bodies (Algorithm 1 step 1, Algorithm 2 step 2;     */
/* <contcoeff>, <restcoef> of Sec. 3.3).  The paper takes its contact  */
/* model from its host framework without stating it; reading: a linear */
/* spring-dashpot normal force between particles of different bodies   */
/* closer than the contact distance dc (the particle spacing):          */
/*   delta = dc - r, n = (x_i - x_j) / r, k = kc E* dc^(dim - 2),        */
/*   1/E* = (1 - nu_i^2)/E_i + (1 - nu_j^2)/E_j,                          */
/*   m* = m_i m_j / (m_i + m_j), e = (e_i + e_j) / 2,                     */
/*   zeta = -ln e / sqrt(pi^2 + ln^2 e), c = 2 zeta sqrt(k m*),           */
/*   F_i = (k delta - c (v_i - v_j).n) n,                                 */
/* for which a head-on pair leaves with relative speed e times the one  */
/* it came with (the damped oscillator's half period).                  */
/* Friction (<kfric>, also unstated; reading): Coulomb's law, the       */
/* tangential force opposing the sliding velocity v_t = v_ij - v_n n     */
/* with magnitude mu max(f_n, 0) while sliding, regularised near rest    */
/* by a viscous bound c_t |v_t| with c_t = 2 sqrt(k m*) (the critical    */
/* damping of the normal spring), so that an explicit step does not     */
/* chatter around v_t = 0:                                              */
/*   F_i = f_n n - min(mu max(f_n, 0), c_t |v_t|, m* |v_t| / dt) v_t/|v_t|,*/
/* mu = (mu_i + mu_j) / 2.  The last bound (dt > 0: the step the force   */
/* acts over) lets friction at most stop the sliding in one explicit     */
/* step; it is below c_t |v_t| only when the normal spring's omega dt    */
/* exceeds 1/2, where c_t |v_t| alone would reverse v_t.                 */
/* ------------------------------------------------------------------ */
int orc_contact_force(int dim, double dc, double kc, const double *xi, const double *xj, const double *vi,
                      const double *vj, double mi, double mj, double cinv_i, double cinv_j, double ei, double ej,
                      double mu, double dt, double *F) {
    double d[3] = {0, 0, 0}, r2 = 0.0;
    F[0] = F[1] = F[2] = 0.0;
    for (int k = 0; k < dim; k++) {
        d[k] = xi[k] - xj[k];
        r2 += d[k] * d[k];
    }
    if (!(r2 < dc * dc) || r2 == 0.0) return 0;
    double r = sqrt(r2);
    double kn = kc * pow(dc, dim - 2) / (cinv_i + cinv_j);
    double ms = mi * mj / (mi + mj);
    double e = 0.5 * (ei + ej);
    double zeta = 0.0;
    if (e < 1.0) {
        double le = log(e);
        zeta = -le / sqrt(M_PI * M_PI + le * le);
    }
    double cd = 2.0 * zeta * sqrt(kn * ms);
    double vn = 0.0;
    for (int k = 0; k < dim; k++) vn += (vi[k] - vj[k]) * d[k] / r;
    double f = kn * (dc - r) - cd * vn;
    for (int k = 0; k < dim; k++) F[k] = f * d[k] / r;
    if (mu > 0.0 && f > 0.0) {
        double vt[3] = {0, 0, 0}, vt2 = 0.0;
        for (int k = 0; k < dim; k++) {
            vt[k] = (vi[k] - vj[k]) - vn * d[k] / r;
            vt2 += vt[k] * vt[k];
        }
        if (vt2 > 0.0) {
            double vtm = sqrt(vt2);
            double ft = fmin(mu * f, 2.0 * sqrt(kn * ms) * vtm);
            if (dt > 0.0) ft = fmin(ft, ms * vtm / dt);
            for (int k = 0; k < dim; k++) F[k] -= ft * vt[k] / vtm;
        }
    }
    return 1;
}

static double mat_cinv(const orc_material *m) { return (1.0 - m->nu * m->nu) / m->E; }

/* Contact accelerations of all particles from the current u and v (all pairs of different bodies). */
static void contact_accel(orc_ctx *c) {
    const int64_t n = c->n;
    const int d = c->p.dim;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double xi[3], a[3] = {0, 0, 0};
        for (int k = 0; k < 3; k++) xi[k] = c->X0[3 * i + k] + c->u[3 * i + k];
        const orc_material *mi = &c->mat[c->mid[i]];
        const double massi = mi->rho * c->vol[i];
        for (int64_t j = 0; j < n; j++) {
            if (c->spec[j] == c->spec[i]) continue;
            double xj[3], F[3];
            for (int k = 0; k < 3; k++) xj[k] = c->X0[3 * j + k] + c->u[3 * j + k];
            const orc_material *mj = &c->mat[c->mid[j]];
            const double mu = c->kfric ? 0.5 * (c->kfric[c->spec[i]] + c->kfric[c->spec[j]]) : 0.0;
            if (orc_contact_force(d, c->dc, c->kc, xi, xj, &c->v[3 * i], &c->v[3 * j], massi, mj->rho * c->vol[j],
                                  mat_cinv(mi), mat_cinv(mj), c->rest[c->spec[i]], c->rest[c->spec[j]], mu,
                                  c->dt[c->spec[i]], F))
                for (int k = 0; k < d; k++) a[k] += F[k] / massi;
        }
        for (int k = 0; k < 3; k++) c->accc[3 * i + k] = a[k];
    }
}

/* Bodies = the specimens: contact acts between particles of different specimens, which then share one
 * clock.  kc = <contcoeff>, dc = contact distance, rest[nspec] = <restcoef> per body. */
int orc_set_contact(orc_ctx *c, double kc, double dc, int nspec, const double *rest) {
    if (!c || c->n <= 0 || nspec != c->nspec || !rest || !(kc > 0.0) || !(dc > 0.0)) return ORC_ERR_ARG;
    if (c->p.dt_mode == ORC_DT_ADAPTIVE) return ORC_ERR_ARG;
    for (int s = 0; s < nspec; s++)
        if (!(rest[s] > 0.0 && rest[s] <= 1.0)) return ORC_ERR_ARG;
    free(c->rest);
    c->rest = (double *)malloc(sizeof(double) * nspec);
    memcpy(c->rest, rest, sizeof(double) * nspec);
    free(c->accc);
    c->accc = (double *)calloc(3 * c->n, sizeof(double));
    c->kc = kc;
    c->dc = dc;
    c->contact = 1;
    c->built = 0;
    return ORC_OK;
}

/* Friction coefficients <kfric> per body (after orc_set_contact; all 0 = no friction). */
int orc_set_contact_friction(orc_ctx *c, int nspec, const double *kfric) {
    if (!c || !c->contact || nspec != c->nspec || !kfric) return ORC_ERR_ARG;
    for (int s = 0; s < nspec; s++)
        if (!(kfric[s] >= 0.0 && isfinite(kfric[s]))) return ORC_ERR_ARG;
    free(c->kfric);
    c->kfric = (double *)malloc(sizeof(double) * nspec);
    memcpy(c->kfric, kfric, sizeof(double) * nspec);
    return ORC_OK;
}

/* Contact potential of the current state: sum over pairs of 1/2 k delta^2. */
double orc_contact_energy(const orc_ctx *c) {
    if (!c || !c->contact) return 0.0;
    double E = 0.0;
    for (int64_t i = 0; i < c->n; i++)
        for (int64_t j = i + 1; j < c->n; j++) {
            if (c->spec[j] == c->spec[i]) continue;
            double r2 = 0.0;
            for (int k = 0; k < c->p.dim; k++) {
                double dd = c->X0[3 * i + k] + c->u[3 * i + k] - c->X0[3 * j + k] - c->u[3 * j + k];
                r2 += dd * dd;
            }
            if (!(r2 < c->dc * c->dc)) continue;
            double kn = c->kc * pow(c->dc, c->p.dim - 2) / (mat_cinv(&c->mat[c->mid[i]]) + mat_cinv(&c->mat[c->mid[j]]));
            double dl = c->dc - sqrt(r2);
            E += 0.5 * kn * dl * dl;
        }
    return E;
}

/* The value a condition prescribes for component k of particle i (factor f = bc_factor >= 0): the
 * ramped constant, or the expression's value; returns 0 when the expression skips it. */
static int bc_value(const orc_bc *b, int phase, int64_t i, int k, double f, double *out) {
    if (b->exval[0]) {
        const int ph = b->exval[phase] ? phase : 0;
        if (b->exskip[ph][3 * i + k]) return 0;
        *out = b->exval[ph][3 * i + k];
        return 1;
    }
    *out = f * b->value[k];
    return 1;
}

/* Step sizes per specimen (eq. dt_criterion), from the state the next step starts from. */
static void step_sizes(orc_ctx *c) {
    for (int s = 0; s < c->nspec; s++) {
        double h = c->p.h;
        if (c->p.dt_mode == ORC_DT_FIXED) {
            c->dt[s] = c->p.fixed_dt;
        } else if (c->p.dt_mode == ORC_DT_CFL_STATIC) {
            c->dt[s] = c->p.cfl * h / c->cmax[s];
        } else {
            double dtv = h / (c->cmax[s] + c->vmax[s]);
            double dta = c->amax[s] > 0.0 ? sqrt(h / c->amax[s]) : INFINITY;
            c->dt[s] = c->p.cfl * (dtv < dta ? dtv : dta);
        }
    }
}

/* Sets the step sizes of the next step (orc_time then reports them), so that a caller can evaluate
 * time-dependent expressions for it. */
int orc_prepare_step(orc_ctx *c) {
    if (!c || !c->built) return ORC_ERR_STATE;
    step_sizes(c);
    return ORC_OK;
}

/* One step of Algorithm 1 (or 2) for all particles. */
static int one_step(orc_ctx *c) {
    int64_t n = c->n;
    int d = c->p.dim;
    step_sizes(c);
    /* Algorithm 2, predictor: the forces of this step act at the half level,
     *   u_{n+1/2} = u_n + dt/2 v_n,  v_{n+1/2} = v_n + dt/2 a_{n-1/2},  s_{n+1/2} = s_n + dt/2 sdot_n;
     * reading: velocity BCs hold at t_{n+1/2} for v_{n+1/2} (which enters the viscosity), and
     * s_{n+1/2} is kept in [0, 1].  v_n is kept for the corrector. */
    const int leap = c->p.integrator == 2;
    double *vn_save = NULL;
    if (leap) {
        vn_save = (double *)malloc(sizeof(double) * 3 * n);
        memcpy(vn_save, c->v, sizeof(double) * 3 * n);
        for (int64_t i = 0; i < n; i++) {
            int sp = c->spec[i];
            double dt = c->dt[sp], th = c->t[sp] + 0.5 * dt;
            for (int k = 0; k < d; k++) {
                c->u[3 * i + k] = c->u[3 * i + k] + 0.5 * dt * vn_save[3 * i + k];
                c->v[3 * i + k] = vn_save[3 * i + k] + 0.5 * dt * c->acc[3 * i + k];
            }
            for (int b = 0; b < c->nbc; b++) {
                const orc_bc *bc = &c->bc[b];
                if (bc->kind != ORC_BC_VEL || !bc->mask[i]) continue;
                double f = bc_factor(bc, th);
                if (f < 0.0) continue;
                for (int k = 0; k < d; k++) {
                    double val;
                    if ((bc->comp_mask & (1 << k)) && bc_value(bc, 1, i, k, f, &val)) c->v[3 * i + k] = val;
                }
            }
            if (is_fracture(c, i)) {
                double sh = c->s[i] + 0.5 * dt * c->sdot[i];
                sh = sh < 0.0 ? 0.0 : (sh > 1.0 ? 1.0 : sh);
                /* <restrictphi>: the bound holds at the half level too, with its value at t_{n+1/2} */
                for (int b = 0; b < c->nbc; b++) {
                    const orc_bc *bc = &c->bc[b];
                    if (bc->kind != ORC_BC_PHASE_BOUND || !bc->mask[i] || !(bc->comp_mask & 1)) continue;
                    double f = bc_factor(bc, th), val;
                    if (f < 0.0 || !bc_value(bc, 1, i, 0, f, &val)) continue;
                    val = val < 0.0 ? 0.0 : (val > 1.0 ? 1.0 : val); /* an expression's value, kept in [0, 1] */
                    if (sh < val) sh = val;
                }
                c->s[i] = sh;
            }
        }
    }
    /* contact between bodies (Algorithm 1 step 1; Algorithm 2 step 2, at the half level) */
    if (c->contact) contact_accel(c);
    double *Fpn = (double *)malloc(sizeof(double) * 9 * n);
    double *epn = (double *)malloc(sizeof(double) * n);
    /* Step 2: F and stress for every particle (from u_n, s_n; Algorithm 2: the half level) */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        deformation_gradient(c, c->u, i, &c->F[9 * i]);
        memcpy(&Fpn[9 * i], &c->Fp[9 * i], 9 * sizeof(double));
        epn[i] = c->ep[i];
        constitutive(c, i, &c->F[9 * i], 1, &c->P[9 * i], NULL, &Fpn[9 * i], &epn[i]);
    }
    /* Step 2 (cont.): acceleration, viscosity, external forces; phase field */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        const orc_material *mi = &c->mat[c->mid[i]];
        double lam, mu, kap;
        lame(mi, &lam, &mu, &kap);
        double c0 = orc_sound_speed(mi);
        double rho_i = mi->rho, h = c->p.h;
        double a[3] = {0, 0, 0};
        double lap = 0.0;
        const double *Pi = &c->P[9 * i], *Fi = &c->F[9 * i];
        double Fi_inv[9], Fi_invT[9], Ji = m_det(Fi);
        m_inv(Fi, Fi_inv);
        m_tr(Fi_inv, Fi_invT);
        for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; e++) {
            int64_t j = c->col[e];
            const orc_material *mj = &c->mat[c->mid[j]];
            double gt[3], g[3], r0[3], r;
            corrected_grad(c, i, j, gt, g, r0, &r);
            /* L_j . gradW_ij (the correction of particle j applied to the same raw gradient) */
            const double *Lj = &c->L[9 * j];
            double gtj[3] = {0, 0, 0};
            for (int q = 0; q < d; q++)
                for (int b = 0; b < d; b++) gtj[q] += Lj[3 * q + b] * g[b];
            const double *Pj = &c->P[9 * j];
            /* eq. MomentumEqTLSPH, symmetric form: (1/rho0i) V0j (P_i L_i + P_j L_j) gradW_ij */
            for (int k = 0; k < d; k++) {
                double s1 = 0.0;
                for (int q = 0; q < d; q++) s1 += Pi[3 * k + q] * gt[q] + Pj[3 * k + q] * gtj[q];
                a[k] += c->vol[j] * s1 / rho_i;
            }
            /* artificial viscosity (eq. artViscCoef), active for pairs in relative compression */
            double vij_xij = 0.0, vij_Xij = 0.0;
            for (int k = 0; k < d; k++) {
                double vij = c->v[3 * i + k] - c->v[3 * j + k];
                double xij = (c->X0[3 * i + k] + c->u[3 * i + k]) - (c->X0[3 * j + k] + c->u[3 * j + k]);
                vij_xij += vij * xij;
                vij_Xij += vij * r0[k];
            }
            if (vij_xij < 0.0) {
                double G = h * vij_Xij / (r * r + 0.001 * h * h);
                double pi = (mi->beta2 * G * G - mi->beta1 * c0 * G) / rho_i;
                double mass_j = mj->rho * c->vol[j];
                /* reading: Pv = -J pi F^-T (dissipative); literal paper: +J pi F^-1 */
                const double *Mv = c->p.visc_literal ? Fi_inv : Fi_invT;
                double sg = c->p.visc_literal ? 1.0 : -1.0;
                for (int k = 0; k < d; k++) {
                    double s1 = 0.0;
                    for (int q = 0; q < d; q++) s1 += Mv[3 * k + q] * gt[q];
                    a[k] += mass_j * sg * Ji * pi * s1;
                }
            }
            /* eq. phasefieldLapLacian */
            if (is_fracture(c, i)) {
                const double *gg = c->p.lap_uncorrected ? g : gt;
                double rg = 0.0;
                for (int k = 0; k < d; k++) rg += r0[k] * gg[k];
                lap += 2.0 * (c->s[i] - c->s[j]) * c->vol[j] * rg / (r * r);
            }
        }
        /* external forces (gravity and the force conditions) are kept apart as well, for their work */
        double ae[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < d; k++) {
            a[k] += c->p.gravity[k] + (c->contact ? c->accc[3 * i + k] : 0.0);
            ae[k] = c->p.gravity[k];
        }
        double mass = rho_i * c->vol[i];
        /* force BCs at the time of the forces: t_n (Algorithm 1), t_{n+1/2} (Algorithm 2) */
        double t_n = c->t[c->spec[i]] + (leap ? 0.5 * c->dt[c->spec[i]] : 0.0);
        for (int b = 0; b < c->nbc; b++) {
            const orc_bc *bc = &c->bc[b];
            if (bc->kind == ORC_BC_VEL || bc->kind == ORC_BC_PHASE_BOUND || !bc->mask[i]) continue;
            double f = bc_factor(bc, t_n);
            if (f < 0.0) continue;
            for (int k = 0; k < d; k++) {
                double val;
                if (!(bc->comp_mask & (1 << k)) || !bc_value(bc, 0, i, k, f, &val)) continue;
                double aek;
                if (bc->kind == ORC_BC_TRACTION) aek = val * bc->area / mass;
                else if (bc->kind == ORC_BC_ACCEL) aek = val;
                else aek = val / ((double)bc->count * mass);
                a[k] += aek;
                ae[k] += aek;
            }
        }
        for (int k = 0; k < 3; k++) {
            c->acc[3 * i + k] = k < d ? a[k] : 0.0;
            c->aext[3 * i + k] = k < d ? ae[k] : 0.0;
        }
        c->lap[i] = lap;
        if (is_fracture(c, i)) {
            /* eq. phasefieldddot: sdd = r - gamma sdot, with
             *   r = c^2/(2 eps0) (2 eps0 lap + (1 - s)/(2 eps0) - 2 s H/Gc)   (all terms but the damping),
             *   gamma = (c/eps0) sqrt(4 eps0 H/Gc + 1)                     (the damping of M, eq. Mparameter1),
             *   k = c^2/(2 eps0) (1/(2 eps0) + 2 H/Gc)                     (-dr/ds).
             * reading: the local terms are taken at the new time level,
             *   sdot_{n+1} = (sdot_n + dt r_n) / (1 + dt gamma + dt^2 k),  s_{n+1} = s_n + dt sdot_{n+1}.
             * The explicit update of Algorithm 1 diverges once dt gamma > 2, which crack tips
             * reach, contradicting the monotone, non-wave-like evolution M is chosen for
             * (Sec. 2.2); the fixed points are unchanged. */
            double e0 = mi->eps0, Gc = mi->Gc, Hh = c->Hh[i], s = c->s[i];
            double r = c0 * c0 / (2.0 * e0) * (2.0 * e0 * lap + (1.0 - s) / (2.0 * e0) - 2.0 * s * Hh / Gc);
            double k = c0 * c0 / (2.0 * e0) * (1.0 / (2.0 * e0) + 2.0 * Hh / Gc);
            double gam = c0 / e0 * sqrt(4.0 * e0 * Hh / Gc + 1.0);
            c->pf_b[i] = r;
            c->pf_k[i] = k;
            c->pf_g[i] = gam;
        }
    }
    /* Step 3-4: boundary conditions and update (Algorithm 1) */
    for (int s = 0; s < c->nspec; s++) { c->vmax[s] = 0.0; c->amax[s] = 0.0; }
    int nonfinite = 0;
    for (int64_t i = 0; i < n; i++) {
        int sp = c->spec[i];
        double dt = c->dt[sp], t1 = c->t[sp] + dt;
        double vn[3];
        /* v_{n+1} = v_n + dt a (Algorithm 1: a_n; Algorithm 2: a_{n+1/2}, from the saved v_n) */
        const double *vold = leap ? &vn_save[3 * i] : &c->v[3 * i];
        for (int k = 0; k < 3; k++) vn[k] = vold[k] + (k < d ? dt * c->acc[3 * i + k] : 0.0);
        int vmask = 0;
        for (int b = 0; b < c->nbc; b++) { /* velocity BCs at t_{n+1} */
            const orc_bc *bc = &c->bc[b];
            if (bc->kind != ORC_BC_VEL || !bc->mask[i]) continue;
            double f = bc_factor(bc, t1);
            if (f < 0.0) continue;
            for (int k = 0; k < d; k++) {
                double val;
                if ((bc->comp_mask & (1 << k)) && bc_value(bc, 0, i, k, f, &val)) {
                    vn[k] = val;
                    vmask |= 1 << k;
                }
            }
        }
        /* external work (Sec. 3.5 energy tracking): the work of the external forces along the step's
         * displacement increment u_{n+1} - u_n, which is dt v_{n+1} (Algorithm 1) or dt (v_n + v_{n+1}) / 2
         * (Algorithm 2).  On a component a velocity condition holds, the external force is its reaction
         * m (v_{n+1} - v_n) / dt - m a_interactions (a_interactions = a - a_ext) */
        {
            const double mass = c->mat[c->mid[i]].rho * c->vol[i];
            double wk = 0.0;
            for (int k = 0; k < d; k++) {
                const double aext = c->aext[3 * i + k];
                const double fe = (vmask & (1 << k)) ? mass * ((vn[k] - vold[k]) / dt - (c->acc[3 * i + k] - aext))
                                                     : mass * aext;
                const double dk = leap ? 0.5 * dt * (vold[k] + vn[k]) : dt * vn[k];
                wk += fe * dk;
            }
            c->wext[i] += wk;
        }
        double vv = 0.0, aa = 0.0;
        /* u_{n+1} = u_n + dt v_{n+1} (Algorithm 1); u_{n+1/2} + dt/2 v_{n+1} (Algorithm 2) */
        const double du = leap ? 0.5 * dt : dt;
        for (int k = 0; k < d; k++) {
            c->v[3 * i + k] = vn[k];
            c->u[3 * i + k] = c->u[3 * i + k] + du * vn[k];
            vv += vn[k] * vn[k];
            aa += c->acc[3 * i + k] * c->acc[3 * i + k];
        }
        vv = sqrt(vv);
        aa = sqrt(aa);
        if (!isfinite(vv) || !isfinite(aa)) nonfinite = 1;
        if (vv > c->vmax[sp]) c->vmax[sp] = vv;
        if (aa > c->amax[sp]) c->amax[sp] = aa;
        if (is_fracture(c, i)) {
            /* the printed form (pf_explicit): sddot_n = r_n - gamma sdot_n (r holds the local stiffness term
             * at s_n), sdot_{n+1} = sdot_n + dt sddot_n */
            double sd1 = c->p.pf_explicit ? c->sdot[i] + dt * (c->pf_b[i] - c->pf_g[i] * c->sdot[i])
                                          : (c->sdot[i] + dt * c->pf_b[i]) /
                                                (1.0 + dt * c->pf_g[i] + dt * dt * c->pf_k[i]);
            c->sdd[i] = (sd1 - c->sdot[i]) / dt;
            c->sdot[i] = sd1;
            /* s_{n+1} = s_n + dt sdot_{n+1} (Algorithm 1); s_{n+1/2} + dt/2 sdot_{n+1} (Algorithm 2) */
            double sn = c->s[i] + du * c->sdot[i];
            sn = sn < 0.0 ? 0.0 : (sn > 1.0 ? 1.0 : sn); /* reading: s kept in [0, 1] */
            /* <restrictphi> (Sec. 3.3, used in Sec. 4 to keep particles near loads intact): the particles a
             * bound covers keep s_{n+1} >= its value at t_{n+1}; reading: s alone is raised, sdot is kept */
            for (int b = 0; b < c->nbc; b++) {
                const orc_bc *bc = &c->bc[b];
                if (bc->kind != ORC_BC_PHASE_BOUND || !bc->mask[i] || !(bc->comp_mask & 1)) continue;
                double f = bc_factor(bc, t1), val;
                if (f < 0.0 || !bc_value(bc, 0, i, 0, f, &val)) continue;
                val = val < 0.0 ? 0.0 : (val > 1.0 ? 1.0 : val); /* an expression's value, kept in [0, 1] */
                if (sn < val) sn = val;
            }
            c->s[i] = sn;
        }
        memcpy(&c->Fp[9 * i], &Fpn[9 * i], 9 * sizeof(double));
        c->ep[i] = epn[i];
        if (c->status[i] == 1) c->noconv++;
    }
    for (int s = 0; s < c->nspec; s++) c->t[s] += c->dt[s];
    c->step++;
    free(Fpn);
    free(epn);
    free(vn_save);
    return nonfinite ? ORC_ERR_NONFINITE : ORC_OK;
}

int orc_step(orc_ctx *c, int64_t nsteps) {
    if (!c || !c->built) return ORC_ERR_STATE;
    for (int64_t k = 0; k < nsteps; k++) {
        int st = one_step(c);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* state access                                                        */
/* ------------------------------------------------------------------ */
#define ORC_F_U 0
#define ORC_F_V 1
#define ORC_F_X 2
#define ORC_F_S 3
#define ORC_F_SDOT 4
#define ORC_F_H 5
#define ORC_F_EPSP 6
#define ORC_F_P 7
#define ORC_F_F 8
#define ORC_F_FP 9
#define ORC_F_L 10
#define ORC_F_ACC 11
#define ORC_F_CPINV 12
#define ORC_F_SDD 13
#define ORC_F_LAP 14

/* F and P evaluated at the current state without committing the state
 * (J2 runs a trial return map from the stored F_p). */
static void eval_FP(orc_ctx *c, double *Fout, double *Pout, double *psi) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < c->n; i++) {
        double Fp[9], ep;
        deformation_gradient(c, c->u, i, &Fout[9 * i]);
        memcpy(Fp, &c->Fp[9 * i], sizeof Fp);
        ep = c->ep[i];
        constitutive(c, i, &Fout[9 * i], 0, &Pout[9 * i], psi ? &psi[i] : NULL, Fp, &ep);
    }
}

int orc_read(orc_ctx *c, int field, double *out) {
    if (!c || !out || c->n <= 0) return ORC_ERR_ARG;
    int64_t n = c->n;
    int d = c->p.dim;
    switch (field) {
    case ORC_F_U:
    case ORC_F_V:
    case ORC_F_X:
    case ORC_F_ACC:
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < d; k++) {
                double x = field == ORC_F_U ? c->u[3 * i + k]
                         : field == ORC_F_V ? c->v[3 * i + k]
                         : field == ORC_F_ACC ? c->acc[3 * i + k]
                                              : c->X0[3 * i + k] + c->u[3 * i + k];
                out[d * i + k] = x;
            }
        return ORC_OK;
    case ORC_F_S: memcpy(out, c->s, sizeof(double) * n); return ORC_OK;
    case ORC_F_SDOT: memcpy(out, c->sdot, sizeof(double) * n); return ORC_OK;
    case ORC_F_H: memcpy(out, c->Hh, sizeof(double) * n); return ORC_OK;
    case ORC_F_SDD: memcpy(out, c->sdd, sizeof(double) * n); return ORC_OK;
    case ORC_F_LAP: memcpy(out, c->lap, sizeof(double) * n); return ORC_OK;
    case ORC_F_EPSP: memcpy(out, c->ep, sizeof(double) * n); return ORC_OK;
    case ORC_F_FP: memcpy(out, c->Fp, sizeof(double) * 9 * n); return ORC_OK;
    case ORC_F_L: memcpy(out, c->L, sizeof(double) * 9 * n); return ORC_OK;
    case ORC_F_CPINV:
        for (int64_t i = 0; i < n; i++) {
            double Fi[9], FiT[9];
            m_inv(&c->Fp[9 * i], Fi);
            m_tr(Fi, FiT);
            m_mul(Fi, FiT, &out[9 * i]);
        }
        return ORC_OK;
    case ORC_F_P:
    case ORC_F_F: {
        if (!c->built) return ORC_ERR_STATE;
        double *Fb = (double *)malloc(sizeof(double) * 9 * n), *Pb = (double *)malloc(sizeof(double) * 9 * n);
        eval_FP(c, Fb, Pb, NULL);
        memcpy(out, field == ORC_F_P ? Pb : Fb, sizeof(double) * 9 * n);
        free(Fb);
        free(Pb);
        return ORC_OK;
    }
    default: return ORC_ERR_ARG;
    }
}

int orc_write(orc_ctx *c, int field, const double *in) {
    if (!c || !in || c->n <= 0) return ORC_ERR_ARG;
    int64_t n = c->n;
    int d = c->p.dim;
    switch (field) {
    case ORC_F_U:
    case ORC_F_V:
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < d; k++) (field == ORC_F_U ? c->u : c->v)[3 * i + k] = in[d * i + k];
        return ORC_OK;
    case ORC_F_S: memcpy(c->s, in, sizeof(double) * n); return ORC_OK;
    case ORC_F_SDOT: memcpy(c->sdot, in, sizeof(double) * n); return ORC_OK;
    case ORC_F_H: memcpy(c->Hh, in, sizeof(double) * n); return ORC_OK;
    case ORC_F_EPSP: memcpy(c->ep, in, sizeof(double) * n); return ORC_OK;
    case ORC_F_FP: memcpy(c->Fp, in, sizeof(double) * 9 * n); return ORC_OK;
    default: return ORC_ERR_ARG;
    }
}

/*
 * Energies of the current state (Sec. 3.5 energy tracking):
 * out[0] kinetic sum 1/2 m |v|^2, out[1] strain sum V psi_e (degraded),
 * out[2] fracture sum V Gc ((1-s)^2/(4 eps0) + eps0 |grad s|^2),
 * out[3] plastic work sum V (sigma_y0 eps_p + H eps_p^2 / 2),
 * out[4] external work since the start: the sum over steps and particles of the work of the
 *        external forces (gravity, force conditions, reactions of velocity conditions) along the
 *        step's displacement increment (one_step),
 * out[5] time of specimen 0.
 */
int orc_energies(orc_ctx *c, double *out) {
    if (!c || !out || !c->built) return ORC_ERR_STATE;
    int64_t n = c->n;
    int d = c->p.dim;
    double *Fb = (double *)malloc(sizeof(double) * 9 * n), *Pb = (double *)malloc(sizeof(double) * 9 * n);
    double *psi = (double *)malloc(sizeof(double) * n);
    eval_FP(c, Fb, Pb, psi);
    double ke = 0, se = 0, fe = 0, pw = 0, we = 0;
    for (int64_t i = 0; i < n; i++) {
        const orc_material *m = &c->mat[c->mid[i]];
        double vv = 0.0;
        for (int k = 0; k < d; k++) vv += c->v[3 * i + k] * c->v[3 * i + k];
        ke += 0.5 * m->rho * c->vol[i] * vv;
        se += c->vol[i] * psi[i];
        we += c->wext[i];
        if (m->model == ORC_MODEL_J2)
            pw += c->vol[i] * (m->sigma_y0 * c->ep[i] + 0.5 * m->H_hard * c->ep[i] * c->ep[i]);
        if (is_fracture(c, i)) {
            double gs[3] = {0, 0, 0};
            for (int64_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; e++) {
                int64_t j = c->col[e];
                double gt[3], g[3], r0[3], r;
                corrected_grad(c, i, j, gt, g, r0, &r);
                for (int k = 0; k < d; k++) gs[k] += c->vol[j] * (c->s[j] - c->s[i]) * gt[k];
            }
            double g2 = gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2];
            double om = 1.0 - c->s[i];
            fe += c->vol[i] * m->Gc * (om * om / (4.0 * m->eps0) + m->eps0 * g2);
        }
    }
    out[0] = ke;
    out[1] = se;
    out[2] = fe;
    out[3] = pw;
    out[4] = we;
    out[5] = c->t[0];
    free(Fb);
    free(Pb);
    free(psi);
    return ORC_OK;
}

int64_t orc_noconv(const orc_ctx *c) { return c ? c->noconv : -1; }
int64_t orc_step_count(const orc_ctx *c) { return c ? c->step : -1; }
int orc_time(const orc_ctx *c, int spec, double *t, double *dt) {
    if (!c || spec < 0 || spec >= c->nspec) return ORC_ERR_ARG;
    *t = c->t[spec];
    *dt = c->dt[spec];
    return ORC_OK;
}
