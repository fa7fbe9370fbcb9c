// Constitutive updates of the TLSPH step (device code).
//
// The models take the displacement gradient G = F - I (so that small
// strains keep their relative precision in FP32) and return the second
// Piola-Kirchhoff stress S.
//
//  * St. Venant-Kirchhoff with the spectral split of the Green-Lagrange strain
//    (Sec. 2.3.1): S = s^2 S+ + S-, S+- = lambda {tr E}+- I + 2 mu E+-, where E+-
//    keep the positive / negative eigenvalues of E.
//  * Neo-Hookean with the J-split of the phase-field degradation (Sec. 2.3.2):
//      S = s^2 (Svol + Siso)       J >= 1
//      S = Svol + s^2 Siso         J <  1
//    Svol = kappa/2 (J^2 - 1) C^-1, Siso = mu J^-2/3 (I - tr(C)/3 C^-1).  The
//    stress is the derivative of the stated energy with respect to C/2 (the
//    printed formula writes b^-1; C^-1 is the frame-indifferent derivative).
//  * Finite-strain J2 plasticity (Sec. 2.3.3).  The plastic state is kept as
//    C_p^-1 = F_p^-1 F_p^-T (stored as K = C_p^-1 - I): the stress, the trial
//    state and the exponential-map update depend on F_p only through it.
//    With A = C_p^-1 C (similar to the elastic C_e), the trial flow direction
//    commutes with A, so the residual of the return map (eq. J2_residual) is a
//    scalar function of the eigenvalues of A; the Illinois / regula-falsi
//    iteration with bracket doubling runs on that scalar, and the accepted
//    increment updates C_p^-1 <- exp(-2 dgamma N~) C_p^-1 with a scaling and
//    squaring Taylor series, followed by the isochoric projection det = 1.
#pragma once
#include "tensor3.cuh"

namespace tl {

template <typename T> struct MatT {
    int model;      // 1 SVK, 2 NH, 3 J2
    int fracture;   // phase field on
    T rho, mu, kappa, sy0, Hh, beta1, beta2, c0, Gc, eps0, s_lim, mass_scale;
    T lam;          // Lame's first parameter
    T cinv;         // (1 - nu^2) / E, the material's share of the contact modulus 1/E*
};

// x + x^2/2 - log(1 + x) (= (J^2 - 1)/2 - ln J with x = J - 1), series near 0
template <typename T> TL_HD T xp_minus_log(T x) {
    if (t_abs(x) < T(0.01)) {
        // x^2 - x^3/3 + x^4/4 - ... - x^11/11
        T r = T(-1.0 / 11.0);
        r = r * x + T(1.0 / 10.0);
        r = r * x - T(1.0 / 9.0);
        r = r * x + T(1.0 / 8.0);
        r = r * x - T(1.0 / 7.0);
        r = r * x + T(1.0 / 6.0);
        r = r * x - T(1.0 / 5.0);
        r = r * x + T(1.0 / 4.0);
        r = r * x - T(1.0 / 3.0);
        r = r * x + T(1.0);
        return r * x * x;
    }
    return x + T(0.5) * x * x - t_log1p(x);
}

// tr(I + X) - 3 det(I + X)^(1/3) without first-order cancellation (for X with real
// spectrum): with a = 1 + tr X / 3 and B = dev X, det(a I + B) = a^3 (1 + x),
// x = -tr(B^2) / (2 a^2) + det(B) / a^3, so the difference is -3 a ((1 + x)^(1/3) - 1).
template <typename T> TL_HD T iso_excess(const M3<T> &X) {
    const T t3 = trace(X) / T(3);
    const T a = T(1) + t3;
    M3<T> B = X;
    B.a[0] -= t3;
    B.a[4] -= t3;
    B.a[8] -= t3;
    const T x = -trace_mul(B, B) / (T(2) * a * a) + det(B) / (a * a * a);
    return T(-3) * a * t_expm1(t_log1p(x) / T(3));
}

// Kinematics shared by both models.
template <typename T> struct Kin {
    M3<T> E2;    // C - I = G + G^T + G^T G
    M3<T> Ci;    // C^-1
    T Jm1;       // J - 1
    T Jm23;      // J^-2/3
    T Jm23m1;    // J^-2/3 - 1
};
template <typename T> TL_HD Kin<T> kinematics(const M3<T> &G) {
    Kin<T> k;
    k.E2 = mul_tn(G, G);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) k.E2.a[3 * i + j] += G.a[3 * i + j] + G.a[3 * j + i];
    k.Jm1 = det_eye_plus_m1(G);
    M3<T> C = k.E2;
    C.a[0] += T(1);
    C.a[4] += T(1);
    C.a[8] += T(1);
    inverse(C, k.Ci);
    T lJ = t_log1p(k.Jm1);
    k.Jm23m1 = t_expm1(T(-2.0 / 3.0) * lJ);
    k.Jm23 = T(1) + k.Jm23m1;
    return k;
}

// Neo-Hookean stress and energy split.  psi_plus / psi_minus of eq. ksipNH / ksinNH.
template <typename T>
TL_HD void nh_stress(const Kin<T> &k, T s, const MatT<T> &m, M3<T> &S, T &psi_plus, T &psi_minus) {
    T trE2 = trace(k.E2);
    M3<T> dE = k.E2;
    dE.a[0] -= trE2 / T(3);
    dE.a[4] -= trE2 / T(3);
    dE.a[8] -= trE2 / T(3);
    // Siso = mu J^-2/3 (I - tr C / 3 C^-1) = mu J^-2/3 C^-1 dev(C - I)
    M3<T> Siso = sym_part(mul(k.Ci, dE));
    T fi = m.mu * k.Jm23;
    T fv = T(0.5) * m.kappa * k.Jm1 * (k.Jm1 + T(2));
    T U = T(0.5) * m.kappa * xp_minus_log(k.Jm1);
    // psibar = mu/2 (tr bbar - 3) = mu/2 J^-2/3 (tr C - 3 J^2/3)
    T psibar = T(0.5) * m.mu * k.Jm23 * iso_excess(k.E2);
    T s2 = s * s;
    T cv, ci;
    if (k.Jm1 >= T(0)) {
        cv = s2 * fv;
        ci = s2 * fi;
        psi_plus = U + psibar;
        psi_minus = T(0);
    } else {
        cv = fv;
        ci = s2 * fi;
        psi_plus = psibar;
        psi_minus = U;
    }
#pragma unroll
    for (int q = 0; q < 9; q++) S.a[q] = cv * k.Ci.a[q] + ci * Siso.a[q];
}

// Eigenvalues of a traceless 3x3 matrix with real spectrum (trigonometric form).
template <typename T> TL_HD void eig_traceless(const M3<T> &B, T q2, T e[3]) {
    T p = q2 / T(6);
    if (!(p > T(0))) {
        e[0] = e[1] = e[2] = T(0);
        return;
    }
    T q = T(0.5) * det(B);
    T sp = t_sqrt(p);
    T r = q / (p * sp);
    r = t_min(T(1), t_max(T(-1), r));
    T phi = t_acos(r) / T(3);
    T two_sp = T(2) * sp;
    e[0] = two_sp * t_cos(phi);
    e[1] = two_sp * t_cos(phi + T(2.0943951023931953));
    e[2] = -e[0] - e[1];
}

// Positive part of the symmetric 2x2 matrix [[a, b], [b, d]] with eigenvalues p1 >= p2: all of
// it when p2 >= 0, nothing when p1 <= 0, else p1 (A - p2 I) / (p1 - p2) (the spectral projector
// onto the p1 eigenvector, scaled by p1).
template <typename T> TL_HD void pos_part2(T a, T b, T d, T &pa, T &pb, T &pd, T &p1, T &p2) {
    const T m = T(0.5) * (a + d), h = T(0.5) * (a - d);
    const T r = t_sqrt(h * h + b * b);
    p1 = m + r;
    p2 = m - r;
    if (p2 >= T(0)) {
        pa = a;
        pb = b;
        pd = d;
    } else if (p1 <= T(0)) {
        pa = pb = pd = T(0);
    } else {  // p1 > 0 > p2, so r > 0
        const T f = p1 / (T(2) * r);
        pa = f * (a - p2);
        pb = f * b;
        pd = f * (d - p2);
    }
}

// Spectral split of a symmetric strain (eq. GLstratinP): Ep = Q diag({lambda_a}+) Q^T and the
// eigenvalues l[3].  In 2D (plane strain) E has the in-plane block and E33 = 0.  In 3D the
// deviator, scaled to unit largest entry, gives by the trigonometric form its eigenvalue
// farthest from the other two; that one is accurate and separated from the others by at
// least half the spectral range, so its eigenvector n, the largest cross product of two rows
// of (dev E - e I), is accurate too.  The other two eigenvalues are those of the 2x2 block of E
// in the plane orthogonal to n, found in closed form, so near-equal eigenvalues (which the
// trigonometric form resolves only to sqrt(eps)) keep full accuracy.
template <typename T, int DIM> TL_HD void strain_split(const M3<T> &E, M3<T> &Ep, T l[3]) {
    if (DIM == 2) {
        T pa, pb, pd;
        pos_part2(E.a[0], E.a[1], E.a[4], pa, pb, pd, l[0], l[1]);
        l[2] = T(0);
        Ep = m3_zero<T>();
        Ep.a[0] = pa;
        Ep.a[1] = Ep.a[3] = pb;
        Ep.a[4] = pd;
        return;
    }
    const T t = trace(E) / T(3);
    M3<T> B = E;
    B.a[0] -= t;
    B.a[4] -= t;
    B.a[8] -= t;
    T sc = T(0);
#pragma unroll
    for (int q = 0; q < 9; q++) sc = t_max(sc, t_abs(B.a[q]));
    if (!(sc > T(0))) {  // isotropic
        l[0] = l[1] = l[2] = t;
        Ep = t > T(0) ? E : m3_zero<T>();
        return;
    }
    const T isc = T(1) / sc;
#pragma unroll
    for (int q = 0; q < 9; q++) B.a[q] *= isc;
    T e[3];
    eig_traceless(B, trace_mul(B, B), e);  // e[0] largest, e[1] smallest, e[2] between
    const T ei = (e[0] - e[2] >= e[2] - e[1]) ? e[0] : e[1];
    // eigenvector of ei: null vector of M = B - ei I from the largest cross product of two rows
    T r[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r[i][j] = B.a[3 * i + j] - (i == j ? ei : T(0));
    T n[3] = {T(0), T(0), T(0)}, best = T(-1);
#pragma unroll
    for (int pr = 0; pr < 3; pr++) {
        const int i = pr == 2 ? 1 : 0, j = pr == 0 ? 1 : 2;
        const T c0 = r[i][1] * r[j][2] - r[i][2] * r[j][1];
        const T c1 = r[i][2] * r[j][0] - r[i][0] * r[j][2];
        const T c2 = r[i][0] * r[j][1] - r[i][1] * r[j][0];
        const T nn = c0 * c0 + c1 * c1 + c2 * c2;
        if (nn > best) {
            best = nn;
            n[0] = c0;
            n[1] = c1;
            n[2] = c2;
        }
    }
    T inv = T(1) / t_sqrt(best);
    n[0] *= inv;
    n[1] *= inv;
    n[2] *= inv;
    // orthonormal u, v spanning the plane orthogonal to n: u = e_k x n for the axis k least aligned with n
    T u[3];
    const T a0 = t_abs(n[0]), a1 = t_abs(n[1]), a2 = t_abs(n[2]);
    if (a0 <= a1 && a0 <= a2) {
        u[0] = T(0), u[1] = -n[2], u[2] = n[1];
    } else if (a1 <= a2) {
        u[0] = n[2], u[1] = T(0), u[2] = -n[0];
    } else {
        u[0] = -n[1], u[1] = n[0], u[2] = T(0);
    }
    inv = T(1) / t_sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] *= inv;
    u[1] *= inv;
    u[2] *= inv;
    const T v[3] = {n[1] * u[2] - n[2] * u[1], n[2] * u[0] - n[0] * u[2], n[0] * u[1] - n[1] * u[0]};
    // the 2x2 block of B in (u, v)
    T Bu[3], Bv[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Bu[i] = B.a[3 * i] * u[0] + B.a[3 * i + 1] * u[1] + B.a[3 * i + 2] * u[2];
        Bv[i] = B.a[3 * i] * v[0] + B.a[3 * i + 1] * v[1] + B.a[3 * i + 2] * v[2];
    }
    const T buu = u[0] * Bu[0] + u[1] * Bu[1] + u[2] * Bu[2];
    const T buv = v[0] * Bu[0] + v[1] * Bu[1] + v[2] * Bu[2];
    const T bvv = v[0] * Bv[0] + v[1] * Bv[1] + v[2] * Bv[2];
    T pa, pb, pd;
    pos_part2(sc * buu + t, sc * buv, sc * bvv + t, pa, pb, pd, l[1], l[2]);
    l[0] = sc * ei + t;
    const T lo = t_min(l[0], l[2]), hi = t_max(l[0], l[1]);
    if (lo >= T(0)) {
        Ep = E;
        return;
    }
    if (hi <= T(0)) {
        Ep = m3_zero<T>();
        return;
    }
    const T li = t_max(l[0], T(0));
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            Ep.a[3 * i + j] = li * n[i] * n[j] + pa * u[i] * u[j] + pb * (u[i] * v[j] + v[i] * u[j]) + pd * v[i] * v[j];
}

// St. Venant-Kirchhoff stress with the spectral split (eq. elasEnergyP, elasEnergyN, 2PK_SVK1,
// 2PK_SVK2): S = s^2 (lambda {tr E}+ I + 2 mu E+) + lambda {tr E}- I + 2 mu E-, E = (C - I) / 2.
template <typename T, int DIM>
TL_HD void svk_stress(const Kin<T> &k, T s, const MatT<T> &m, M3<T> &S, T &psi_plus, T &psi_minus) {
    M3<T> E;
#pragma unroll
    for (int q = 0; q < 9; q++) E.a[q] = T(0.5) * k.E2.a[q];
    M3<T> Ep;
    T l[3];
    strain_split<T, DIM>(E, Ep, l);
    const T tr = trace(E);
    const T trp = t_max(tr, T(0)), trm = t_min(tr, T(0));
    T sp2 = T(0), sm2 = T(0);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const T lp = t_max(l[q], T(0)), lm = t_min(l[q], T(0));
        sp2 += lp * lp;
        sm2 += lm * lm;
    }
    psi_plus = T(0.5) * m.lam * trp * trp + m.mu * sp2;
    psi_minus = T(0.5) * m.lam * trm * trm + m.mu * sm2;
    const T s2 = s * s, mu2 = T(2) * m.mu;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const T id = (q % 4 == 0) ? T(1) : T(0);
        S.a[q] = s2 * (m.lam * trp * id + mu2 * Ep.a[q]) + (m.lam * trm * id + mu2 * (E.a[q] - Ep.a[q]));
    }
}

// exp(X) - I by scaling and squaring of a Taylor series (order 6 in FP32, 12 in FP64).
template <typename T> TL_HD M3<T> expm1_mat(const M3<T> &X) {
    T nrm2 = T(0);
#pragma unroll
    for (int q = 0; q < 9; q++) nrm2 += X.a[q] * X.a[q];
    int ks = 0;
    T scale = T(1);
    while (nrm2 * scale * scale > T(1.0 / 64.0) && ks < 40) {
        scale *= T(0.5);
        ks++;
    }
    M3<T> B;
#pragma unroll
    for (int q = 0; q < 9; q++) B.a[q] = X.a[q] * scale;
    constexpr int order = sizeof(T) == 4 ? 6 : 12;
    // Horner: E1 = B (I + B/2 (I + B/3 (... (I + B/order))))
    M3<T> R = m3_eye<T>();
#pragma unroll
    for (int m = order; m >= 2; m--) {
        M3<T> t = mul(B, R);
        T inv = T(1) / T(m);
#pragma unroll
        for (int q = 0; q < 9; q++) R.a[q] = t.a[q] * inv;
        R.a[0] += T(1);
        R.a[4] += T(1);
        R.a[8] += T(1);
    }
    M3<T> E1 = mul(B, R);
    for (int s = 0; s < ks; s++) {  // expm1(2Y) = E1 (E1 + 2 I)
        M3<T> sq = mul(E1, E1);
#pragma unroll
        for (int q = 0; q < 9; q++) E1.a[q] = T(2) * E1.a[q] + sq.a[q];
    }
    return E1;
}

template <typename T> struct J2Tol;
// FP32 stops when the bracket is two ulps wide: adjacent floats are up to 1.19e-7 apart relative to the
// larger, so a narrower width could not be met when the residual's rounding stays above res sy0.
template <> struct J2Tol<float> {
    static constexpr float res = 1e-5f, width = 2.5e-7f;
    static constexpr int maxit = 100;
};
template <> struct J2Tol<double> {
    static constexpr double res = 1e-10, width = 1e-14;
    static constexpr int maxit = 100;
};

// Residual r(dgamma) of eq. J2_residual in the eigenbasis of A = C_p^-1 C.
template <typename T> struct J2Res {
    T delta[3], n[3], c_eq, sy0, Hh, epn;
    TL_HD T operator()(T dg) const {
        T dp[3];
#pragma unroll
        for (int a = 0; a < 3; a++) dp[a] = delta[a] + (T(1) + delta[a]) * t_expm1(T(-2) * dg * n[a]);
        T mean = (dp[0] + dp[1] + dp[2]) / T(3);
        T s2 = T(0);
#pragma unroll
        for (int a = 0; a < 3; a++) s2 += (dp[a] - mean) * (dp[a] - mean);
        return c_eq * t_sqrt(s2) - (sy0 + Hh * (epn + dg));
    }
};

// Trial state of the J2 update: C_p^-1 held fixed, D = A - I with A = C_p^-1 C, its deviator,
// the trial equivalent stress sigma_tr = sqrt(3/2) mu J^-2/3 |dev D| and the yield function
// f = sigma_tr - (sigma_y0 + H eps_p) whose sign decides elastic / plastic ahead of eq. J2_residual.
// K6 = (xx, yy, zz, xy, xz, yz) of C_p^-1 - I.
template <typename T> struct J2Trial {
    M3<T> K, D, dev;
    T trD3, q2, c_eq, sig_tr, syn, f;
};
template <typename T> TL_HD J2Trial<T> j2_trial(const Kin<T> &k, const T K6[6], T ep, const MatT<T> &m) {
    J2Trial<T> t;
    t.K.a[0] = K6[0]; t.K.a[4] = K6[1]; t.K.a[8] = K6[2];
    t.K.a[1] = t.K.a[3] = K6[3];
    t.K.a[2] = t.K.a[6] = K6[4];
    t.K.a[5] = t.K.a[7] = K6[5];
    // D = A - I = K + E2 + K E2
    t.D = mul(t.K, k.E2);
#pragma unroll
    for (int q = 0; q < 9; q++) t.D.a[q] += t.K.a[q] + k.E2.a[q];
    t.trD3 = trace(t.D) / T(3);
    t.dev = t.D;
    t.dev.a[0] -= t.trD3;
    t.dev.a[4] -= t.trD3;
    t.dev.a[8] -= t.trD3;
    t.q2 = t_max(trace_mul(t.dev, t.dev), T(0));
    t.c_eq = T(1.2247448713915890) * m.mu * k.Jm23;  // sqrt(3/2) mu J^-2/3
    t.sig_tr = t.c_eq * t_sqrt(t.q2);
    t.syn = m.sy0 + m.Hh * ep;
    t.f = t.sig_tr - t.syn;
    return t;
}

// Second Piola-Kirchhoff stress of the J2 model at a plastic state, from dev(D) of that state:
// S = mu J^-2/3 (C_p^-1 - tr(A)/3 C^-1) + kappa/2 (J^2 - 1) C^-1 = mu J^-2/3 C^-1 dev(D)^T + ...
// With the trial state (C_p^-1 of the last step) it is the elastic predictor.
template <typename T> TL_HD M3<T> j2_stress(const Kin<T> &k, const M3<T> &dev, const MatT<T> &m) {
    const M3<T> Siso = sym_part(mul(k.Ci, transpose(dev)));
    const T fi = m.mu * k.Jm23;
    const T fv = T(0.5) * m.kappa * k.Jm1 * (k.Jm1 + T(2));
    M3<T> S;
#pragma unroll
    for (int q = 0; q < 9; q++) S.a[q] = fi * Siso.a[q] + fv * k.Ci.a[q];
    return S;
}

// J2 update.  K6 = (xx, yy, zz, xy, xz, yz) of C_p^-1 - I.  Returns 0, or 1 if the
// bracket / iteration did not converge (the state is still updated with the last iterate).
template <typename T>
TL_HD int j2_update(const Kin<T> &k, const T K6[6], T ep, const MatT<T> &m, T K6out[6], T &ep_out,
                                         M3<T> &S, T &dgamma) {
    const J2Trial<T> tr = j2_trial(k, K6, ep, m);
    M3<T> K = tr.K, D = tr.D, dev = tr.dev;
    T trD3 = tr.trD3;
    const T q2 = tr.q2, c_eq = tr.c_eq, sig_tr = tr.sig_tr, syn = tr.syn, f = tr.f;
    int status = 0;
    T dg = T(0);
#pragma unroll
    for (int q = 0; q < 6; q++) K6out[q] = K6[q];
    if (f > T(0)) {
        J2Res<T> r;
        T e[3];
        eig_traceless(dev, q2, e);
        T kn = T(1.5) * m.mu * k.Jm23 / sig_tr;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            r.delta[a] = e[a] + trD3;
            r.n[a] = kn * e[a];
        }
        r.c_eq = c_eq;
        r.sy0 = m.sy0;
        r.Hh = m.Hh;
        r.epn = ep;
        // bracket: L = 0, R = max((sigma_tr - sigma_y) / (3 mu + H), eps), doubled until r(R) <= 0.  r falls
        // from f to about -sigma_y where the frozen flow has removed the deviator and rises again beyond:
        // a doubling that lands past that minimum with r still positive (r rose) has stepped over the
        // negative interval, and a golden-section search for the minimum on the last interval stops at
        // the first point with r <= 0 (the doubling goes on if it finds none: near r = 0 rounding alone
        // can make r rise).
        T L = T(0), rL = f;
        T eps_b = T(1e-12) * syn / m.mu;
        const T R0 = t_max(f / (T(3) * m.mu + m.Hh), eps_b);
        T R = R0;
        T rR = r(R);
        T Rp = T(0);
        for (int nd = 0; rR > T(0) && nd < 60; nd++) {
            const T Rn = T(2) * R;
            const T rn = r(Rn);
            if (rn > T(0) && rn >= rR) {
                const T g = T(0.6180339887498949);
                T a = Rp, b = Rn;
                T c1 = b - g * (b - a), d1 = a + g * (b - a);
                T rc = r(c1), rd = r(d1);
                bool found = false;
                for (int k = 0; k < 80; k++) {
                    if (rc <= T(0)) {
                        R = c1;
                        rR = rc;
                        found = true;
                        break;
                    }
                    if (rd <= T(0)) {
                        R = d1;
                        rR = rd;
                        found = true;
                        break;
                    }
                    if (rc < rd) {
                        b = d1;
                        d1 = c1;
                        rd = rc;
                        c1 = b - g * (b - a);
                        rc = r(c1);
                    } else {
                        a = c1;
                        c1 = d1;
                        rc = rd;
                        d1 = a + g * (b - a);
                        rd = r(d1);
                    }
                }
                if (found) break;
                // no point below zero (r rose only by rounding near r = 0): keep doubling
            }
            Rp = R;
            R = Rn;
            rR = rn;
        }
        T x = R;
        if (!(rR <= T(0))) {
            // no bracket (a trial far outside the yield surface): keep the state finite with the
            // small-strain estimate and report the particle as non-converged
            status = 1;
            x = R0;
        }
        if (rR != T(0) && status == 0) {
            int it = 0;
            for (; it < J2Tol<T>::maxit; it++) {
                T den = rR - rL;
                x = den != T(0) ? R - rR * (R - L) / den : T(0.5) * (L + R);
                T rx = r(x);
                if (t_abs(rx) <= J2Tol<T>::res * m.sy0 || t_abs(R - L) <= J2Tol<T>::width * t_abs(R)) break;
                if ((rx < T(0) && rR > T(0)) || (rx > T(0) && rR < T(0))) {
                    L = R;
                    rL = rR;
                } else {
                    rL = T(0.5) * rL;
                }
                R = x;
                rR = rx;
            }
            if (it == J2Tol<T>::maxit) status = 1;
        }
        dg = x;
        // C_p^-1 <- exp(-2 dg N~) C_p^-1, N~ = (3 mu J^-2/3 / (2 sigma_tr)) dev(A)
        M3<T> X;
        T sc = T(-2) * dg * kn;
#pragma unroll
        for (int q = 0; q < 9; q++) X.a[q] = sc * dev.a[q];
        M3<T> E1 = expm1_mat(X);
        M3<T> E1K = mul(E1, K);
        M3<T> Kn;
#pragma unroll
        for (int q = 0; q < 9; q++) Kn.a[q] = K.a[q] + E1.a[q] + E1K.a[q];
        Kn = sym_part(Kn);
        // isochoric projection det(C_p^-1) = 1
        T detm1 = det_eye_plus_m1(Kn);
        T fm1 = t_expm1(-t_log1p(detm1) / T(3));
#pragma unroll
        for (int q = 0; q < 9; q++) Kn.a[q] = Kn.a[q] * (T(1) + fm1);
        Kn.a[0] += fm1;
        Kn.a[4] += fm1;
        Kn.a[8] += fm1;
        K = Kn;
        K6out[0] = K.a[0]; K6out[1] = K.a[4]; K6out[2] = K.a[8];
        K6out[3] = K.a[1]; K6out[4] = K.a[2]; K6out[5] = K.a[5];
        // stress from the updated state
        D = mul(K, k.E2);
#pragma unroll
        for (int q = 0; q < 9; q++) D.a[q] += K.a[q] + k.E2.a[q];
        trD3 = trace(D) / T(3);
        dev = D;
        dev.a[0] -= trD3;
        dev.a[4] -= trD3;
        dev.a[8] -= trD3;
    }
    ep_out = ep + dg;
    dgamma = dg;
    S = j2_stress(k, dev, m);
    return status;
}

// Strain energy of the J2 model, psi_vol(J) + psi_iso(Cbar_e) (evaluated at a given C_p^-1).
template <typename T> TL_HD T j2_energy(const Kin<T> &k, const T K6[6], const MatT<T> &m) {
    // tr(C_e) = tr(C_p^-1 C) = 3 + tr(D)
    M3<T> K;
    K.a[0] = K6[0]; K.a[4] = K6[1]; K.a[8] = K6[2];
    K.a[1] = K.a[3] = K6[3];
    K.a[2] = K.a[6] = K6[4];
    K.a[5] = K.a[7] = K6[5];
    M3<T> D = mul(K, k.E2);
#pragma unroll
    for (int q = 0; q < 9; q++) D.a[q] += K.a[q] + k.E2.a[q];
    T vol = T(0.5) * m.kappa * xp_minus_log(k.Jm1);
    T iso = T(0.5) * m.mu * k.Jm23 * iso_excess(D);  // mu/2 (tr Cbar_e - 3), det C_e = J^2
    return vol + iso;
}

}  // namespace tl
