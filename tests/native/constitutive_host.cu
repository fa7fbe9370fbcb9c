// Host build of the library's constitutive device code (csrc/constitutive.cuh) so that
// tests can compare it with the FP64 oracle on the CPU, without a GPU.
#include "../../paper_2602_15149_b300/csrc/constitutive.cuh"

using namespace tl;

template <typename T> static MatT<T> mat(double E, double nu, double sy0, double Hh) {
    MatT<T> m{};
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
    m.model = 3;
    m.mu = (T)mu;
    m.kappa = (T)(lam + 2.0 * mu / 3.0);
    m.lam = (T)lam;
    m.sy0 = (T)sy0;
    m.Hh = (T)Hh;
    return m;
}

template <typename T>
static int j2(const double *G, const double *K6, double ep, double E, double nu, double sy0, double Hh, double *K6o,
              double *epo, double *S, double *dg) {
    M3<T> g;
    for (int q = 0; q < 9; q++) g.a[q] = (T)G[q];
    T k6[6], k6o[6], e, d;
    for (int q = 0; q < 6; q++) k6[q] = (T)K6[q];
    Kin<T> kin = kinematics(g);
    M3<T> s;
    int st = j2_update(kin, k6, (T)ep, mat<T>(E, nu, sy0, Hh), k6o, e, s, d);
    for (int q = 0; q < 6; q++) K6o[q] = k6o[q];
    for (int q = 0; q < 9; q++) S[q] = s.a[q];
    *epo = e;
    *dg = d;
    return st;
}

template <typename T>
static void nh(const double *G, double sphase, double E, double nu, double *S, double *pp, double *pm) {
    M3<T> g;
    for (int q = 0; q < 9; q++) g.a[q] = (T)G[q];
    MatT<T> m = mat<T>(E, nu, 0.0, 0.0);
    m.model = 2;
    Kin<T> kin = kinematics(g);
    M3<T> s;
    T a, b;
    nh_stress(kin, (T)sphase, m, s, a, b);
    for (int q = 0; q < 9; q++) S[q] = s.a[q];
    *pp = a;
    *pm = b;
}

template <typename T, int DIM>
static void svk(const double *G, double sphase, double E, double nu, double *S, double *pp, double *pm) {
    M3<T> g;
    for (int q = 0; q < 9; q++) g.a[q] = (T)G[q];
    MatT<T> m = mat<T>(E, nu, 0.0, 0.0);
    m.model = 1;
    Kin<T> kin = kinematics(g);
    M3<T> s;
    T a, b;
    svk_stress<T, DIM>(kin, (T)sphase, m, s, a, b);
    for (int q = 0; q < 9; q++) S[q] = s.a[q];
    *pp = a;
    *pm = b;
}

extern "C" {
void hc_svk(int prec, int dim, const double *G, double s, double E, double nu, double *S, double *pp, double *pm) {
    if (prec == 64) {
        if (dim == 3) svk<double, 3>(G, s, E, nu, S, pp, pm);
        else svk<double, 2>(G, s, E, nu, S, pp, pm);
    } else {
        if (dim == 3) svk<float, 3>(G, s, E, nu, S, pp, pm);
        else svk<float, 2>(G, s, E, nu, S, pp, pm);
    }
}
int hc_j2_d(const double *G, const double *K6, double ep, double E, double nu, double sy0, double Hh, double *K6o,
            double *epo, double *S, double *dg) {
    return j2<double>(G, K6, ep, E, nu, sy0, Hh, K6o, epo, S, dg);
}
int hc_j2_f(const double *G, const double *K6, double ep, double E, double nu, double sy0, double Hh, double *K6o,
            double *epo, double *S, double *dg) {
    return j2<float>(G, K6, ep, E, nu, sy0, Hh, K6o, epo, S, dg);
}
void hc_nh_d(const double *G, double s, double E, double nu, double *S, double *pp, double *pm) {
    nh<double>(G, s, E, nu, S, pp, pm);
}
void hc_nh_f(const double *G, double s, double E, double nu, double *S, double *pp, double *pm) {
    nh<float>(G, s, E, nu, S, pp, pm);
}
}
