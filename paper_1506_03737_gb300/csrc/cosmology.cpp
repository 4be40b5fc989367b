// Host FP64 background cosmology of the library: growth factors, Kick-Drift coefficients and
// the BBKS linear power spectrum normalised to sigma_8.
//
// Units H0 = 1, Mpc/h. Flat LCDM: E(a) = sqrt(Om a^-3 + 1 - Om).
// Growth (the exact 2LPT growth factors that §2.1's Eq. eq:2LPTgrowth approximates):
//   d/da (a^3 E D1') = 1.5 Om D1 / (a^2 E),   d/da (a^3 E D2') = 1.5 Om (D2 - D1^2) / (a^2 E),
// integrated in ln a with classical RK4 from the growing mode at a = 1e-5 and normalised to
// D1(1) = 1. The momentum per unit LPT displacement is P = a^3 E dD/da.
// Kick-Drift (§2.3) with p = a^3 E dx/da, dp/da = 1.5 Om F / (a^2 E):
//   Quinn:    kick = 1.5 Om int da/(a^2 E) over [a_{i-1/2}, a_{i+1/2}],  drift = int da/(a^3 E)
//   modified: kick = 1.5 Om (a_{i+1/2}^n - a_{i-1/2}^n) / (n a_i^(n-1)) / (a_i^2 E_i),
//             drift = a_{i+1/2}^-n int a^(n-3)/E da over [a_i, a_{i+1}]   (Eq. eq:modifiedt)
#include "cosmology.h"

#include <cmath>

namespace colapm {

static double hubble(double a, double om) { return std::sqrt(om / (a * a * a) + 1.0 - om); }

// RK4 in ln a from 1e-5 to `a`, returns unnormalised (D1, P1, D2, P2).
static void growth_raw(double a, double om, double y[4]) {
    const int steps = 8192;
    const double l0 = std::log(1e-5), l1 = std::log(a), h = (l1 - l0) / steps;
    auto rhs = [om](double lna, const double* v, double* d) {
        const double x = std::exp(lna), e = hubble(x, om);
        d[0] = v[1] / (x * x * e);
        d[1] = 1.5 * om * v[0] / (x * e);
        d[2] = v[3] / (x * x * e);
        d[3] = 1.5 * om * (v[2] - v[0] * v[0]) / (x * e);
    };
    const double a0 = 1e-5, e0 = hubble(a0, om);
    y[0] = a0;
    y[1] = a0 * a0 * a0 * e0;
    y[2] = -3.0 / 7.0 * a0 * a0;
    y[3] = a0 * a0 * a0 * e0 * (-6.0 / 7.0 * a0);
    double lna = l0;
    for (int s = 0; s < steps; ++s) {
        double k1[4], k2[4], k3[4], k4[4], t[4];
        rhs(lna, y, k1);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k1[i];
        rhs(lna + 0.5 * h, t, k2);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k2[i];
        rhs(lna + 0.5 * h, t, k3);
        for (int i = 0; i < 4; ++i) t[i] = y[i] + h * k3[i];
        rhs(lna + h, t, k4);
        for (int i = 0; i < 4; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        lna += h;
    }
}

Growth growth_at(double a, double om) {
    double y[4], y1[4];
    growth_raw(a, om, y);
    growth_raw(1.0, om, y1);
    const double n = y1[0];
    return Growth{y[0] / n, y[2] / (n * n), y[1] / n, y[3] / (n * n)};
}

// Composite 5-point Gauss-Legendre on `panels` equal panels.
template <typename F>
static double integrate(F f, double lo, double hi, int panels = 256) {
    static const double x[5] = {0.0, -0.5384693101056831, 0.5384693101056831, -0.9061798459386640,
                                0.9061798459386640};
    static const double w[5] = {0.5688888888888889, 0.4786286704993665, 0.4786286704993665, 0.2369268850561891,
                                0.2369268850561891};
    const double h = (hi - lo) / panels;
    double s = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double c = lo + (p + 0.5) * h;
        double q = 0.0;
        for (int i = 0; i < 5; ++i) q += w[i] * f(c + 0.5 * h * x[i]);
        s += 0.5 * h * q;
    }
    return s;
}

static double kick_coef(double lo, double hi, double af, double om, int stepping, double n) {
    double k;
    if (stepping == 1) {
        k = integrate([om](double x) { return 1.0 / (x * x * hubble(x, om)); }, lo, hi);
    } else {
        k = (std::pow(hi, n) - std::pow(lo, n)) / (n * std::pow(af, n - 1.0)) / (af * af * hubble(af, om));
    }
    return 1.5 * om * k;
}

double comoving_distance(double a, double om) {
    if (a >= 1.0) return 0.0;
    return 2997.92458 * integrate([om](double x) { return 1.0 / (x * x * hubble(x, om)); }, a, 1.0, 1024);
}

double drift_coef(double a0, double a1, double am, double om, int stepping, double n) {
    if (stepping == 1) return integrate([om](double x) { return 1.0 / (x * x * x * hubble(x, om)); }, a0, a1);
    return std::pow(am, -n) * integrate([om, n](double x) { return std::pow(x, n - 3.0) / hubble(x, om); }, a0, a1);
}

StepTable make_step_table(double om, double z_init, double z_final, int n_steps, int spacing, int stepping,
                          double nlpt) {
    StepTable t;
    const double a0 = 1.0 / (1.0 + z_init), an = 1.0 / (1.0 + z_final);
    t.a.resize(n_steps + 1);
    for (int i = 0; i <= n_steps; ++i) {
        const double f = (double)i / n_steps;
        t.a[i] = spacing == 1 ? a0 * std::pow(an / a0, f) : a0 + (an - a0) * f;
    }
    t.g.resize(n_steps + 1);
    for (int i = 0; i <= n_steps; ++i) t.g[i] = growth_at(t.a[i], om);
    t.kick.resize(n_steps);
    t.drift.resize(n_steps);
    for (int i = 0; i < n_steps; ++i) {
        const double ah = 0.5 * (t.a[i] + t.a[i + 1]);
        const double alo = i == 0 ? t.a[0] : 0.5 * (t.a[i - 1] + t.a[i]);
        t.kick[i] = kick_coef(alo, ah, t.a[i], om, stepping, nlpt);
        t.drift[i] = drift_coef(t.a[i], t.a[i + 1], ah, om, stepping, nlpt);
    }
    const double ahl = 0.5 * (t.a[n_steps - 1] + t.a[n_steps]);
    t.kick_final = kick_coef(ahl, t.a[n_steps], t.a[n_steps], om, stepping, nlpt);
    return t;
}

double growth_matter_era(double om) {
    double y[4];
    growth_raw(1.0, om, y);
    return y[0];   // D1(1) with D1 = a deep in matter domination
}

// BBKS transfer function, q = k / (Om h).
double bbks(double k, double om, double h) {
    const double q = k / (om * h);
    if (q < 1e-12) return 1.0;
    const double x = 2.34 * q;
    const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    return std::log1p(x) / x * std::pow(poly, -0.25);
}

static double tophat(double x) {
    if (std::fabs(x) < 1e-3) return 1.0 - x * x / 10.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

LinearPk::LinearPk(double om, double h, double ns, double sigma8) : om_(om), h_(h), ns_(ns), amp_(1.0) {
    // sigma^2(8) = (1/2pi^2) int k^3 P W^2(8k) dln k, composite Simpson in ln k over [1e-5, 1e2].
    const int n = 1 << 16;
    const double l0 = std::log(1e-5), l1 = std::log(1e2), dh = (l1 - l0) / n;
    double s = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double k = std::exp(l0 + i * dh);
        const double w = tophat(8.0 * k);
        const double f = k * k * k * shape(k) * w * w;
        s += f * (i == 0 || i == n ? 1.0 : (i % 2 ? 4.0 : 2.0));
    }
    const double s2 = s * dh / 3.0 / (2.0 * M_PI * M_PI);
    amp_ = sigma8 * sigma8 / s2;
}

double LinearPk::shape(double k) const {
    const double t = bbks(k, om_, h_);
    return std::pow(k, ns_) * t * t;
}

double LinearPk::operator()(double k) const { return amp_ * shape(k); }

}  // namespace colapm
