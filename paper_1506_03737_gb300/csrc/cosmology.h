// Host FP64 cosmology of the library (see cosmology.cpp).
#pragma once

#include <vector>

namespace colapm {

struct Growth {
    double d1, d2, p1, p2;   // D1, D2 and P = a^3 E dD/da
};

Growth growth_at(double a, double om);

// D1(a = 1) normalised to D1 = a in matter domination (the growth of the primordial potential's
// density from the matter era to z = 0).
double growth_matter_era(double om);

// Drift coefficient over [a0, a1] with the momentum taken at am (§2.3): Quinn (stepping 1) or
// modified with n = nLPT (stepping 0).
double drift_coef(double a0, double a1, double am, double om, int stepping, double n);

// Comoving distance to scale factor a, R_L(a) = (c / H0) int_a^1 da' / (a'^2 E(a')), Mpc/h (§6).
double comoving_distance(double a, double om);

// BBKS (1986) transfer function, Gamma = om h, k in h/Mpc.
double bbks(double k, double om, double h);

struct StepTable {
    std::vector<double> a;       // a_0 .. a_N
    std::vector<Growth> g;       // growth at a_i
    std::vector<double> kick;    // 1.5 Om x kick integral, step i
    std::vector<double> drift;   // drift integral, step i
    double kick_final = 0.0;     // closing half kick to a_N
};

// spacing: 0 linear in a, 1 logarithmic; stepping: 0 modified (nlpt), 1 Quinn.
StepTable make_step_table(double om, double z_init, double z_final, int n_steps, int spacing, int stepping,
                          double nlpt);

class LinearPk {
  public:
    LinearPk(double om, double h, double ns, double sigma8);
    double operator()(double k) const;   // (Mpc/h)^3 at z = 0, k in h/Mpc

  private:
    double shape(double k) const;
    double om_, h_, ns_, amp_;
};

}  // namespace colapm
