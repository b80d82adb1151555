// Host-side construction of the C1 sum-of-Gaussians decomposition (Algorithm 1).
#pragma once

#include <string>

namespace rbsog {

struct SogDecomp {
    double lam = 0, rc = 0, eps = 0;
    double h = 0, t0 = 0, w = 1;   // t_m = t0 + m h, weight w on m = M2 (Eq. 37)
    int M1 = 0, M2 = 0;
    int mtot() const { return M1 + M2 + 1; }
};

// mode: 0 minimal, 1 bound, 2 table (M1, M2 given).  Returns false with a message on failure.
bool build_sog(double lam, double rc, double eps, int mode, int M1, int M2, SogDecomp *out, std::string *err);

// Pieces of Eq. (1) and Eq. (37) used by the host to derive device constants.
double sog_f(double t, double r, double lam);
double sog_far(const SogDecomp &s, double r);
double sog_max_error(const SogDecomp &s);

}  // namespace rbsog
