// Host-side description of one simulated system (internal to the library): the SOG
// decomposition, box and cell geometry, device constants and sampling tables, shared by
// the single-system context and the batch of systems.
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "common.cuh"
#include "sog_host.h"

namespace rbsog {

struct HostSystem {
    rbsog_params p{};
    uint32_t N = 0;
    double lam = 0, kT = 0, a_ws = 0, V = 0, Q2 = 0, qsum = 0, S = 0, Ufar0 = 0, Uself = 0, Fhat0 = 0;
    SogDecomp sog;
    Box box{};
    NearConsts nconsts{};
    Yterms y{};                          // the kernel's Yukawa terms (one, or two for EGS)
    std::vector<double> sA, sb;          // Fhat(k) = sum_m A_m exp(-k^2 / (4 b_m)), b_m = e^{t_m}
    // sampling tables (alias tables of the Gaussian mixture and of each axis)
    std::vector<double> mix_prob, ax_prob;
    std::vector<int> mix_alias, ax_off, ax_nmax, ax_alias;
};

// Validate parameters and build everything host-side (no device work).  Returns an
// RBSOG_* status and a message.
// Alias "keep" thresholds in integer form: for the 53-bit integer U of a uniform draw
// u = U 2^-53, u < prob exactly when U < ceil(prob 2^53), so the device decides with an
// integer compare (no FP64 operation) and the same outcome.
inline std::vector<unsigned long long> alias_thresholds(const std::vector<double> &prob) {
    std::vector<unsigned long long> t(prob.size());
    for (size_t i = 0; i < prob.size(); ++i) t[i] = (unsigned long long)std::ceil(prob[i] * 9007199254740992.0);
    return t;
}

int setup_system(const rbsog_params &p, int64_t N, const double *q, const double *m, HostSystem *hs,
                 std::string *err);

// The sampler's signed far-field transform: with two Yukawa terms (EGS) Fhat may change
// sign, so coef carries Fhat / Fhat_env; with one term it is positive and nfh = 0.
template <class Args>
inline void fill_signed_fhat(const Yterms &y, const std::vector<double> &sA, const std::vector<double> &sb,
                             Args *a) {
    a->nfh = y.n > 1 ? (int)sA.size() : 0;
    for (int i = 0; i < a->nfh; ++i) {
        a->fA[i] = sA[i];
        a->finv4b[i] = 1.0 / (4.0 * sb[i]);
    }
}
// S = sum_{k != 0} calF(k) Fhat(k) by a device lattice sum (synchronous).
int system_S(HostSystem *hs, std::string *err);

}  // namespace rbsog
