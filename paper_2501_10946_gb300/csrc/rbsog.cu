// C ABI of the RBSOG force step on GB300: context, initialisation and the step sequence.
//
// One force evaluation (Algorithm 2, steps "draw", "far force", "near force"):
//   bin -> scan -> scatter/sort -> gather      cell list in cell-sorted order
//   sample                                     P modes from P(k) (Eq. 59)
//   near                                       Eq. (55) first term
//   rho -> rho_final                           rho(k_l), U*_F (Eq. 60)
//   far (+ closing half kick)                  Eq. (60) force, total force
//   energy                                     Eq. (49) terms and kinetic energy
// rbsog_step captures this sequence once as a CUDA graph (with the opening half kick
// and drift fused into "bin") and replays it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/rbsog.h"
#include "common.cuh"
#include "kernels.h"
#include "sog_host.h"
#include "system.h"

using namespace rbsog;

struct rbsog_ctx {
    rbsog_params p{};
    uint32_t N = 0;
    int prec = 1;
    std::string err;
    SogDecomp sog;
    double lam = 0, kT = 0, a_ws = 0, V = 0, Q2 = 0, qsum = 0, S = 0, Ufar0 = 0, Uself = 0, Fhat0 = 0;
    Box box{};
    NearConsts nconsts{};
    std::vector<double> sA, sb;   // Fhat coefficients A_m (signed, with the term weights) and b_m
    Yterms y{};                   // the kernel's Yukawa terms
    // device buffers
    State rest{}, work{};
    double *q_user = nullptr, *invm_user = nullptr;   // caller-order charges and 1/m
    uint32_t *pos = nullptr;       // place in the rest order of each caller index
    bool pos_valid = false;        // pos belongs to the current rest order
    double *stage_a = nullptr, *stage_b = nullptr, *stage_c = nullptr;
    void *F = nullptr, *Fn = nullptr, *rec_w = nullptr, *rec_id = nullptr, *rec = nullptr;   // records: work, id, cell order
    uint32_t *cell = nullptr, *slot = nullptr, *count = nullptr, *tile_sums = nullptr, *cell_start = nullptr;
    unsigned long long *keys = nullptr;
    unsigned long long *mix_thr = nullptr, *ax_thr = nullptr;
    int *mix_alias = nullptr, *ax_off = nullptr, *ax_nmax = nullptr, *ax_alias = nullptr;
    int *modes = nullptr, *inject_m = nullptr;
    double *coef = nullptr;
    double2 *partial = nullptr, *rho = nullptr, *rho_wsum = nullptr;
    unsigned int *rho_wdone = nullptr;
    void *gtab = nullptr;
    double *Ufar = nullptr, *U_part = nullptr, *K_part = nullptr, *energy = nullptr, *escratch = nullptr;
    unsigned int *edone = nullptr;
    int G = 0, nU = 0, nK = 0;
    DevCounters *ctr = nullptr;
    std::vector<void *> allocs;
    cudaStream_t cap_stream = nullptr;
    // the structure factor runs beside the near field on this stream inside a step
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_bin = nullptr, ev_join = nullptr;
    // rbsog_step_get: the positions' read-back runs on dl_stream from ev_sorted (recorded
    // after the cell sort of the last step, when enqueue is given it) while the forces
    // are computed; ev_dl marks the inverse order ready for the velocities and forces
    cudaStream_t dl_stream = nullptr;
    cudaEvent_t ev_sorted = nullptr, ev_dl = nullptr;
    bool mark_sorted = false;
    cudaGraphExec_t graph = nullptr;
    bool force_valid = false;
    bool energy_valid = false;     // the energy partials belong to the current state
    uint32_t n_owned = 0;          // particles 0 .. n_owned-1 enter rho (domain decomposition)
    bool partial_done = false;     // rbsog_forces_partial ran; rbsog_forces_complete may follow
    SamplerTables tab{};
    // Metropolis-Hastings chains (RBSOG_SAMPLER_MH)
    bool mh = false;
    int *mh_m = nullptr;
    unsigned long long *mh_t = nullptr;
    // instantaneous temperature (RBSOG_KT_INSTANT): kinetic-energy partials of k_bin, the
    // distinct |k|^2 of the mode support with their weights, and {k_B T V, S, k_B T}
    bool instT = false;
    double *Kb_part = nullptr, *shell_k2 = nullptr, *shell_W = nullptr, *temp_part = nullptr, *temp_out = nullptr;
    unsigned int *temp_done = nullptr;
    int nshell = 0;
    // profiling: events around each kernel group of eager force evaluations
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> prof_spans;   // (group, (start ev, end ev))
};

static std::string g_init_error;

namespace rbsog {
// message for rbsog_last_error(NULL) from calls that have no context
void set_global_error(const std::string &msg) { g_init_error = msg; }
}  // namespace rbsog

namespace {

const double kPi = 3.14159265358979323846;


// Vose's alias method, both work lists used as stacks filled in ascending index order.
void vose(const std::vector<double> &w, std::vector<double> *prob, std::vector<int> *alias) {
    const int n = (int)w.size();
    double total = 0.0;
    for (double x : w) total += x;
    std::vector<double> sc(n);
    for (int i = 0; i < n; ++i) sc[i] = (w[i] * n) / total;
    prob->assign(n, 0.0);
    alias->resize(n);
    for (int i = 0; i < n; ++i) (*alias)[i] = i;
    std::vector<int> small, large;
    for (int i = 0; i < n; ++i) (sc[i] < 1.0 ? small : large).push_back(i);
    while (!small.empty() && !large.empty()) {
        int lo = small.back(); small.pop_back();
        int g = large.back(); large.pop_back();
        (*prob)[lo] = sc[lo];
        (*alias)[lo] = g;
        sc[g] = (sc[g] + sc[lo]) - 1.0;
        (sc[g] < 1.0 ? small : large).push_back(g);
    }
    while (!large.empty()) { (*prob)[large.back()] = 1.0; large.pop_back(); }
    while (!small.empty()) { (*prob)[small.back()] = 1.0; small.pop_back(); }
}


}  // namespace

namespace rbsog {

int setup_system(const rbsog_params &p, int64_t N, const double *q_host, const double *m_host, HostSystem *hs,
                 std::string *err) {
    auto bad = [&](int code, const char *msg) {
        *err = msg;
        return code;
    };
    if (!q_host || !m_host) return bad(RBSOG_EINVAL, "q or m is NULL");
    if (N < 2 || N > 0x7fffffffLL) return bad(RBSOG_EINVAL, "N must be in [2, 2^31)");
    for (int d = 0; d < 3; ++d)
        if (!(p.box[d] > 0)) return bad(RBSOG_EINVAL, "box lengths must be > 0");
    if (!(p.kappa > 0)) return bad(RBSOG_EINVAL, "kappa must be > 0");
    if (p.P < 1 || p.P > 4096) return bad(RBSOG_EINVAL, "P must be in [1, 4096]");
    if (p.precision != RBSOG_FP64 && p.precision != RBSOG_FP32) return bad(RBSOG_EINVAL, "bad precision");
    if (p.ensemble != RBSOG_NVE && p.ensemble != RBSOG_LANGEVIN) return bad(RBSOG_EINVAL, "bad ensemble");
    if (p.sog_mode < 0 || p.sog_mode > 2) return bad(RBSOG_EINVAL, "bad sog_mode");
    if (p.sampling < 0 || p.sampling > 3) return bad(RBSOG_EINVAL, "bad sampling measure");
    const double Lmin = std::fmin(p.box[0], std::fmin(p.box[1], p.box[2]));
    if (!(p.r_c > 0) || p.r_c > 0.5 * Lmin) return bad(RBSOG_EINVAL, "need 0 < r_c <= min(L)/2");
    if (!(p.dt >= 0)) return bad(RBSOG_EINVAL, "dt must be >= 0");
    for (int64_t i = 0; i < N; ++i)
        if (!(m_host[i] > 0) || !std::isfinite(q_host[i])) return bad(RBSOG_EINVAL, "masses must be > 0");
    HostSystem &h = *hs;
    h.p = p;
    h.N = (uint32_t)N;
    h.V = (p.box[0] * p.box[1]) * p.box[2];
    h.a_ws = p.a_ws > 0 ? p.a_ws : std::cbrt(3.0 * h.V / (4.0 * kPi * (double)N));
    h.lam = h.a_ws / p.kappa;
    h.kT = p.kT > 0 ? p.kT : 1.0 / (h.a_ws * p.Gamma);
    if (!(h.kT > 0) || !std::isfinite(h.kT)) return bad(RBSOG_EINVAL, "k_B T must be > 0 (Gamma > 0 or kT > 0)");
    // Yukawa terms: the kernel itself, or the two of the EGS screening (Sec. 1), whose
    // transform 4 pi / (k^2 eps(k)) splits by partial fractions as 4 pi [B / (k^2 + beta) +
    // A / (k^2 + alpha)], alpha, beta = 2 (1 +- s) / (nu lambda^2), s = sqrt(1 - nu),
    // B = (1 + s) / (2 s), A = -(1 - s) / (2 s); each term has its own SOG decomposition
    const double nu = p.egs_nu;
    if (!(nu >= 0.0 && nu <= 0.96)) return bad(RBSOG_EINVAL, "egs_nu must be in [0, 0.96]");
    if (nu > 0.0 && p.sog_mode == RBSOG_SOG_TABLE)
        return bad(RBSOG_EINVAL, "the EGS screening takes sog_mode MINIMAL or BOUND");
    int nterms = 1;
    double yc[2] = {1.0, 0.0}, ylam[2] = {h.lam, h.lam};
    if (nu > 0.0) {
        const double s = std::sqrt(1.0 - nu);
        const double beta = 2.0 * (1.0 - s) / (nu * h.lam * h.lam);
        const double alpha = 2.0 * (1.0 + s) / (nu * h.lam * h.lam);
        yc[0] = (1.0 + s) / (2.0 * s);
        ylam[0] = 1.0 / std::sqrt(beta);
        yc[1] = -(1.0 - s) / (2.0 * s);
        ylam[1] = 1.0 / std::sqrt(alpha);
        nterms = 2;
    }
    SogDecomp sogs[2];
    int mt = 0;
    for (int k = 0; k < nterms; ++k) {
        if (!build_sog(ylam[k], p.r_c, p.sog_eps, p.sog_mode, p.sog_M1, p.sog_M2, &sogs[k], err))
            return RBSOG_ENOCONV;
        mt += sogs[k].mtot();
    }
    h.sog = sogs[0];
    if (mt > kMaxGauss) return bad(RBSOG_EUNSUPPORTED, "more than 40 Gaussians");
    h.y.n = nterms;
    for (int k = 0; k < 2; ++k) {
        h.y.c[k] = yc[k];
        h.y.inv_lam2[k] = 1.0 / (ylam[k] * ylam[k]);
    }
    h.Q2 = 0.0;
    h.qsum = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        h.Q2 += q_host[i] * q_host[i];
        h.qsum += q_host[i];
    }
    if (!(h.Q2 > 0)) return bad(RBSOG_EINVAL, "all charges are zero");
    // the context's own sum for the self energy; the whole system's for calF, S and the
    // k = 0 term when the context holds one domain of it
    const double Q2_own = h.Q2;
    if (!(p.q2_total >= 0.0)) return bad(RBSOG_EINVAL, "q2_total must be >= 0");
    if (p.q2_total > 0.0) {
        h.Q2 = p.q2_total;
        h.qsum = p.qsum_total;
    }
    // box and cells
    Box &bx = h.box;
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        bx.L[d] = p.box[d];
        bx.invL[d] = 1.0 / p.box[d];
        bx.invL32[d] = bx.invL[d] * 4294967296.0;
        int n = (int)std::floor(p.box[d] / p.r_c);
        bx.nc[d] = n >= 3 ? n : 1;
        ncell *= bx.nc[d];
        bx.L_2m32[d] = p.box[d] * 2.3283064365386963e-10;
        bx.L_2m64[d] = p.box[d] * 5.421010862427522e-20;
        bx.L_2m32f[d] = (float)bx.L_2m32[d];
        bx.tpl[d] = 6.283185307179586 / p.box[d];
    }
    if (ncell > (1LL << 28)) return bad(RBSOG_EINVAL, "too many cells (box / r_c too large)");
    bx.ncell = (int)ncell;
    // SOG constants (Eqs. 37, 54, 56-57)
    const double log2e = 1.4426950408889634;
    NearConsts &nc = h.nconsts;
    nc.mtot = mt;
    nc.inv_lam = 1.0 / ylam[0];
    nc.rc2 = p.r_c * p.r_c;
    nc.inv_lam_log2e_f = (float)(log2e / ylam[0]);
    nc.inv_lam_f = (float)(1.0 / ylam[0]);
    nc.rc2_f = (float)nc.rc2;
    nc.y1 = yc[0];
    nc.ly1_f = (float)std::log2(yc[0]);
    nc.two = nterms > 1 ? 1 : 0;
    nc.y2 = yc[1];
    nc.inv_lam2 = 1.0 / ylam[1];
    nc.ly2_f = nterms > 1 ? (float)std::log2(std::fabs(yc[1])) : 0.f;
    nc.sgn2_f = yc[1] < 0.0 ? -1.f : 1.f;
    nc.inv_lam2_log2e_f = (float)(log2e / ylam[1]);
    nc.inv_lam2_f = (float)(1.0 / ylam[1]);
    h.Fhat0 = 0.0;
    h.sA.clear();
    h.sb.clear();
    double F0 = 0.0;
    int gi = 0;
    for (int k = 0; k < nterms; ++k) {
        const SogDecomp &sg = sogs[k];
        for (int m = -sg.M1; m <= sg.M2; ++m, ++gi) {
            const double t = sg.t0 + m * sg.h;
            const double w = (m == sg.M2) ? sg.w : 1.0;
            const double b = std::exp(t);
            const double f0 = sog_f(t, 0.0, ylam[k]);
            const double a = yc[k] * (sg.h * w * f0);     // the term's weight times Eq. (37)'s
            nc.a[gi] = a;
            nc.b[gi] = b;
            nc.c[gi] = -2.0 * b * a;
            nc.af[gi] = (float)a;
            nc.bl2f[gi] = (float)(b * log2e);
            nc.cf[gi] = (float)(-2.0 * b * a);
            const double A = yc[k] * (sg.h * w * std::pow(kPi, 1.5) * f0 * std::exp(-1.5 * t));
            h.sA.push_back(A);
            h.sb.push_back(b);
            h.Fhat0 += A;
            F0 += a;
        }
    }
    h.Uself = -0.5 * Q2_own * F0;
    h.Ufar0 = h.Fhat0 * h.qsum * h.qsum / (2.0 * h.V);
    // sampling tables (Eq. 59): the measure's mixture of separable components.  calF of
    // Eq. (62) and calF = 1 draw from Fhat (component m: Gaussian m, plain per-axis tables;
    // Eq. 62 adds a rejection step); calF = k^2 uses k^2 Fhat = sum_m sum_a k_a^2 (...):
    // component 3m + a has a k_a^2-weighted table on axis a and plain tables elsewhere.
    const double LN_1E18 = 41.44653167389282;
    std::vector<double> mixw;
    h.ax_off.clear();
    h.ax_nmax.clear();
    h.ax_prob.clear();
    h.ax_alias.clear();
    auto add_table = [&](const std::vector<double> &w, int *off) {
        std::vector<double> pr;
        std::vector<int> al;
        vose(w, &pr, &al);
        *off = (int)h.ax_prob.size();
        h.ax_prob.insert(h.ax_prob.end(), pr.begin(), pr.end());
        h.ax_alias.insert(h.ax_alias.end(), al.begin(), al.end());
    };
    for (int i = 0; i < mt; ++i) {
        const double b = h.sb[i];
        int off_plain[3], off_sq[3], nmax[3];
        double theta[3], sigma[3];
        for (int a = 0; a < 3; ++a) {
            const int nm = (int)std::ceil(std::sqrt(4.0 * b * LN_1E18) / bx.tpl[a]);
            std::vector<double> g(2 * nm + 1), g2(2 * nm + 1);
            for (int n = -nm; n <= nm; ++n) {
                const double kk = bx.tpl[a] * n;
                const double e = std::exp(-(kk * kk) / (4.0 * b));
                g[n + nm] = e;
                g2[n + nm] = (kk * kk) * e;
            }
            double th = 0.0, sg = 0.0;
            for (double x : g) th += x;
            for (double x : g2) sg += x;
            nmax[a] = nm;
            theta[a] = th;
            sigma[a] = sg;
            add_table(g, &off_plain[a]);
            if (p.sampling == RBSOG_SAMPLING_K2) add_table(g2, &off_sq[a]);
        }
        if (p.sampling == RBSOG_SAMPLING_K2) {
            for (int a = 0; a < 3; ++a) {
                double w = std::fabs(h.sA[i]) * sigma[a];
                for (int c = 0; c < 3; ++c) {
                    if (c != a) w = w * theta[c];
                    h.ax_off.push_back(c == a ? off_sq[c] : off_plain[c]);
                    h.ax_nmax.push_back(nmax[c]);
                }
                mixw.push_back(w);
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                h.ax_off.push_back(off_plain[c]);
                h.ax_nmax.push_back(nmax[c]);
            }
            mixw.push_back(std::fabs(h.sA[i]) * ((theta[0] * theta[1]) * theta[2]));
        }
    }
    vose(mixw, &h.mix_prob, &h.mix_alias);
    return RBSOG_OK;
}

int system_S(HostSystem *hs, std::string *err) {
    HostSystem &h = *hs;
    SArgs a{};
    a.mtot = (int)h.sA.size();
    double bmax = 0.0;
    for (int i = 0; i < a.mtot; ++i) {
        a.A[i] = std::fabs(h.sA[i]);     // the envelope of the far field's transform
        a.inv4b[i] = 1.0 / (4.0 * h.sb[i]);
        if (h.sb[i] > bmax) bmax = h.sb[i];
    }
    a.kmax2 = 4.0 * bmax * std::log(1e17);
    for (int d = 0; d < 3; ++d) {
        a.tpl[d] = h.box.tpl[d];
        a.nmax[d] = (int)std::floor(std::sqrt(a.kmax2) / h.box.tpl[d]) + 1;
    }
    a.kTV = h.kT * h.V;
    a.Q2 = h.Q2;
    a.y = h.y;
    a.measure = h.p.sampling;
    const int nb = 2 * a.nmax[0] + 1;
    double *parts = nullptr;
    cudaError_t e = cudaMalloc(&parts, nb * sizeof(double));
    if (e != cudaSuccess) {
        *err = std::string("CUDA error in alloc S: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? RBSOG_ENOMEM : RBSOG_ECUDA;
    }
    launch_S(a, parts, 0);
    std::vector<double> hv(nb);
    e = cudaMemcpy(hv.data(), parts, nb * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(parts);
    if (e != cudaSuccess) {
        *err = std::string("CUDA error in S kernel: ") + cudaGetErrorString(e);
        return RBSOG_ECUDA;
    }
    double S = 0.0;
    for (double x : hv) S += x;
    h.S = S;
    return RBSOG_OK;
}

// The distinct |k|^2 of the mode support (k != 0, |k|^2 <= kmax2 of system_S) with weights
// W = (number of modes) x Fhat_env(k), so that S(T) = sum_j calF(k2_j; T) W_j.  Axes of equal
// length are grouped, and a mode's key is the sum of m_a^2 over each group (one integer
// |m|^2 for a cubic box), so modes related by sign changes and by permutations of equal
// axes share one entry.  Sorted by k2.
int shell_table(const HostSystem &h, std::vector<double> *k2out, std::vector<double> *Wout, std::string *err) {
    double bmax = 0.0;
    for (double b : h.sb) bmax = std::max(bmax, b);
    const double kmax2 = 4.0 * bmax * std::log(1e17);
    int grp[3] = {0, 0, 0}, ng = 1;
    const double *L = h.box.L;
    grp[1] = (L[1] == L[0]) ? 0 : ng++;
    grp[2] = (L[2] == L[0]) ? 0 : ((L[2] == L[1]) ? grp[1] : ng++);
    double tpl2[3];
    int nmax[3];
    for (int d = 0; d < 3; ++d) {
        tpl2[grp[d]] = h.box.tpl[d] * h.box.tpl[d];
        nmax[d] = (int)std::floor(std::sqrt(kmax2) / h.box.tpl[d]) + 1;
    }
    const unsigned long long B = (unsigned long long)3 * (unsigned long long)nmax[0] * nmax[0] +
                                 3ull * nmax[1] * nmax[1] + 3ull * nmax[2] * nmax[2] + 1ull;
    if ((double)B * (double)B * (double)B > 1.8e19) {
        *err = "instantaneous temperature: the mode support is too large for the |k|^2 table";
        return RBSOG_EUNSUPPORTED;
    }
    std::unordered_map<unsigned long long, double> cnt;
    for (int mx = 0; mx <= nmax[0]; ++mx) {
        const double kx = h.box.tpl[0] * mx;
        for (int my = 0; my <= nmax[1]; ++my) {
            const double ky = h.box.tpl[1] * my;
            for (int mz = 0; mz <= nmax[2]; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                const double kz = h.box.tpl[2] * mz;
                if (kx * kx + ky * ky + kz * kz > kmax2) break;
                unsigned long long key[3] = {0, 0, 0};
                key[grp[0]] += (unsigned long long)mx * mx;
                key[grp[1]] += (unsigned long long)my * my;
                key[grp[2]] += (unsigned long long)mz * mz;
                const double mult = (mx ? 2.0 : 1.0) * (my ? 2.0 : 1.0) * (mz ? 2.0 : 1.0);
                cnt[key[0] + B * (key[1] + B * key[2])] += mult;
            }
            if (cnt.size() > (1u << 22)) {
                *err = "instantaneous temperature: more than 2^22 distinct |k|^2 (box too large or too anisotropic)";
                return RBSOG_EUNSUPPORTED;
            }
        }
    }
    std::vector<std::pair<double, double>> ent;
    ent.reserve(cnt.size());
    for (const auto &kv : cnt) {
        unsigned long long k = kv.first;
        double k2 = 0.0;
        for (int g = 0; g < ng; ++g) {
            k2 += tpl2[g] * (double)(k % B);
            k /= B;
        }
        double fe = 0.0;
        for (size_t i = 0; i < h.sA.size(); ++i) fe += std::fabs(h.sA[i]) * std::exp(-k2 / (4.0 * h.sb[i]));
        ent.push_back({k2, kv.second * fe});
    }
    std::sort(ent.begin(), ent.end());
    k2out->resize(ent.size());
    Wout->resize(ent.size());
    for (size_t j = 0; j < ent.size(); ++j) {
        (*k2out)[j] = ent[j].first;
        (*Wout)[j] = ent[j].second;
    }
    return RBSOG_OK;
}

}  // namespace rbsog

namespace {

int fail(rbsog_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return code;
}

int cuda_fail(rbsog_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? RBSOG_ENOMEM : RBSOG_ECUDA, m);
}

#define CK(call, where)                                    \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

template <typename T>
cudaError_t dalloc(rbsog_ctx *c, T **ptr, size_t count) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e == cudaSuccess) {
        c->allocs.push_back(p);
        *ptr = (T *)p;
    }
    return e;
}

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The address a kernel reads or writes ptr through: ptr for device and managed memory,
// the mapped device address of pinned host memory, nullptr for memory the device cannot
// address (pageable host memory goes through a staging buffer and a copy).
template <typename T>
T *device_view(T *ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return ptr;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) return (T *)at.devicePointer;
    return nullptr;
}

// pos for the current rest order, computed once per order (a state upload and every force
// evaluation reorder the particles)
void ensure_pos(rbsog_ctx *c, cudaStream_t st) {
    if (c->pos_valid) return;
    launch_rest_pos(c->rest.id, c->N, c->pos, st);
    c->pos_valid = true;
}

int build_sampler(rbsog_ctx *c, const HostSystem &hs) {
    const int mt = (int)hs.mix_prob.size();   // mixture components
    const std::vector<unsigned long long> mp = alias_thresholds(hs.mix_prob), axp = alias_thresholds(hs.ax_prob);
    const std::vector<int> &ma = hs.mix_alias, &off = hs.ax_off, &nmax = hs.ax_nmax, &axa = hs.ax_alias;
    CK(dalloc(c, &c->mix_thr, mt), "alloc sampler");
    CK(dalloc(c, &c->mix_alias, mt), "alloc sampler");
    CK(dalloc(c, &c->ax_off, 3 * mt), "alloc sampler");
    CK(dalloc(c, &c->ax_nmax, 3 * mt), "alloc sampler");
    CK(dalloc(c, &c->ax_thr, axp.size()), "alloc sampler");
    CK(dalloc(c, &c->ax_alias, axa.size()), "alloc sampler");
    CK(cudaMemcpy(c->mix_thr, mp.data(), mt * sizeof(unsigned long long), cudaMemcpyHostToDevice), "upload sampler");
    CK(cudaMemcpy(c->mix_alias, ma.data(), mt * sizeof(int), cudaMemcpyHostToDevice), "upload sampler");
    CK(cudaMemcpy(c->ax_off, off.data(), 3 * mt * sizeof(int), cudaMemcpyHostToDevice), "upload sampler");
    CK(cudaMemcpy(c->ax_nmax, nmax.data(), 3 * mt * sizeof(int), cudaMemcpyHostToDevice), "upload sampler");
    CK(cudaMemcpy(c->ax_thr, axp.data(), axp.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice),
       "upload sampler");
    CK(cudaMemcpy(c->ax_alias, axa.data(), axa.size() * sizeof(int), cudaMemcpyHostToDevice), "upload sampler");
    c->tab = SamplerTables{mt, c->mix_thr, c->mix_alias, c->ax_off, c->ax_nmax, c->ax_thr, c->ax_alias};
    return RBSOG_OK;
}

const char *kProfNames[RBSOG_NPROF] = {"bin", "scan", "sort", "gather", "sample", "near", "rho", "rho_final",
                                       "far", "close"};

// Record a profiling boundary on st (no-op unless profiling); returns the event index.
size_t prof_mark(rbsog_ctx *c, cudaStream_t st) {
    if (!c->prof) return 0;
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return 0;
        c->ev_pool.push_back(e);
    }
    cudaEventRecord(c->ev_pool[c->ev_used], st);
    return c->ev_used++;
}

struct ProfScope {
    rbsog_ctx *c;
    cudaStream_t st;
    int group;
    size_t e0;
    ProfScope(rbsog_ctx *c_, cudaStream_t st_, int g) : c(c_), st(st_), group(g), e0(prof_mark(c_, st_)) {}
    ~ProfScope() {
        if (c->prof) c->prof_spans.push_back({group, {e0, prof_mark(c, st)}});
    }
};

// Enqueue one force evaluation (and, with integrate != 0, one full step).
// part = 1: stop after the structure factor (the first half of a domain's evaluation)
int enqueue(rbsog_ctx *c, cudaStream_t st, int integrate, double *F_user, double *Fn_user, double *Ff_user,
            int advance, int part = 0) {
    c->pos_valid = false;   // the cell sort reorders the particles
    const int prec = c->prec;
    const uint32_t N = c->N;
    BinArgs b{};
    b.in = c->rest; b.out = c->work; b.F = c->F; b.integrate = integrate;
    b.dt = c->p.dt; b.c1 = std::exp(-c->p.langevin_gamma * c->p.dt); b.kT = c->kT; b.seed = c->p.seed;
    b.okT = (1.0 - b.c1 * b.c1) * b.kT;
    set_bin_floats(b);
    b.ctr = c->ctr; b.N = N; b.stride = N; b.cell_base = 0; b.box = c->box; b.rec_w = c->rec_w; b.rec_id = c->rec_id; b.cell = c->cell;
    b.slot = c->slot; b.count = c->count;
    b.K_part = c->instT ? c->Kb_part : nullptr;
    SampleArgs sa{};
    sa.tab = c->tab; sa.P = c->p.P; sa.seed = c->p.seed;
    for (int d = 0; d < 3; ++d) sa.tpl[d] = c->box.tpl[d];
    sa.A = c->kT * c->V; sa.Q2 = c->Q2; sa.y = c->y; sa.S = c->S; sa.V = c->V;
    fill_signed_fhat(c->y, c->sA, c->sb, &sa);
    sa.measure = c->p.sampling;
    sa.Q2a = c->p.sampling == RBSOG_SAMPLING_DEBYE ? (4.0 * kPi) * c->Q2 : c->Q2;
    sample_set_prefilter(&sa);
    sa.ctr = c->ctr; sa.inject_m = c->inject_m; sa.m_out = c->modes; sa.coef_out = c->coef;
    sa.temp = c->instT ? c->temp_out : nullptr;
    TempArgs ta{};
    ta.K_part = c->Kb_part; ta.nK = (int)((N + 255) / 256); ta.two_3N = 2.0 / (3.0 * (double)N);
    ta.V = c->V; ta.Q2 = c->Q2; ta.y = c->y; ta.measure = c->p.sampling;
    ta.k2 = c->shell_k2; ta.W = c->shell_W; ta.n = c->nshell;
    ta.part = c->temp_part; ta.done = c->temp_done; ta.out = c->temp_out;
    MHChainArgs mc{};
    mc.m = c->mh_m; mc.t = c->mh_t;
    mc.sweeps = c->p.mh_sweeps > 0 ? c->p.mh_sweeps : 1;
    mc.burnin = c->p.mh_burnin == 0 ? 64 : (c->p.mh_burnin < 0 ? 0 : c->p.mh_burnin);
    // the k-sample: temperature first when calF takes the instantaneous one (it needs the
    // kinetic energy k_bin leaves), then the i.i.d. draw or the chains
    auto sample = [&](cudaStream_t s2) {
        if (c->instT) launch_temperature(ta, s2);
        if (c->mh) launch_sample_mh(sa, mc, s2);
        else launch_sample(sa, s2);
    };
    RhoArgs ra{};
    ra.rec = c->rec_id; ra.N = c->n_owned; ra.m = c->modes; ra.P = c->p.P; ra.partial = c->partial; ra.G = c->G;
    RhoFinalArgs rf{};
    rf.partial = c->partial; rf.G = c->G; rf.P = c->p.P; rf.m = c->modes; rf.coef = c->coef;
    for (int d = 0; d < 3; ++d) rf.tpl[d] = c->box.tpl[d];
    rf.rho = c->rho; rf.gtab = c->gtab; rf.Ufar = c->Ufar; rf.ctr = c->ctr;
    rf.wsum = c->rho_wsum; rf.wdone = c->rho_wdone;
    // The structure factor needs the particle records (in id order) and the k-sample, not
    // the cell list: outside profiling the sample runs on a side stream from the start of
    // the step, and rho and rho_final follow there as soon as k_bin has written the
    // records, beside the rest of the cell list and the near field (special-function unit
    // against integer, memory and FMA work); far waits for both streams.  Profiling keeps
    // one stream so every group's events time that group alone.
    const bool fork = !c->prof;
    cudaStream_t sr = st;
    if (fork) {
        if (cudaEventRecord(c->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "fork the structure-factor stream");
        sr = c->side_stream;
        if (!c->instT) sample(sr);
    }
    { ProfScope ps(c, st, 0); launch_bin(prec, b, st); }
    if (fork) {
        if (cudaEventRecord(c->ev_bin, st) != cudaSuccess || cudaStreamWaitEvent(sr, c->ev_bin, 0) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "hand the records to the structure-factor stream");
        if (c->instT) sample(sr);
        launch_rho(prec, ra, sr);
        launch_rho_final(prec, rf, sr);
    }
    { ProfScope ps(c, st, 1); launch_scan(c->count, c->tile_sums, c->cell_start, c->box.ncell, N, st); }
    {
        ProfScope ps(c, st, 2);
        launch_scatter(c->cell, c->slot, c->cell_start, c->work.id, N, c->keys, st);
    }
    GatherArgs g{};
    g.in = c->work; g.out = c->rest; g.keys = c->keys; g.cell = c->cell; g.cell_start = c->cell_start; g.ctr = c->ctr;
    g.c_off = nullptr; g.R = 1; g.rec_w = c->rec_w; g.rec = c->rec; g.N = N;
    { ProfScope ps(c, st, 3); launch_gather(prec, g, st); }
    if (c->mark_sorted && cudaEventRecord(c->ev_sorted, st) != cudaSuccess)
        return fail(c, RBSOG_ECUDA, "record the sorted state");
    if (!fork) { ProfScope ps(c, st, 4); sample(st); }
    NearArgs na{};
    na.nc = c->nconsts; na.rec = c->rec; na.cell_start = c->cell_start; na.box = c->box; na.N = N; na.stride = N;
    na.Fn = c->Fn;
    na.U_part = c->U_part;
    na.ctr = c->ctr;
    { ProfScope ps(c, st, 5); c->nU = launch_near(prec, na, st); }
    if (fork) {
        if (cudaEventRecord(c->ev_join, sr) != cudaSuccess || cudaStreamWaitEvent(st, c->ev_join, 0) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "join the structure-factor stream");
    } else {
        { ProfScope ps(c, st, 6); launch_rho(prec, ra, st); }
        { ProfScope ps(c, st, 7); launch_rho_final(prec, rf, st); }
    }
    if (part) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
        return RBSOG_OK;
    }
    FarArgs fa{};
    fa.rec = c->rec; fa.N = N; fa.stride = N; fa.P = c->p.P; fa.gtab = c->gtab; fa.m = c->modes; fa.Fn = c->Fn; fa.F = c->F;
    fa.st = c->rest; fa.integrate = integrate ? 1 : 0; fa.dt = c->p.dt; fa.K_part = c->K_part;
    fa.F_user = F_user; fa.Fn_user = Fn_user; fa.Ff_user = Ff_user; fa.ctr = c->ctr;
    { ProfScope ps(c, st, 8); c->nK = launch_far(prec, fa, st); }
    { ProfScope ps(c, st, 9); launch_close_eval(c->ctr, advance, st); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    c->energy_valid = true;
    return RBSOG_OK;
}

int check_device_errors(rbsog_ctx *c) {
    DevCounters h;
    CK(cudaMemcpy(&h, c->ctr, sizeof h, cudaMemcpyDeviceToHost), "read device status");
    if (h.err & kErrCellOverflow) return fail(c, RBSOG_EOVERFLOW, "a cell holds more than 4096 particles");
    if (h.err & kErrSampler) return fail(c, RBSOG_ETIMEOUT, "k-sampler exceeded its attempt limit");
    if (h.err & kErrNearStage) return fail(c, RBSOG_ETIMEOUT, "near-field staging wait exceeded its limit");
    return RBSOG_OK;
}

// The energies of the last force evaluation: its near, kinetic and per-mode partials
// reduced in a fixed order (k_energy), then read back.  Synchronous.
int read_energy(rbsog_ctx *c, rbsog_energy *e, cudaStream_t st) {
    if (!c->energy_valid)
        return fail(c, RBSOG_EINVAL, "no force evaluation since the last state upload: no energies to read");
    EnergyArgs ea{};
    ea.U_part = c->U_part; ea.nU = c->nU; ea.K_part = c->K_part; ea.nK = c->nK; ea.Ufar = c->Ufar;
    ea.nUfar = c->p.P;
    ea.Ufar0 = c->Ufar0; ea.Uself = c->Uself; ea.out = c->energy; ea.ctr = c->ctr;
    ea.scratch = c->escratch; ea.done = c->edone;
    launch_energy(ea, st);
    CK(cudaGetLastError(), "energy reduction");
    double h[5];
    CK(cudaMemcpyAsync(h, c->energy, sizeof h, cudaMemcpyDeviceToHost, st), "read energy");
    DevCounters hc;
    CK(cudaMemcpyAsync(&hc, c->ctr, sizeof hc, cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "synchronize");
    e->U_near = h[0]; e->U_far = h[1]; e->U_self = h[2]; e->kinetic = h[3]; e->total = h[4];
    e->step = hc.step;
    return check_device_errors(c);
}

}  // namespace

extern "C" {

int rbsog_init(const rbsog_params *params, int64_t N, const double *q_host, const double *m_host, rbsog_ctx **out) {
    if (!out) return fail(nullptr, RBSOG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !q_host || !m_host) return fail(nullptr, RBSOG_EINVAL, "params, q or m is NULL");
    const rbsog_params &p = *params;
    HostSystem hs;
    {
        std::string err;
        const int code = setup_system(p, N, q_host, m_host, &hs, &err);
        if (code != RBSOG_OK) return fail(nullptr, code, err);
    }
    if (p.sampler != RBSOG_SAMPLER_IID && p.sampler != RBSOG_SAMPLER_MH)
        return fail(nullptr, RBSOG_EINVAL, "bad sampler");
    if (p.temperature != RBSOG_KT_TARGET && p.temperature != RBSOG_KT_INSTANT)
        return fail(nullptr, RBSOG_EINVAL, "bad temperature source");
    if (p.sampler == RBSOG_SAMPLER_MH && hs.y.n != 1)
        return fail(nullptr, RBSOG_EUNSUPPORTED, "the Metropolis-Hastings sampler takes the Yukawa kernel (egs_nu = 0)");
    if (p.mh_sweeps < 0) return fail(nullptr, RBSOG_EINVAL, "mh_sweeps must be >= 0");
    std::vector<double> shell_k2, shell_W;
    const bool instT = p.temperature == RBSOG_KT_INSTANT &&
                       (p.sampling == RBSOG_SAMPLING_ADAPTIVE || p.sampling == RBSOG_SAMPLING_DEBYE);
    if (instT) {
        std::string err;
        const int code = shell_table(hs, &shell_k2, &shell_W, &err);
        if (code != RBSOG_OK) return fail(nullptr, code, err);
    }
    rbsog_ctx *c = new rbsog_ctx();
    c->p = p;
    c->mh = p.sampler == RBSOG_SAMPLER_MH;
    c->n_owned = (uint32_t)N;
    c->instT = instT;
    c->nshell = (int)shell_k2.size();
    c->N = (uint32_t)N;
    c->prec = p.precision;
    c->V = hs.V; c->a_ws = hs.a_ws; c->lam = hs.lam; c->kT = hs.kT; c->Q2 = hs.Q2; c->qsum = hs.qsum;
    c->sog = hs.sog; c->box = hs.box; c->nconsts = hs.nconsts; c->sA = hs.sA; c->sb = hs.sb; c->y = hs.y;
    c->Fhat0 = hs.Fhat0; c->Uself = hs.Uself; c->Ufar0 = hs.Ufar0;
    const Box &bx = c->box;

    // device
    int r = RBSOG_OK;
    auto bail = [&](int code) {
        rbsog_free(c);
        return code;
    };
    if (cudaSetDevice(p.device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, RBSOG_ECUDA, "cudaSetDevice failed (no usable CUDA device)");
    }
    const size_t n = c->N, n3 = 3 * n;
    const size_t real = c->prec == RBSOG_FP32 ? 4 : 8;
    State *sts[2] = {&c->rest, &c->work};
    for (State *s : sts) {
        if (dalloc(c, &s->rx, n) || dalloc(c, &s->ry, n) || dalloc(c, &s->rz, n) || dalloc(c, &s->vx, n) ||
            dalloc(c, &s->vy, n) || dalloc(c, &s->vz, n) || dalloc(c, &s->invm, n) || dalloc(c, &s->q, n) ||
            dalloc(c, &s->id, n)) {
            g_init_error = "device allocation failed (state)";
            return bail(RBSOG_ENOMEM);
        }
    }
    unsigned char *Fb = nullptr, *Fnb = nullptr, *recwb = nullptr, *recib = nullptr, *recb = nullptr;
    const int ntiles = (bx.ncell + kScanTile - 1) / kScanTile;
    c->G = rho_blocks(c->prec, c->N, p.P);
    const size_t gtab_bytes = (size_t)p.P * 64;
    if (dalloc(c, &c->q_user, n) || dalloc(c, &c->invm_user, n) || dalloc(c, &c->pos, n) || dalloc(c, &c->stage_a, n3) ||
        dalloc(c, &c->stage_b, n3) || dalloc(c, &c->stage_c, n3) || dalloc(c, &Fb, n3 * real) ||
        dalloc(c, &Fnb, n3 * real) || dalloc(c, &recwb, n * 4 * real) || dalloc(c, &recib, n * 4 * real) || dalloc(c, &recb, n * 4 * real) ||
        dalloc(c, &c->cell, n) || dalloc(c, &c->slot, n) || dalloc(c, &c->count, (size_t)bx.ncell) ||
        dalloc(c, &c->tile_sums, (size_t)ntiles) || dalloc(c, &c->cell_start, (size_t)bx.ncell + 1) ||
        dalloc(c, &c->keys, n) || dalloc(c, &c->modes, 3 * (size_t)p.P) ||
        dalloc(c, &c->inject_m, 3 * (size_t)p.P) || dalloc(c, &c->coef, (size_t)p.P) ||
        dalloc(c, &c->partial, (size_t)c->G * 8 * p.P) || dalloc(c, &c->rho, (size_t)p.P) ||
        dalloc(c, &c->rho_wsum, 8 * (size_t)p.P) || dalloc(c, &c->rho_wdone, ((size_t)p.P + 31) / 32) ||
        cudaMemset(c->rho_wdone, 0, sizeof(unsigned int) * (((size_t)p.P + 31) / 32)) != cudaSuccess ||
        dalloc(c, (unsigned char **)&c->gtab, gtab_bytes) || dalloc(c, &c->Ufar, (size_t)p.P) ||
        dalloc(c, &c->U_part, 8 * std::max((n + 127) / 128, (size_t)bx.ncell) + 8) || dalloc(c, &c->K_part, (n + 255) / 256 + 1) ||
        dalloc(c, &c->energy, 8) || dalloc(c, &c->escratch, 3 * (size_t)kEnergyBlocks) || dalloc(c, &c->edone, 1) ||
        dalloc(c, &c->ctr, 1)) {
        g_init_error = "device allocation failed";
        return bail(RBSOG_ENOMEM);
    }
    c->F = Fb; c->Fn = Fnb; c->rec_w = recwb; c->rec_id = recib; c->rec = recb;
    if (c->mh) {
        if (dalloc(c, &c->mh_m, 3 * (size_t)p.P) || dalloc(c, &c->mh_t, (size_t)p.P) ||
            cudaMemset(c->mh_m, 0, 3 * sizeof(int) * (size_t)p.P) != cudaSuccess ||
            cudaMemset(c->mh_t, 0, sizeof(unsigned long long) * (size_t)p.P) != cudaSuccess) {
            g_init_error = "device allocation failed (sampler chains)";
            return bail(RBSOG_ENOMEM);
        }
    }
    if (c->instT) {
        const size_t ns = shell_k2.size();
        if (dalloc(c, &c->Kb_part, (n + 255) / 256) || dalloc(c, &c->shell_k2, ns) || dalloc(c, &c->shell_W, ns) ||
            dalloc(c, &c->temp_part, (size_t)kTempBlocks) || dalloc(c, &c->temp_out, 3) ||
            dalloc(c, &c->temp_done, 1) || cudaMemset(c->temp_done, 0, sizeof(unsigned int)) != cudaSuccess ||
            cudaMemcpy(c->shell_k2, shell_k2.data(), ns * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->shell_W, shell_W.data(), ns * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            g_init_error = "device allocation failed (temperature table)";
            return bail(RBSOG_ENOMEM);
        }
    }
    std::vector<double> invm_host(n);
    for (size_t i = 0; i < n; ++i) invm_host[i] = 1.0 / m_host[i];
    if (cudaMemset(c->count, 0, sizeof(uint32_t) * bx.ncell) != cudaSuccess ||
        cudaMemset(c->ctr, 0, sizeof(DevCounters)) != cudaSuccess ||
        cudaMemset(c->edone, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemcpy(c->q_user, q_host, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->invm_user, invm_host.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->dl_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_sorted, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_dl, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_bin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        g_init_error = "device initialisation failed";
        return bail(RBSOG_ECUDA);
    }
    if ((r = build_sampler(c, hs)) != RBSOG_OK) {
        g_init_error = c->err;
        return bail(r);
    }
    {
        std::string err;
        if ((r = system_S(&hs, &err)) != RBSOG_OK) {
            g_init_error = err;
            return bail(r);
        }
        c->S = hs.S;
    }
    if (c->instT) {
        // until the first evaluation: the target temperature
        const double t0[3] = {c->kT * c->V, c->S, c->kT};
        if (cudaMemcpy(c->temp_out, t0, sizeof t0, cudaMemcpyHostToDevice) != cudaSuccess) {
            g_init_error = "device initialisation failed";
            return bail(RBSOG_ECUDA);
        }
    }
    // a valid (zero) state so every call is defined before rbsog_set_state
    if (cudaMemset(c->stage_a, 0, n3 * sizeof(double)) != cudaSuccess) {
        g_init_error = "device initialisation failed";
        return bail(RBSOG_ECUDA);
    }
    launch_set_state(c->stage_a, nullptr, c->q_user, c->invm_user, c->rest, c->N, c->box, c->ctr, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        g_init_error = "device initialisation failed";
        return bail(RBSOG_ECUDA);
    }
    *out = c;
    return RBSOG_OK;
}

// Caller buffers: device memory and pinned host memory are read and written by the kernels
// themselves (the latter through its mapped address, in whole lines over the host link);
// other host memory goes through a staging buffer and a copy.
int rbsog_set_state(rbsog_ctx *c, const double *r, const double *v, void *stream) {
    if (!c || !r) return fail(c, RBSOG_EINVAL, "ctx or r is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)c->N * sizeof(double);
    const double *rd = device_view(r), *vd = v ? device_view(v) : nullptr;
    if (!rd) {
        CK(cudaMemcpyAsync(c->stage_a, r, bytes, cudaMemcpyDefault, st), "copy r");
        rd = c->stage_a;
    }
    if (v && !vd) {
        CK(cudaMemcpyAsync(c->stage_b, v, bytes, cudaMemcpyDefault, st), "copy v");
        vd = c->stage_b;
    }
    launch_set_state(rd, vd, c->q_user, c->invm_user, c->rest, c->N, c->box, c->ctr, st);
    CK(cudaGetLastError(), "set_state");
    c->force_valid = false;
    c->energy_valid = false;
    c->partial_done = false;
    c->pos_valid = false;
    return RBSOG_OK;
}

int rbsog_set_state_forces(rbsog_ctx *c, const double *r, const double *v, const double *F, void *stream) {
    if (int code = rbsog_set_state(c, r, v, stream)) return code;
    if (!F) return RBSOG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double *Fd = device_view(F);
    if (!Fd) {
        CK(cudaMemcpyAsync(c->stage_c, F, 3 * (size_t)c->N * sizeof(double), cudaMemcpyDefault, st), "copy F");
        Fd = c->stage_c;
    }
    launch_set_forces(c->prec, Fd, c->F, c->N, c->ctr, st);
    CK(cudaGetLastError(), "set forces");
    c->force_valid = true;
    return RBSOG_OK;
}

int rbsog_get_forces(rbsog_ctx *c, double *F, void *stream) {
    if (!c || !F) return fail(c, RBSOG_EINVAL, "ctx or F is NULL");
    if (!c->force_valid) return fail(c, RBSOG_EINVAL, "no forces at the current state yet");
    cudaStream_t st = (cudaStream_t)stream;
    double *Fv = device_view(F);
    double *Fd = Fv ? Fv : c->stage_c;
    ensure_pos(c, st);
    launch_get_forces(c->prec, c->pos, c->F, c->N, Fd, st);
    CK(cudaGetLastError(), "get forces");
    if (!Fv) CK(cudaMemcpyAsync(F, Fd, 3 * (size_t)c->N * sizeof(double), cudaMemcpyDefault, st), "copy F out");
    CK(cudaStreamSynchronize(st), "synchronize");
    return check_device_errors(c);
}

int rbsog_set_state_forces_f32(rbsog_ctx *c, const double *r, const double *v, const float *F, void *stream) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    if (c->prec != RBSOG_FP32) return fail(c, RBSOG_EINVAL, "FP32 forces need precision RBSOG_FP32");
    if (int code = rbsog_set_state(c, r, v, stream)) return code;
    if (!F) return RBSOG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const float *Fd = device_view(F);
    if (!Fd) {
        CK(cudaMemcpyAsync(c->stage_c, F, 3 * (size_t)c->N * sizeof(float), cudaMemcpyDefault, st), "copy F");
        Fd = (const float *)c->stage_c;
    }
    launch_set_forces_f32(Fd, (float *)c->F, c->N, c->ctr, st);
    CK(cudaGetLastError(), "set forces");
    c->force_valid = true;
    return RBSOG_OK;
}

int rbsog_get_forces_f32(rbsog_ctx *c, float *F, void *stream) {
    if (!c || !F) return fail(c, RBSOG_EINVAL, "ctx or F is NULL");
    if (c->prec != RBSOG_FP32) return fail(c, RBSOG_EINVAL, "FP32 forces need precision RBSOG_FP32");
    if (!c->force_valid) return fail(c, RBSOG_EINVAL, "no forces at the current state yet");
    cudaStream_t st = (cudaStream_t)stream;
    float *Fv = device_view(F);
    float *Fd = Fv ? Fv : (float *)c->stage_c;
    ensure_pos(c, st);
    launch_get_forces_f32(c->pos, (const float *)c->F, c->N, Fd, st);
    CK(cudaGetLastError(), "get forces");
    if (!Fv) CK(cudaMemcpyAsync(F, Fd, 3 * (size_t)c->N * sizeof(float), cudaMemcpyDefault, st), "copy F out");
    CK(cudaStreamSynchronize(st), "synchronize");
    return check_device_errors(c);
}

int rbsog_get_state(rbsog_ctx *c, double *r, double *v, uint64_t *step, void *stream) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)c->N * sizeof(double);
    double *rv = r ? device_view(r) : nullptr, *vv = v ? device_view(v) : nullptr;
    double *rd = r ? (rv ? rv : c->stage_a) : nullptr, *vd = v ? (vv ? vv : c->stage_b) : nullptr;
    ensure_pos(c, st);
    launch_get_state(c->rest, c->pos, c->N, rd, vd, st);
    CK(cudaGetLastError(), "get_state");
    if (r && !rv) CK(cudaMemcpyAsync(r, rd, bytes, cudaMemcpyDefault, st), "copy r out");
    if (v && !vv) CK(cudaMemcpyAsync(v, vd, bytes, cudaMemcpyDefault, st), "copy v out");
    DevCounters hc;
    CK(cudaMemcpyAsync(&hc, c->ctr, sizeof hc, cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (step) *step = hc.step;
    return check_device_errors(c);
}

static int forces_impl(rbsog_ctx *c, double *F, double *Fn, double *Ff, rbsog_energy *e, void *stream) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)c->N * sizeof(double);
    double *outs[3] = {F, Fn, Ff};
    double *stage[3] = {c->stage_a, c->stage_b, c->stage_c};
    double *dev[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i)
        if (outs[i]) dev[i] = is_device_ptr(outs[i]) ? outs[i] : stage[i];
    int r = enqueue(c, st, 0, dev[0], dev[1], dev[2], 0);
    if (r) return r;
    c->force_valid = true;
    for (int i = 0; i < 3; ++i)
        if (outs[i] && dev[i] != outs[i])
            CK(cudaMemcpyAsync(outs[i], dev[i], bytes, cudaMemcpyDefault, st), "copy forces out");
    if (e) return read_energy(c, e, st);
    for (int i = 0; i < 3; ++i)
        if (outs[i] && dev[i] != outs[i]) CK(cudaStreamSynchronize(st), "synchronize");
    return RBSOG_OK;
}

int rbsog_forces(rbsog_ctx *c, double *F, rbsog_energy *e, void *stream) {
    return forces_impl(c, F, nullptr, nullptr, e, stream);
}

int rbsog_forces_split(rbsog_ctx *c, double *F_near, double *F_far, rbsog_energy *e, void *stream) {
    return forces_impl(c, nullptr, F_near, F_far, e, stream);
}

int rbsog_step(rbsog_ctx *c, int32_t nsteps, rbsog_energy *e, void *stream) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(c, RBSOG_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->force_valid && nsteps > 0) {
        int r = enqueue(c, st, 0, nullptr, nullptr, nullptr, 0);
        if (r) return r;
        c->force_valid = true;
    }
    if (c->prof) {
        const int mode = c->p.ensemble == RBSOG_LANGEVIN ? 2 : 1;
        for (int i = 0; i < nsteps; ++i) {
            int r = enqueue(c, st, mode, nullptr, nullptr, nullptr, 1);
            if (r) return r;
        }
        if (e) return read_energy(c, e, st);
        return RBSOG_OK;
    }
    if (nsteps > 0 && !c->graph) {
        const int mode = c->p.ensemble == RBSOG_LANGEVIN ? 2 : 1;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int r = enqueue(c, c->cap_stream, mode, nullptr, nullptr, nullptr, 1);
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
        if (r) return r;
        CK(e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        CK(e3, "graph instantiate");
    }
    if (nsteps > 0) c->pos_valid = false;
    for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(c->graph, st), "graph launch");
    if (e) return read_energy(c, e, st);
    return RBSOG_OK;
}

int rbsog_step_get(rbsog_ctx *c, int32_t nsteps, double *r, double *v, void *F, int32_t f32, rbsog_energy *e,
                   void *stream) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    if (nsteps < 1) return fail(c, RBSOG_EINVAL, "nsteps < 1");
    if (F && f32 && c->prec != RBSOG_FP32) return fail(c, RBSOG_EINVAL, "FP32 forces need precision RBSOG_FP32");
    cudaStream_t st = (cudaStream_t)stream;
    if (nsteps > 1)
        if (int code = rbsog_step(c, nsteps - 1, nullptr, stream)) return code;
    if (!c->force_valid) {
        if (int code = enqueue(c, st, 0, nullptr, nullptr, nullptr, 0)) return code;
        c->force_valid = true;
    }
    // the last step launched one kernel at a time, with an event once the cell sort has
    // put the new positions in their final order
    const int mode = c->p.ensemble == RBSOG_LANGEVIN ? 2 : 1;
    c->mark_sorted = true;
    const int code = enqueue(c, st, mode, nullptr, nullptr, nullptr, 1);
    c->mark_sorted = false;
    if (code) return code;
    const size_t N = c->N;
    // positions (final after the sort) and the inverse order, beside the force kernels;
    // the copy engine moves them so that no SM is taken from the forces
    cudaStream_t dl = c->dl_stream;
    CK(cudaStreamWaitEvent(dl, c->ev_sorted, 0), "wait for the sorted state");
    launch_rest_pos(c->rest.id, c->N, c->pos, dl);
    if (r) {
        double *rv = device_view(r);
        const bool dev = rv && is_device_ptr(r);
        launch_get_state(c->rest, c->pos, c->N, dev ? rv : c->stage_a, nullptr, dl);
        if (!dev) CK(cudaMemcpyAsync(r, c->stage_a, 3 * N * sizeof(double), cudaMemcpyDefault, dl), "copy r out");
    }
    CK(cudaGetLastError(), "positions read-back");
    CK(cudaEventRecord(c->ev_dl, dl), "positions read-back");
    CK(cudaStreamWaitEvent(st, c->ev_dl, 0), "join the read-back");
    c->pos_valid = true;
    // velocities (final after the closing kick) and forces, after the step
    if (v) {
        double *vv = device_view(v);
        launch_get_state(c->rest, c->pos, c->N, nullptr, vv ? vv : c->stage_b, st);
        if (!vv) CK(cudaMemcpyAsync(v, c->stage_b, 3 * N * sizeof(double), cudaMemcpyDefault, st), "copy v out");
    }
    if (F) {
        if (f32) {
            float *Fv = device_view((float *)F);
            float *Fd = Fv ? Fv : (float *)c->stage_c;
            launch_get_forces_f32(c->pos, (const float *)c->F, c->N, Fd, st);
            if (!Fv) CK(cudaMemcpyAsync(F, Fd, 3 * N * sizeof(float), cudaMemcpyDefault, st), "copy F out");
        } else {
            double *Fv = device_view((double *)F);
            double *Fd = Fv ? Fv : c->stage_c;
            launch_get_forces(c->prec, c->pos, c->F, c->N, Fd, st);
            if (!Fv) CK(cudaMemcpyAsync(F, Fd, 3 * N * sizeof(double), cudaMemcpyDefault, st), "copy F out");
        }
    }
    CK(cudaGetLastError(), "read-back");
    if (e) return read_energy(c, e, st);
    CK(cudaStreamSynchronize(st), "synchronize");
    return check_device_errors(c);
}

int rbsog_set_owned(rbsog_ctx *c, int64_t n_owned) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    if (n_owned < 1 || n_owned > (int64_t)c->N) return fail(c, RBSOG_EINVAL, "n_owned must be in [1, N]");
    CK(cudaDeviceSynchronize(), "synchronize");
    c->n_owned = (uint32_t)n_owned;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return RBSOG_OK;
}

int rbsog_forces_partial(rbsog_ctx *c, double *rho_partial, void *stream) {
    if (!c || !rho_partial) return fail(c, RBSOG_EINVAL, "ctx or rho_partial is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (int r = enqueue(c, st, 0, nullptr, nullptr, nullptr, 0, 1)) return r;
    CK(cudaMemcpyAsync(rho_partial, c->rho, sizeof(double2) * (size_t)c->p.P, cudaMemcpyDefault, st), "copy rho");
    CK(cudaStreamSynchronize(st), "synchronize");
    c->partial_done = true;
    c->energy_valid = false;
    return check_device_errors(c);
}

int rbsog_forces_complete(rbsog_ctx *c, const double *rho, double *F, void *stream) {
    if (!c || !rho) return fail(c, RBSOG_EINVAL, "ctx or rho is NULL");
    if (!c->partial_done) return fail(c, RBSOG_EINVAL, "rbsog_forces_partial must come first");
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = c->prec;
    const size_t P = (size_t)c->p.P;
    // the summed rho as the only nonzero per-block partial: the fixed-order reduction of
    // rho_final then returns it exactly and builds the gather table and the U*_F terms
    CK(cudaMemsetAsync(c->partial, 0, sizeof(double2) * (size_t)c->G * 8 * P, st), "clear partials");
    CK(cudaMemcpyAsync(c->partial, rho, sizeof(double2) * P, cudaMemcpyDefault, st), "copy rho");
    RhoFinalArgs rf{};
    rf.partial = c->partial; rf.G = c->G; rf.P = c->p.P; rf.m = c->modes; rf.coef = c->coef;
    for (int d = 0; d < 3; ++d) rf.tpl[d] = c->box.tpl[d];
    rf.rho = c->rho; rf.gtab = c->gtab; rf.Ufar = c->Ufar; rf.ctr = c->ctr; rf.keep_draw = 1;
    rf.wsum = c->rho_wsum; rf.wdone = c->rho_wdone;
    launch_rho_final(prec, rf, st);
    const size_t bytes = 3 * (size_t)c->N * sizeof(double);
    double *Fd = nullptr;
    if (F) Fd = is_device_ptr(F) ? F : c->stage_a;
    FarArgs fa{};
    fa.rec = c->rec; fa.N = c->N; fa.stride = c->N; fa.P = c->p.P; fa.gtab = c->gtab; fa.m = c->modes; fa.Fn = c->Fn;
    fa.F = c->F; fa.st = c->rest; fa.integrate = 0; fa.dt = c->p.dt; fa.K_part = c->K_part;
    fa.F_user = Fd; fa.ctr = c->ctr;
    c->nK = launch_far(prec, fa, st);
    launch_close_eval(c->ctr, 0, st);
    CK(cudaGetLastError(), "kernel launch");
    if (F && Fd != F) CK(cudaMemcpyAsync(F, Fd, bytes, cudaMemcpyDefault, st), "copy forces out");
    CK(cudaStreamSynchronize(st), "synchronize");
    c->partial_done = false;
    c->force_valid = true;
    c->energy_valid = false;
    return check_device_errors(c);
}

int rbsog_slab_split(int64_t N, const double *r, const double *box, int32_t axis, int32_t nslabs, int32_t slab,
                     double halo, int64_t *idx_out, int64_t *n_owned, int64_t *n_local) {
    if (N < 1 || !r || !box || !idx_out || !n_owned || !n_local) return fail(nullptr, RBSOG_EINVAL, "bad argument");
    if (axis < 0 || axis > 2 || nslabs < 1 || slab < 0 || slab >= nslabs || !(box[axis] > 0) || !(halo >= 0))
        return fail(nullptr, RBSOG_EINVAL, "bad axis, slab count, slab or halo");
    const double L = box[axis], w = L / nslabs;
    if (!(halo <= 0.5 * L)) return fail(nullptr, RBSOG_EINVAL, "halo must be at most half the box");
    const double lo = slab * w, hi = (slab + 1) * w;
    auto wrap = [&](double x) {
        double y = x - L * std::floor(x / L);
        return (y >= L) ? y - L : y;
    };
    // slab of a wrapped coordinate: floor(x / w), clamped for the rounding at the top
    auto slab_of = [&](double x) {
        int k = (int)std::floor(wrap(x) / w);
        return k < 0 ? 0 : (k >= nslabs ? nslabs - 1 : k);
    };
    int64_t no = 0;
    for (int64_t i = 0; i < N; ++i)
        if (slab_of(r[3 * i + axis]) == slab) idx_out[no++] = i;
    int64_t nl = no;
    if (nslabs > 1)
        for (int64_t i = 0; i < N; ++i) {
            const double x = wrap(r[3 * i + axis]);
            if (slab_of(r[3 * i + axis]) == slab) continue;
            // periodic distance from x to the slab interval [lo, hi)
            const double d_lo = std::fmod(lo - x + 2.0 * L, L), d_hi = std::fmod(x - hi + 2.0 * L, L);
            if (std::fmin(d_lo, d_hi) < halo) idx_out[nl++] = i;
        }
    *n_owned = no;
    *n_local = nl;
    return RBSOG_OK;
}

int rbsog_set_ksample(rbsog_ctx *c, const int32_t *m_host, int32_t P) {
    if (!c || !m_host) return fail(c, RBSOG_EINVAL, "ctx or m is NULL");
    if (P != c->p.P) return fail(c, RBSOG_EINVAL, "P differs from the context's P");
    for (int l = 0; l < P; ++l)
        if (m_host[3 * l] == 0 && m_host[3 * l + 1] == 0 && m_host[3 * l + 2] == 0)
            return fail(c, RBSOG_EINVAL, "mode (0,0,0) is not in the sampled support");
    CK(cudaDeviceSynchronize(), "synchronize");
    CK(cudaMemcpy(c->inject_m, m_host, 3 * sizeof(int32_t) * P, cudaMemcpyHostToDevice), "copy modes");
    int one = 1;
    CK(cudaMemcpy(&c->ctr->inject, &one, sizeof(int), cudaMemcpyHostToDevice), "set inject flag");
    return RBSOG_OK;
}

int rbsog_get_ksample(rbsog_ctx *c, int32_t *m_host, double *coef_host) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    CK(cudaDeviceSynchronize(), "synchronize");
    if (m_host) CK(cudaMemcpy(m_host, c->modes, 3 * sizeof(int32_t) * c->p.P, cudaMemcpyDeviceToHost), "copy modes");
    if (coef_host) CK(cudaMemcpy(coef_host, c->coef, sizeof(double) * c->p.P, cudaMemcpyDeviceToHost), "copy coef");
    return check_device_errors(c);
}

int rbsog_get_rho(rbsog_ctx *c, double *rho_host) {
    if (!c || !rho_host) return fail(c, RBSOG_EINVAL, "ctx or rho is NULL");
    CK(cudaDeviceSynchronize(), "synchronize");
    CK(cudaMemcpy(rho_host, c->rho, sizeof(double2) * c->p.P, cudaMemcpyDeviceToHost), "copy rho");
    return RBSOG_OK;
}

int rbsog_get_cells(rbsog_ctx *c, int32_t *nc, uint32_t *cell_start, uint32_t *perm) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    CK(cudaDeviceSynchronize(), "synchronize");
    if (nc) for (int d = 0; d < 3; ++d) nc[d] = c->box.nc[d];
    if (cell_start)
        CK(cudaMemcpy(cell_start, c->cell_start, sizeof(uint32_t) * ((size_t)c->box.ncell + 1), cudaMemcpyDeviceToHost),
           "copy cell_start");
    if (perm) CK(cudaMemcpy(perm, c->rest.id, sizeof(uint32_t) * c->N, cudaMemcpyDeviceToHost), "copy perm");
    return check_device_errors(c);
}

int rbsog_get_temperature(rbsog_ctx *c, double *kT, double *S) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    double v[3] = {c->kT * c->V, c->S, c->kT};
    if (c->instT) {
        CK(cudaDeviceSynchronize(), "synchronize");
        CK(cudaMemcpy(v, c->temp_out, sizeof v, cudaMemcpyDeviceToHost), "copy temperature");
    }
    if (kT) *kT = v[2];
    if (S) *S = v[1];
    return RBSOG_OK;
}

int rbsog_get_sog(rbsog_ctx *c, double *h, double *t0, int32_t *M1, int32_t *M2, double *w, double *lam, double *S) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    if (h) *h = c->sog.h;
    if (t0) *t0 = c->sog.t0;
    if (M1) *M1 = c->sog.M1;
    if (M2) *M2 = c->sog.M2;
    if (w) *w = c->sog.w;
    if (lam) *lam = c->sog.lam;
    if (S) *S = c->S;
    return RBSOG_OK;
}

int rbsog_profile(rbsog_ctx *c, int32_t enable) {
    if (!c) return fail(c, RBSOG_EINVAL, "ctx is NULL");
    CK(cudaDeviceSynchronize(), "synchronize");
    c->prof = enable != 0;
    c->ev_used = 0;
    c->prof_spans.clear();
    return RBSOG_OK;
}

int rbsog_profile_read(rbsog_ctx *c, double *ms, int64_t *launches) {
    if (!c || !ms || !launches) return fail(c, RBSOG_EINVAL, "ctx, ms or launches is NULL");
    CK(cudaDeviceSynchronize(), "synchronize");
    for (int g = 0; g < RBSOG_NPROF; ++g) { ms[g] = 0.0; launches[g] = 0; }
    for (auto &sp : c->prof_spans) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev_pool[sp.second.first], c->ev_pool[sp.second.second]), "event time");
        ms[sp.first] += t;
        launches[sp.first] += 1;
    }
    c->ev_used = 0;
    c->prof_spans.clear();
    return RBSOG_OK;
}

const char *rbsog_profile_name(int32_t group) {
    return (group >= 0 && group < RBSOG_NPROF) ? kProfNames[group] : "";
}

int rbsog_build_sog(double lam, double r_c, double eps, int32_t mode, int32_t M1, int32_t M2, double *out6) {
    if (!out6) return fail(nullptr, RBSOG_EINVAL, "out6 is NULL");
    if (mode < 0 || mode > 2) return fail(nullptr, RBSOG_EINVAL, "bad sog mode");
    SogDecomp s;
    std::string err;
    if (!build_sog(lam, r_c, eps, mode, M1, M2, &s, &err)) return fail(nullptr, RBSOG_ENOCONV, err);
    out6[0] = s.h;
    out6[1] = s.t0;
    out6[2] = (double)s.M1;
    out6[3] = (double)s.M2;
    out6[4] = s.w;
    out6[5] = sog_max_error(s);
    return RBSOG_OK;
}

const char *rbsog_last_error(const rbsog_ctx *c) { return c ? c->err.c_str() : g_init_error.c_str(); }

void rbsog_free(rbsog_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->dl_stream) cudaStreamDestroy(c->dl_stream);
    if (c->ev_sorted) cudaEventDestroy(c->ev_sorted);
    if (c->ev_dl) cudaEventDestroy(c->ev_dl);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_bin) cudaEventDestroy(c->ev_bin);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

}  // extern "C"
