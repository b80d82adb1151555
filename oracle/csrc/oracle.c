/*
 * FP64 CPU oracle for the random batch sum-of-Gaussians (RBSOG) force step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The CUDA product path never
 * calls it; the two share no source, header or table.
 *
 * Everything here is a plain, slow, FP64 restatement of the paper's formulas
 * (Chen, Liang & Xu, "Random batch sum-of-Gaussians algorithm for molecular
 * dynamics simulations of Yukawa systems in three dimensions"):
 *   f(t,r)      Eq. (1)       integrand of the Yukawa integral representation
 *   F(r)        Eq. (37)      C1 sum-of-Gaussians far part, weight w on m = M2
 *   N(r)        Eq. (33)      near part Y - F inside r_c
 *   F_N1, F_N2  Eqs. (55)-(57) near-field pair force and its two pieces
 *   Fhat(k)     Eqs. (53)-(54) Fourier transform of F
 *   rho(k)      Sec. 2        structure factor sum_j q_j exp(i k.r_j)
 *   U*, F*      Eq. (60)      random-batch estimators
 *   calF(k)     Eq. (62)      Debye-Hueckel correction (first term), eps(k) of Eq. (6)
 *
 * The SOG parameters arrive as a double array
 *   sog = { h, t0, M1, M2, w_M2, lambda }.
 * Vectors are [N][3] row-major doubles.  Box lengths are L[3].
 * Build flags keep IEEE semantics: no fast-math, no FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- kernel pieces -------------------------------------------------- */

/* Eq. (1): f(t,r) = pi^{-1/2} exp(-r^2 e^t - 1/(4 lambda^2 e^t) + t/2). */
static double f_tr(double t, double r, double lam) {
    double et = exp(t);
    return exp(-r * r * et - 1.0 / (4.0 * lam * lam * et) + 0.5 * t) / sqrt(M_PI);
}

static double sog_weight(const double *sog, int m) {
    return (m == (int)sog[3]) ? sog[4] : 1.0;
}

/* Eq. (37): F(r) = h [ w f(t_M2, r) + sum_{m=-M1}^{M2-1} f(t_m, r) ]. */
double orc_sog_F(const double *sog, double r) {
    double h = sog[0], t0 = sog[1], lam = sog[5];
    int M1 = (int)sog[2], M2 = (int)sog[3];
    double s = 0.0;
    for (int m = -M1; m <= M2; ++m) s += sog_weight(sog, m) * f_tr(t0 + m * h, r, lam);
    return h * s;
}

/* Yukawa kernel Y(r) = exp(-r/lambda)/r (Sec. 1). */
static double yukawa(double r, double lam) { return exp(-r / lam) / r; }

/* Eq. (56): F_N1(r) = exp(-r/lambda)(1 + r/lambda)/r^3. */
static double force_n1(double r, double lam) {
    return exp(-r / lam) * (1.0 + r / lam) / (r * r * r);
}

/* Eq. (57): F_N2(r) = -2h [ w e^{t_M2} f(t_M2,r) + sum_{m<M2} e^{t_m} f(t_m,r) ]. */
double orc_force_n2(const double *sog, double r) {
    double h = sog[0], t0 = sog[1], lam = sog[5];
    int M1 = (int)sog[2], M2 = (int)sog[3];
    double s = 0.0;
    for (int m = -M1; m <= M2; ++m) {
        double t = t0 + m * h;
        s += sog_weight(sog, m) * exp(t) * f_tr(t, r, lam);
    }
    return -2.0 * h * s;
}

/* Eq. (54): Fhat(k) = pi^{3/2} h sum^# f(t_m,0) exp(-3 t_m/2 - e^{-t_m} k^2/4). */
double orc_fhat(const double *sog, double k2) {
    double h = sog[0], t0 = sog[1], lam = sog[5];
    int M1 = (int)sog[2], M2 = (int)sog[3];
    double s = 0.0;
    for (int m = -M1; m <= M2; ++m) {
        double t = t0 + m * h;
        s += sog_weight(sog, m) * f_tr(t, 0.0, lam) * exp(-1.5 * t - exp(-t) * k2 / 4.0);
    }
    return pow(M_PI, 1.5) * h * s;
}

/* Eq. (62) first term with eps(k) = 1 + (lambda k)^{-2} (Eq. 6):
 * calF(k) = kT V / (kT V / Q2 + eps(k)^{-1} / k^2),  eps^{-1}/k^2 = 1/(k^2 + lambda^{-2}). */
double orc_calF(double k2, double kT, double V, double Q2, double lam) {
    double epsinv_over_k2 = 1.0 / (k2 + 1.0 / (lam * lam));
    return kT * V / (kT * V / Q2 + epsinv_over_k2);
}

/* Correction calF(k) of the sampling measure P(k) = calF Fhat / S (Eq. 59) for the three
 * choices compared in Sec. 5 (Fig. 9): 0 the adaptive Debye-Hueckel form of Eq. (62) as
 * printed, 1 calF = 1 (the Gaussian itself, as in RBE), 2 calF = k^2 (as in Coulomb
 * RBSOG); and 3 Eq. (62) with the Debye wavenumber of Gaussian units, 4 pi sum q^2 / (kT V)
 * in place of sum q^2 / (kT V) (the Debye-Hueckel <|rho|^2> for Fhat ~ 4 pi/(k^2 + 1/lambda^2)). */
double orc_measure(int measure, double k2, double kT, double V, double Q2, double lam) {
    if (measure == 1) return 1.0;
    if (measure == 2) return k2;
    if (measure == 3) {
        double epsinv_over_k2 = 1.0 / (k2 + 1.0 / (lam * lam));
        return kT * V / (kT * V / Q2 + (4.0 * M_PI) * epsinv_over_k2);
    }
    return orc_calF(k2, kT, V, Q2, lam);
}

/* ---- fixed-point coordinates and the cell list ----------------------- */

/* Fractional coordinate of r in [0,1): u = r (1/L) with the reciprocal rounded to
 * double, f = u - floor(u); f == 1 (from rounding of a tiny negative u) is the same
 * point as f == 0. */
static double frac01(double r, double L) {
    double invL = 1.0 / L;
    double u = r * invL;
    double f = u - floor(u);
    if (f >= 1.0) f = 0.0;
    return f;
}

/* s = floor(f * 2^32) (u32) and floor(f * 2^64) (u64) for every coordinate. */
void orc_fixed_point(int64_t N, const double *r, const double *L, uint32_t *s32, uint64_t *s64) {
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double f = frac01(r[3 * i + a], L[a]);
            if (s32) s32[3 * i + a] = (uint32_t)(uint64_t)floor(f * 4294967296.0);
            if (s64) s64[3 * i + a] = (uint64_t)floor(f * 18446744073709551616.0);
        }
}

/* Cell of a particle: c_a = floor(s_a * n_a / 2^32) with s the u32 coordinate;
 * linear index c = c_x + n_x (c_y + n_y c_z).  Stable counting sort: within a
 * cell, particles appear in ascending index. */
void orc_cell_list(int64_t N, const double *r, const double *L, const int *nc,
                   uint32_t *cell_of, uint32_t *cell_start, uint32_t *perm) {
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    uint32_t *s = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)N);
    uint32_t *cursor = (uint32_t *)calloc((size_t)ncell, sizeof(uint32_t));
    orc_fixed_point(N, r, L, s, NULL);
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t cc[3];
        for (int a = 0; a < 3; ++a) cc[a] = (uint32_t)(((uint64_t)s[3 * i + a] * (uint64_t)nc[a]) >> 32);
        cell_of[i] = cc[0] + (uint32_t)nc[0] * (cc[1] + (uint32_t)nc[1] * cc[2]);
        cell_start[cell_of[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    for (int64_t c = 0; c < ncell; ++c) cursor[c] = cell_start[c];
    for (int64_t i = 0; i < N; ++i) perm[cursor[cell_of[i]]++] = (uint32_t)i;
    free(cursor);
    free(s);
}

/* ---- near field (Eq. 55 first term, U_N of Eq. 50) -------------------- */

static void near_pair(const double *sog, double rc, double qi, double qj, const double *d,
                      double *Fi, double *U) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 >= rc * rc || r2 == 0.0) return;
    double r = sqrt(r2), lam = sog[5];
    double g = qi * qj * (force_n1(r, lam) + orc_force_n2(sog, r));
    Fi[0] += g * d[0];
    Fi[1] += g * d[1];
    Fi[2] += g * d[2];
    *U += 0.5 * qi * qj * (yukawa(r, lam) - orc_sog_F(sog, r));
}

/* All pairs and all periodic images within r_c (valid for any box).  The sum
 * excludes only i == j in the home image (the prime of Eq. 50).  Outputs are
 * produced for the n_out particles listed in idx (all N when idx is NULL);
 * U is the energy share of those particles (the full U_N when idx is NULL). */
void orc_near_images(int64_t N, const double *r, const double *q, const double *L, double rc,
                     const double *sog, int64_t n_out, const int64_t *idx, double *F, double *U) {
    int nmax[3];
    for (int a = 0; a < 3; ++a) nmax[a] = (int)ceil(rc / L[a]) + 1;
    double Utot = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : Utot)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        double Fi[3] = {0.0, 0.0, 0.0}, Ui = 0.0;
        for (int64_t j = 0; j < N; ++j)
            for (int nx = -nmax[0]; nx <= nmax[0]; ++nx)
                for (int ny = -nmax[1]; ny <= nmax[1]; ++ny)
                    for (int nz = -nmax[2]; nz <= nmax[2]; ++nz) {
                        if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {r[3 * i] - r[3 * j] - nx * L[0], r[3 * i + 1] - r[3 * j + 1] - ny * L[1],
                                       r[3 * i + 2] - r[3 * j + 2] - nz * L[2]};
                        near_pair(sog, rc, q[i], q[j], d, Fi, &Ui);
                    }
        F[3 * o] = Fi[0];
        F[3 * o + 1] = Fi[1];
        F[3 * o + 2] = Fi[2];
        Utot += Ui;
    }
    *U = Utot;
}

/* Same sum through a cell list and the minimum image (requires r_c <= L/2).
 * Along an axis with fewer than 3 cells every cell of that axis is visited. */
void orc_near_cells(int64_t N, const double *r, const double *q, const double *L, double rc,
                    const double *sog, const int *nc, const uint32_t *cell_of, const uint32_t *cell_start,
                    const uint32_t *perm, int64_t n_out, const int64_t *idx, double *F, double *U) {
    double Utot = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : Utot)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        uint32_t c = cell_of[i];
        int ci[3] = {(int)(c % (uint32_t)nc[0]), (int)((c / (uint32_t)nc[0]) % (uint32_t)nc[1]),
                     (int)(c / ((uint32_t)nc[0] * (uint32_t)nc[1]))};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (nc[a] >= 3) { lo[a] = -1; hi[a] = 1; }
            else { lo[a] = -ci[a]; hi[a] = nc[a] - 1 - ci[a]; }
        }
        double Fi[3] = {0.0, 0.0, 0.0}, Ui = 0.0;
        for (int dz = lo[2]; dz <= hi[2]; ++dz)
            for (int dy = lo[1]; dy <= hi[1]; ++dy)
                for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                    int cx = (ci[0] + dx + nc[0]) % nc[0], cy = (ci[1] + dy + nc[1]) % nc[1],
                        cz = (ci[2] + dz + nc[2]) % nc[2];
                    uint32_t cn = (uint32_t)cx + (uint32_t)nc[0] * ((uint32_t)cy + (uint32_t)nc[1] * (uint32_t)cz);
                    for (uint32_t k = cell_start[cn]; k < cell_start[cn + 1]; ++k) {
                        int64_t j = perm[k];
                        if (j == i) continue;
                        double d[3];
                        for (int a = 0; a < 3; ++a) {
                            d[a] = r[3 * i + a] - r[3 * j + a];
                            d[a] -= L[a] * nearbyint(d[a] / L[a]);
                        }
                        near_pair(sog, rc, q[i], q[j], d, Fi, &Ui);
                    }
                }
        F[3 * o] = Fi[0];
        F[3 * o + 1] = Fi[1];
        F[3 * o + 2] = Fi[2];
        Utot += Ui;
    }
    *U = Utot;
}

/* ---- far field --------------------------------------------------------- */

/* rho(k_l) = sum_j q_j exp(i k_l . r_j), k_l = 2 pi m_l / L (Sec. 2; k of Sec. 3.3). */
void orc_rho(int64_t N, const double *r, const double *q, const double *L, int P, const int32_t *m,
             double *rho) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int l = 0; l < P; ++l) {
        double k[3];
        for (int a = 0; a < 3; ++a) k[a] = 2.0 * M_PI * m[3 * l + a] / L[a];
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
            re += q[j] * cos(th);
            im += q[j] * sin(th);
        }
        rho[2 * l] = re;
        rho[2 * l + 1] = im;
    }
}

/* Random-batch far force (Eq. 60 with the gradient of |rho|^2 written out):
 * F*_i = -q_i sum_l coef_l k_l Im(exp(-i k_l.r_i) rho_l),
 * Im(exp(-i th) rho) = cos(th) Im rho - sin(th) Re rho. */
void orc_far_rb(int64_t N, const double *r, const double *q, const double *L, int P, const int32_t *m,
                const double *coef, const double *rho, int64_t n_out, const int64_t *idx, double *F) {
    (void)N;
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = idx ? idx[o] : o;
        double Fi[3] = {0.0, 0.0, 0.0};
        for (int l = 0; l < P; ++l) {
            double k[3];
            for (int a = 0; a < 3; ++a) k[a] = 2.0 * M_PI * m[3 * l + a] / L[a];
            double th = k[0] * r[3 * i] + k[1] * r[3 * i + 1] + k[2] * r[3 * i + 2];
            double im = cos(th) * rho[2 * l + 1] - sin(th) * rho[2 * l];
            for (int a = 0; a < 3; ++a) Fi[a] += coef[l] * k[a] * im;
        }
        for (int a = 0; a < 3; ++a) F[3 * o + a] = -q[i] * Fi[a];
    }
}

/* Deterministic far field over every mode 0 < |k|^2 <= kmax2 (Eqs. 53, 55):
 * U_F = (1/2V) sum_k Fhat |rho|^2 (+ the k = 0 term Fhat(0)(sum q)^2/(2V)),
 * F_i = -(q_i/V) sum_k k Fhat Im(exp(-i k.r_i) rho(k)).  O(N K); small N only. */
void orc_far_full(int64_t N, const double *r, const double *q, const double *L, const double *sog,
                  double kmax2, double *F, double *U) {
    double V = L[0] * L[1] * L[2];
    int nmax[3];
    for (int a = 0; a < 3; ++a) nmax[a] = (int)floor(sqrt(kmax2) * L[a] / (2.0 * M_PI)) + 1;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    double qsum = 0.0;
    for (int64_t j = 0; j < N; ++j) qsum += q[j];
    double Uacc = orc_fhat(sog, 0.0) * qsum * qsum / (2.0 * V);
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int mx = -nmax[0]; mx <= nmax[0]; ++mx)
        for (int my = -nmax[1]; my <= nmax[1]; ++my)
            for (int mz = -nmax[2]; mz <= nmax[2]; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                double k[3] = {2.0 * M_PI * mx / L[0], 2.0 * M_PI * my / L[1], 2.0 * M_PI * mz / L[2]};
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 > kmax2) continue;
                double fh = orc_fhat(sog, k2);
                double re = 0.0, im = 0.0;
                for (int64_t j = 0; j < N; ++j) {
                    double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
                    cs[2 * j] = cos(th);
                    cs[2 * j + 1] = sin(th);
                    re += q[j] * cs[2 * j];
                    im += q[j] * cs[2 * j + 1];
                }
                Uacc += fh * (re * re + im * im) / (2.0 * V);
                for (int64_t i = 0; i < N; ++i) {
                    double imv = cs[2 * i] * im - cs[2 * i + 1] * re;
                    for (int a = 0; a < 3; ++a) F[3 * i + a] -= q[i] / V * k[a] * fh * imv;
                }
            }
    free(cs);
    *U = Uacc;
}

/* Normalisation S = sum_{k != 0, |k|^2 <= kmax2} calF(k) Fhat(k) of the sampling
 * measure P(k) = calF Fhat / S (Eq. 59), calF of the chosen measure (orc_measure). */
double orc_S_sum(const double *L, const double *sog, double kT, double Q2, double kmax2, int measure) {
    double V = L[0] * L[1] * L[2], lam = sog[5];
    int nmax[3];
    for (int a = 0; a < 3; ++a) nmax[a] = (int)floor(sqrt(kmax2) * L[a] / (2.0 * M_PI)) + 1;
    double S = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : S)
    for (int mx = -nmax[0]; mx <= nmax[0]; ++mx) {
        double Sx = 0.0;
        for (int my = -nmax[1]; my <= nmax[1]; ++my)
            for (int mz = -nmax[2]; mz <= nmax[2]; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                double kx = 2.0 * M_PI * mx / L[0], ky = 2.0 * M_PI * my / L[1], kz = 2.0 * M_PI * mz / L[2];
                double k2 = kx * kx + ky * ky + kz * kz;
                if (k2 > kmax2) continue;
                Sx += orc_measure(measure, k2, kT, V, Q2, lam) * orc_fhat(sog, k2);
            }
        S += Sx;
    }
    return S;
}

/* ---- real-space pins (independent of the Fourier machinery) ---------- */

/* Real-space image sum of the far kernel F: U = 1/2 sum_n sum_{i,j} q_i q_j F(|r_i - r_j - n o L|)
 * including i == j in the home image (F(0)); force F_i = sum q_i q_j (-F_N2(|d|)) d, since
 * -F'(r)/r = 2h sum^# e^{t_m} f(t_m, r) = -F_N2(r).  Images with |n_a| <= nimg. */
void orc_real_far(int64_t N, const double *r, const double *q, const double *L, const double *sog, int nimg,
                  double *F, double *U) {
    double Utot = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : Utot)
    for (int64_t i = 0; i < N; ++i) {
        double Fi[3] = {0.0, 0.0, 0.0}, Ui = 0.0;
        for (int64_t j = 0; j < N; ++j)
            for (int nx = -nimg; nx <= nimg; ++nx)
                for (int ny = -nimg; ny <= nimg; ++ny)
                    for (int nz = -nimg; nz <= nimg; ++nz) {
                        double d[3] = {r[3 * i] - r[3 * j] - nx * L[0], r[3 * i + 1] - r[3 * j + 1] - ny * L[1],
                                       r[3 * i + 2] - r[3 * j + 2] - nz * L[2]};
                        double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        Ui += 0.5 * q[i] * q[j] * orc_sog_F(sog, rr);
                        if (rr > 0.0) {
                            double g = -q[i] * q[j] * orc_force_n2(sog, rr);
                            for (int a = 0; a < 3; ++a) Fi[a] += g * d[a];
                        }
                    }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = Fi[a];
        Utot += Ui;
    }
    *U = Utot;
}

/* Brute-force periodic Yukawa lattice sum: U = 1/2 sum'_n sum_{i,j} q_i q_j Y(|d|) over every
 * image with |d| <= rcut, F_i = sum q_i q_j exp(-r/lam)(1+r/lam)/r^3 d.  Textbook, method-free. */
void orc_brute_yukawa(int64_t N, const double *r, const double *q, const double *L, double lam, double rcut,
                      double *F, double *U) {
    int nmax[3];
    for (int a = 0; a < 3; ++a) nmax[a] = (int)ceil(rcut / L[a]) + 1;
    double Utot = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : Utot)
    for (int64_t i = 0; i < N; ++i) {
        double Fi[3] = {0.0, 0.0, 0.0}, Ui = 0.0;
        for (int64_t j = 0; j < N; ++j)
            for (int nx = -nmax[0]; nx <= nmax[0]; ++nx)
                for (int ny = -nmax[1]; ny <= nmax[1]; ++ny)
                    for (int nz = -nmax[2]; nz <= nmax[2]; ++nz) {
                        if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
                        double d[3] = {r[3 * i] - r[3 * j] - nx * L[0], r[3 * i + 1] - r[3 * j + 1] - ny * L[1],
                                       r[3 * i + 2] - r[3 * j + 2] - nz * L[2]};
                        double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        if (rr > rcut) continue;
                        Ui += 0.5 * q[i] * q[j] * yukawa(rr, lam);
                        double g = q[i] * q[j] * force_n1(rr, lam);
                        for (int a = 0; a < 3; ++a) Fi[a] += g * d[a];
                    }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = Fi[a];
        Utot += Ui;
    }
    *U = Utot;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the parallel loops above (timing legs only; results do not depend on it
 * beyond the order of the reductions). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
