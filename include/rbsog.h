/*
 * rbsog.h -- C ABI of the GB300 (sm_103a) random batch sum-of-Gaussians force step
 * for 3-D periodic Yukawa systems (Chen, Liang & Xu, "Random batch sum-of-Gaussians
 * algorithm for molecular dynamics simulations of Yukawa systems in three dimensions").
 *
 * One step of Algorithm 2 on the GPU, every part in hand-written CUDA:
 *   cell list (counting sort)  ->  near field, Eq. (55) first term, Eqs. (56)-(57)
 *   k-sampler, Eq. (59)        ->  structure factor rho(k_l) = sum_j q_j e^{i k_l . r_j} (Sec. 2)
 *   far-force gather, Eq. (60) ->  velocity Verlet or Langevin update (Algorithm 2, last step)
 * The SOG decomposition (Algorithm 1, Eqs. (27)-(38)) is built on the host at init.
 *
 * Conventions for every entry point
 *   - Status: each call returns RBSOG_OK (0) or a positive RBSOG_E* code; a message
 *     is available from rbsog_last_error(ctx).  Nothing throws across the ABI, and
 *     there is no CPU fallback: if the GPU path cannot run, the call fails.
 *   - Vectors are [N][3] row-major float64 in the caller's particle order.
 *   - Pointers marked "host or device" may point to host memory (pageable or pinned)
 *     or to device memory on the context's device (unified addressing decides).  The
 *     single-context calls that move [N][3] rows (rbsog_set_state*, rbsog_get_state,
 *     rbsog_get_forces*) read and write device memory and pinned host memory from
 *     their kernels directly (pinned memory through its mapped device address, in
 *     whole lines over the host link) and stage pageable memory through a device
 *     buffer and a copy.  An enqueued call reads its inputs when the stream reaches
 *     it: keep them unchanged until then.
 *   - Pointers marked "host" must be host memory; "device" must be device memory.
 *   - The caller owns every pointer it passes; the library copies what it keeps.
 *     The library owns all of its internal device buffers and frees them in
 *     rbsog_free.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls that
 *     take a stream enqueue their work on it and may return before it completes,
 *     except where marked "synchronous".
 *   - Reduced units: charge and mass are whatever the caller passes; lengths, kappa
 *     and Gamma follow Sec. 5.1 (Gamma = Q^2/(a k_B T) with Q = 1, kappa = a/lambda).
 */
#ifndef RBSOG_H
#define RBSOG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define RBSOG_OK 0
#define RBSOG_EINVAL 1        /* bad argument or parameter (r_c > L/2, P < 1, N < 2, ...) */
#define RBSOG_ENOMEM 2        /* a device allocation failed */
#define RBSOG_ECUDA 3         /* a CUDA runtime call or kernel failed */
#define RBSOG_ETIMEOUT 4      /* a bounded device-side loop hit its limit */
#define RBSOG_ENOCONV 5       /* the SOG construction found no C1 root / no decomposition */
#define RBSOG_EUNSUPPORTED 6  /* a valid request this build does not implement */
#define RBSOG_EOVERFLOW 7     /* a cell holds more particles than the near-field kernel stages */

/* precision */
#define RBSOG_FP64 0          /* every force and phase in FP64 (parity build) */
#define RBSOG_FP32 1          /* FP32 pair and phase arithmetic with compensated sums;
                                 positions and velocities stored in FP64, the positions
                                 accumulating FP32 kick and drift increments; energies
                                 reduced in FP64 */
/* ensemble */
#define RBSOG_NVE 0           /* velocity Verlet */
#define RBSOG_LANGEVIN 1      /* BAOAB Langevin, friction langevin_gamma, target k_B T */
/* sog_mode: how (M1, M2) of Algorithm 1 are chosen */
#define RBSOG_SOG_MINIMAL 0   /* fewest Gaussians with max |Y - F| <= sog_eps on [r_c, 33 lambda] */
#define RBSOG_SOG_BOUND 1     /* ceilings of Eqs. (29)-(30) at the C0 root alpha_1 of Eq. (35) */
#define RBSOG_SOG_TABLE 2     /* sog_M1, sog_M2 given (e.g. a row of Table 1) */

/* Sampling measure P(k) = calF(k) Fhat(k) / S of Eq. (59), S = sum_{k != 0} calF Fhat, and
 * coef_l = S / (P V calF(k_l)) (Eq. 60), for the three corrections compared in Sec. 5
 * (Fig. 9).  Every choice gives an unbiased estimator; they differ in variance. */
#define RBSOG_SAMPLING_ADAPTIVE 0   /* calF of Eq. (62) (Debye-Hueckel structure factor) */
#define RBSOG_SAMPLING_UNIFORM 1    /* calF = 1: P(k) proportional to Fhat (as in RBE) */
#define RBSOG_SAMPLING_K2 2         /* calF = k^2 (as in RBSOG for Coulomb systems) */
#define RBSOG_SAMPLING_DEBYE 3      /* Eq. (62) with the Debye wavenumber of Gaussian units:
                                       4 pi sum q^2 / (kT V) in place of sum q^2 / (kT V) */

/* How the P modes of a force evaluation are drawn from P(k) (Eq. 59). */
#define RBSOG_SAMPLER_IID 0         /* exact independent draws (rejection from the Gaussian
                                       mixture of Fhat); every evaluation's batch is fresh */
#define RBSOG_SAMPLER_MH 1          /* the Metropolis-Hastings method Sec. 4.3 names: P
                                       independent chains, one per batch slot, each an
                                       independence sampler whose proposal is the mixture
                                       draw and whose acceptance is min(1, a(k')/a(k)),
                                       a = calF / sum q^2 (a = 1 for calF = 1 and k^2); the
                                       batch is the chain states, correlated from one
                                       evaluation to the next */

/* Temperature of the adaptive correction calF of Eq. (62). */
#define RBSOG_KT_TARGET 0           /* the target k_B T (Gamma or kT) */
#define RBSOG_KT_INSTANT 1          /* the instantaneous kinetic temperature, computed on the
                                       device at every force evaluation (Sec. 4.3, NVT): k_B T =
                                       2 K / (3 N), K the kinetic energy of the velocities the
                                       step has when the forces are evaluated (after the
                                       opening kick and drift, before the closing kick); S of
                                       Eq. (59) is re-summed at that temperature */

typedef struct rbsog_ctx rbsog_ctx;
typedef struct rbsog_batch rbsog_batch;
typedef struct rbsog_server rbsog_server;

typedef struct rbsog_params {
    double box[3];          /* L_x, L_y, L_z (absolute lengths), each > 0 */
    double kappa;           /* screening parameter a/lambda (Sec. 5.1), > 0 */
    double a_ws;            /* Wigner-Seitz radius a; 0 selects (3V/(4 pi N))^(1/3) */
    double Gamma;           /* bare coupling Q^2/(a k_B T) with Q = 1 (Sec. 5.1) */
    double kT;              /* > 0 overrides k_B T = 1/(a Gamma) */
    double r_c;             /* near-field cutoff (absolute), 0 < r_c <= min(L)/2 */
    double sog_eps;         /* SOG tolerance eps of Algorithm 1, in (0, 0.1] */
    double dt;              /* time step */
    double langevin_gamma;  /* Langevin friction (1/time), used with RBSOG_LANGEVIN */
    uint64_t seed;          /* Philox key for the k-sampler and the Langevin noise; both are
                               counted by force evaluations, which rbsog_set_state does not reset */
    int32_t P;              /* random-batch size, 1 <= P <= 4096 */
    int32_t precision;      /* RBSOG_FP64 | RBSOG_FP32 */
    int32_t ensemble;       /* RBSOG_NVE | RBSOG_LANGEVIN */
    int32_t sog_mode;       /* RBSOG_SOG_MINIMAL | RBSOG_SOG_BOUND | RBSOG_SOG_TABLE */
    int32_t sog_M1;         /* with RBSOG_SOG_TABLE: M1 of Eq. (37) */
    int32_t sog_M2;         /* with RBSOG_SOG_TABLE: M2 of Eq. (37) */
    int32_t device;         /* CUDA device ordinal */
    int32_t sampling;       /* RBSOG_SAMPLING_*: correction calF of the sampling measure (Eq. 59) */
    double egs_nu;          /* 0: the Yukawa kernel.  0 < egs_nu <= 0.96: the gradient-corrected
                               screening eps(k) = 1 + (lambda k)^-2 (1 + egs_nu lambda^2 k^2/4)^-1
                               of Sec. 1, split by partial fractions into two Yukawa kernels
                               B Y_{lambda_B} + A Y_{lambda_A} (A + B = 1, A < 0), each with its
                               own SOG decomposition at r_c and sog_eps (sog_mode MINIMAL or
                               BOUND); the modes are drawn from the envelope of the far
                               field's transform and coef carries Fhat / Fhat_env */
    int32_t sampler;        /* RBSOG_SAMPLER_IID | RBSOG_SAMPLER_MH (the latter: Yukawa kernel,
                               single contexts only) */
    int32_t mh_sweeps;      /* MH: proposals per chain at each force evaluation; 0 selects 1 */
    int32_t mh_burnin;      /* MH: proposals per chain after its start, at the first force
                               evaluation; 0 selects 64, negative selects none */
    int32_t temperature;    /* RBSOG_KT_TARGET | RBSOG_KT_INSTANT (single contexts only; a no-op
                               for calF = 1 and calF = k^2, which do not depend on T) */
    double q2_total;        /* > 0: sum q^2 of the whole system when the context holds one
                               domain of it (rbsog_set_owned); enters calF of Eq. (62), S and
                               the coefficients.  0: the context's own charges */
    double qsum_total;      /* with q2_total > 0: sum q of the whole system (the k = 0 term) */
} rbsog_params;

typedef struct rbsog_energy {
    double U_near;          /* U_N of Eq. (50) over pairs inside r_c */
    double U_far;           /* random-batch estimate U*_F of Eq. (60) plus the k = 0 term */
    double U_self;          /* U_self of Eq. (52) */
    double kinetic;         /* sum_i m_i |v_i|^2 / 2 */
    double total;           /* U_near + U_far + U_self + kinetic (Eq. 49 plus kinetic energy) */
    uint64_t step;          /* steps taken since rbsog_set_state */
} rbsog_energy;

/* Create a context: builds the SOG decomposition of Algorithm 1 on the host, the
 * sampling tables of P(k) (Eq. 59) and its normalisation S on the device, and
 * allocates every device buffer for N particles.  q_host and m_host are host arrays
 * of N charges and N masses (masses > 0), copied.  Synchronous.  On success *out
 * holds the context; on failure *out is NULL and the message is available from
 * rbsog_last_error(NULL). */
int rbsog_init(const rbsog_params *params, int64_t N, const double *q_host, const double *m_host,
               rbsog_ctx **out);

/* Set positions r ([N][3], any real values; wrapped into the box) and velocities v
 * ([N][3]; NULL = zero), host or device pointers.  Resets the step counter and the
 * internal particle order.  The force at the new state is computed by the next
 * rbsog_step or rbsog_forces.  Enqueued on stream. */
int rbsog_set_state(rbsog_ctx *ctx, const double *r, const double *v, void *stream);

/* Copy positions (wrapped into [0, L)) and velocities to r and v ([N][3], host or
 * device; either may be NULL) in the caller's particle order, and the step counter
 * to *step (host; may be NULL).  Synchronous. */
int rbsog_get_state(rbsog_ctx *ctx, double *r, double *v, uint64_t *step, void *stream);

/* As rbsog_set_state, together with the forces F at that state ([N][3] in the caller's
 * order, host or device; NULL = rbsog_set_state), for instance those that
 * rbsog_get_forces returned after a step.  The next rbsog_step then integrates with
 * them (the first kick of Algorithm 2) instead of evaluating forces first, so a loop
 * that uploads r, v and F and reads them back after each step follows the same
 * trajectory, bit for bit, as steps that stay on the device.  The FP32 build keeps F
 * in FP32 (an F that it returned comes back exactly).  Enqueued on stream. */
int rbsog_set_state_forces(rbsog_ctx *ctx, const double *r, const double *v, const double *F, void *stream);

/* The forces at the current state (those of the last force evaluation: Eq. 55, with the
 * far part of that evaluation's draw) into F ([N][3] in the caller's order, host or
 * device).  RBSOG_EINVAL when no force has been evaluated or uploaded since the last
 * rbsog_set_state.  Synchronous. */
int rbsog_get_forces(rbsog_ctx *ctx, double *F, void *stream);

/* FP32 forms of the two calls above, for precision RBSOG_FP32 only (RBSOG_EINVAL for the
 * FP64 build, or for ctx NULL).  That build computes and keeps the forces in FP32, so
 * F ([N][3] floats, caller's order, host or device) carries the same values in half the
 * bytes: a loop through the host that moves F this way follows the same trajectory, bit
 * for bit, as one that moves it in FP64.  rbsog_set_state_forces_f32 with F NULL is
 * rbsog_set_state; it is enqueued on stream.  rbsog_get_forces_f32 fails as
 * rbsog_get_forces does and is synchronous.  F is taken in the caller's particle order:
 * the state upload in the same call resets the internal order to the caller's, and the
 * forces are stored in that order before the next step sorts particles into cells. */
int rbsog_set_state_forces_f32(rbsog_ctx *ctx, const double *r, const double *v, const float *F, void *stream);
int rbsog_get_forces_f32(rbsog_ctx *ctx, float *F, void *stream);

/* Forces at the current positions (Eq. 55 with the far part estimated by Eq. 60)
 * from one fresh draw of P modes (or the set injected by rbsog_set_ksample) into
 * F ([N][3], host or device; NULL = keep internal only).  If e is not NULL the
 * energies are written to *e and the call is synchronous; otherwise enqueued. */
int rbsog_forces(rbsog_ctx *ctx, double *F, rbsog_energy *e, void *stream);

/* As rbsog_forces, with the near part (Eq. 55 first term) in F_near and the
 * random-batch far part (Eq. 60) in F_far; either may be NULL. */
int rbsog_forces_split(rbsog_ctx *ctx, double *F_near, double *F_far, rbsog_energy *e, void *stream);

/* Advance nsteps >= 0 steps of Algorithm 2 (sample, far force, near force,
 * integrate).  The step sequence is captured once as a CUDA graph (on an internal
 * stream) and replayed on `stream`.  If e is not NULL the energies after the last step are written to *e
 * and the call is synchronous.  The energies are those of the last force evaluation, so
 * with nsteps = 0 right after rbsog_set_state or rbsog_set_state_forces(_f32) (no
 * evaluation at the uploaded state yet) an energy request fails with RBSOG_EINVAL. */
int rbsog_step(rbsog_ctx *ctx, int32_t nsteps, rbsog_energy *e, void *stream);

/* Advance nsteps >= 1 steps as rbsog_step and read back the state after them, as
 * rbsog_get_state and rbsog_get_forces(_f32) would: positions r and velocities v
 * ([N][3] doubles), forces F ([N][3], floats when f32 != 0 (FP32 build only), else
 * doubles), all in the caller's order, host or device; any may be NULL; energies to *e
 * when e is not NULL.  The positions are final once the last step has rebuilt its cell
 * list, so they are copied back (copy engine, from a device staging buffer) while that
 * step's forces are computed; velocities and forces follow the step.  Synchronous.
 * RBSOG_EINVAL for nsteps < 1. */
int rbsog_step_get(rbsog_ctx *ctx, int32_t nsteps, double *r, double *v, void *F, int32_t f32, rbsog_energy *e,
                   void *stream);

/* Inject the next force evaluation's modes: m_host is P triples (m_x, m_y, m_z) of
 * integers, not all zero, k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z).  Used once, then
 * sampling resumes.  P must equal the context's P.  Host pointer; synchronous. */
int rbsog_set_ksample(rbsog_ctx *ctx, const int32_t *m_host, int32_t P);

/* The modes and coefficients coef_l = S/(P V calF(k_l)) of the last force
 * evaluation (host arrays of P triples and P doubles; either may be NULL). Synchronous. */
int rbsog_get_ksample(rbsog_ctx *ctx, int32_t *m_host, double *coef_host);

/* rho(k_l) of the last force evaluation as P (Re, Im) pairs (host).  Synchronous. */
int rbsog_get_rho(rbsog_ctx *ctx, double *rho_host);

/* The cell list of the last force evaluation: nc[3] cells per axis, cell_start
 * (n_c^3 + 1 entries) and perm (N entries, the caller's particle index at each
 * cell-sorted position; within a cell, ascending).  Host arrays; any may be NULL.
 * Cells: s_a = floor(frac(r_a (1/L_a)) 2^32) with 1/L_a rounded to double,
 * c_a = floor(s_a n_a / 2^32), c = c_x + n_x (c_y + n_y c_z), n_a = floor(L_a / r_c)
 * when >= 3 else 1.  Synchronous. */
int rbsog_get_cells(rbsog_ctx *ctx, int32_t *nc, uint32_t *cell_start, uint32_t *perm);

/* The SOG decomposition in use (Eq. 37): h, t0, M1, M2, the C1 weight w of m = M2,
 * lambda, and the sampling normalisation S = sum_{k != 0} calF(k) Fhat(k).  With the EGS
 * screening (egs_nu > 0) the decomposition is that of its first Yukawa term, lambda_B,
 * and S is the envelope's.  Host pointers, any may be NULL. */
int rbsog_get_sog(rbsog_ctx *ctx, double *h, double *t0, int32_t *M1, int32_t *M2, double *w, double *lam,
                  double *S);

/* The k_B T and the normalisation S = sum_{k != 0} calF(k) Fhat(k) of the last force
 * evaluation (host pointers, either may be NULL): with RBSOG_KT_INSTANT the instantaneous
 * temperature and the S re-summed at it, else the target k_B T and the S of
 * rbsog_get_sog.  Synchronous. */
int rbsog_get_temperature(rbsog_ctx *ctx, double *kT, double *S);

/* Kernel-group timing.  With enable != 0, rbsog_step and rbsog_forces launch their
 * kernels eagerly (no graph) and record CUDA events on the launching stream around
 * each of the RBSOG_NPROF groups named by rbsog_profile_name: bin (integrator first
 * half + cell binning), scan, sort (scatter + per-cell sort), gather, sample, near,
 * rho, rho_final, far (gather of Eq. 60 + closing half kick), close (the one-thread
 * kernel that ends an evaluation: step counter and forces-valid flag; the energy
 * reduction itself runs only when energies are read).  enable = 0
 * restores graph replay.  Either call discards collected timings.  Synchronous. */
#define RBSOG_NPROF 10
int rbsog_profile(rbsog_ctx *ctx, int32_t enable);

/* Summed event time in milliseconds (ms[RBSOG_NPROF]) and the number of launches
 * (launches[RBSOG_NPROF]) of each group since the last read, then discards them.
 * Host arrays.  Synchronous. */
int rbsog_profile_read(rbsog_ctx *ctx, double *ms, int64_t *launches);

/* Name of profiling group g (0 <= g < RBSOG_NPROF), or "" (static string). */
const char *rbsog_profile_name(int32_t group);

/* Algorithm 1 on the host alone (no device is touched): the C1 SOG decomposition of
 * exp(-r/lambda)/r for cutoff r_c and tolerance eps with (M1, M2) chosen by mode
 * (RBSOG_SOG_*; M1, M2 are read only for RBSOG_SOG_TABLE).  Writes
 * out6 = {h, t0, M1, M2, w, max |Y - F| on the 2000-point grid of [r_c, 33 lambda]}
 * (host array of 6 doubles).  RBSOG_ENOCONV when no C1 root or decomposition exists;
 * the message is then available from rbsog_last_error(NULL). */
int rbsog_build_sog(double lam, double r_c, double eps, int32_t mode, int32_t M1, int32_t M2, double *out6);

/* Structure factor without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code that runs
 * inside a fixed memory budget owned by another allocator, or a latency-critical
 * loop that must not pay for an allocation that can synchronise the device.
 *
 * Computes rho_l = sum_j q_j exp(i k_l . r_j), k_l = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z),
 * with the arithmetic of the FP32 build (2^32 fixed-point phases, FP32 sin/cos with
 * compensated per-block sums, FP64 fixed-order reduction over blocks).
 *   r_dev   device, [N][3] float64 positions (any real values; taken modulo the box)
 *   q_dev   device, [N] float64 charges
 *   box_host host, 3 box lengths > 0
 *   m_dev   device, [P][3] int32 mode triples
 *   rho_dev device, [P][2] float64 output (Re, Im)
 *   stream  cudaStream_t the work is enqueued on; the call returns before it completes.
 * It allocates nothing: its per-block partial sums live in one statically sized
 * device array of 4 MiB (262144 double2 slots) that every GPU loading this library
 * holds until the process exits.  The array needs G x S x P slots, G = min(152,
 * ceil(N/64)) blocks and S = 1..8 particle subsets per block (S = 1 once P > 128), so
 * P up to 1724 is always accepted (up to 4096 when G x P fits, i.e. small N); larger
 * requests fail with RBSOG_EINVAL and a message.  The first call on a device looks the array's device address up with
 * cudaGetSymbolAddress and caches it (with that device current); make that first
 * call before any stream capture.  Every call shares the array, which keeps the last
 * call's contents; each call writes every slot it later reads, so nothing needs
 * clearing.  Calls whose work overlaps on the GPU (different streams, or other host
 * threads) race on the array and must be serialised by the caller.  Errors are
 * reported through rbsog_last_error(NULL). */
int rbsog_rho_noalloc(const double *r_dev, const double *q_dev, int64_t N, const double *box_host,
                      const int32_t *m_dev, int32_t P, double *rho_dev, void *stream);

/* ---- Domain decomposition (Sec. 4.3: local structure factors, a global reduction of
 * rho, a broadcast) ----------------------------------------------------------------------
 * A context can hold one domain of a larger system: its particles are the domain's own
 * ("owned") particles followed by halo copies of the particles of neighbouring domains
 * within the cutoff.  The halo particles take part in the near field of the owned ones
 * and nothing else.  Every domain's context uses the whole system's box, seed and
 * parameters, with q2_total / qsum_total of the whole system, so all domains draw the same
 * modes with the same coefficients.  One force evaluation is then:
 *   rbsog_forces_partial   every domain: cell list and near field of its particles, the
 *                          k-sample, and rho over its owned particles -> partial rho;
 *   (caller)               sum the partial rho over the domains (an all-reduce of 2P
 *                          doubles: MPI, NCCL, gloo, or a host sum);
 *   rbsog_forces_complete  every domain: the far force of Eq. (60) from the summed rho,
 *                          plus the near force, for its particles; the rows of the owned
 *                          particles are the whole system's forces on them.
 * The energies of such an evaluation are not available (RBSOG_EINVAL from an energy read).
 * rbsog_slab_split computes a domain's particle list for slabs along one axis. */

/* The first n_owned particles (1 <= n_owned <= N) are the context's own; only they enter
 * rho(k) (in every evaluation).  Default N.  Synchronous. */
int rbsog_set_owned(rbsog_ctx *ctx, int64_t n_owned);

/* First half of a domain's force evaluation (see above): writes the partial rho over the
 * owned particles as P (Re, Im) pairs to rho_partial (host or device).  One fresh draw of
 * modes (or the injected set).  Synchronous. */
int rbsog_forces_partial(rbsog_ctx *ctx, double *rho_partial, void *stream);

/* Second half: rho (P (Re, Im) pairs, host or device) is the sum of every domain's partial
 * rho; writes the total forces of all the context's particles to F ([N][3], caller order,
 * host or device; may be NULL), valid for the owned ones.  The forces are kept as those
 * of the current state (rbsog_get_forces).  RBSOG_EINVAL unless rbsog_forces_partial came
 * first.  Synchronous. */
int rbsog_forces_complete(rbsog_ctx *ctx, const double *rho, double *F, void *stream);

/* Host only: the particle list of slab `slab` of `nslabs` equal slabs along `axis` (0..2)
 * of the periodic box: idx_out[0 .. *n_owned) are the particles whose wrapped coordinate
 * lies in the slab (ascending index), idx_out[*n_owned .. *n_local) those of other slabs
 * within `halo` of it (periodic distance along the axis; ascending index).  idx_out has
 * room for N entries.  Requires halo <= L / 2 (the near field's minimum image then finds
 * every pair across the slab's faces once).  RBSOG_EINVAL on bad arguments. */
int rbsog_slab_split(int64_t N, const double *r_host, const double *box, int32_t axis, int32_t nslabs,
                     int32_t slab, double halo, int64_t *idx_out, int64_t *n_owned, int64_t *n_local);

/* Message of the last failed call on ctx (or of the last failed rbsog_init when ctx
 * is NULL).  The pointer stays valid until the next call on the same context. */
const char *rbsog_last_error(const rbsog_ctx *ctx);

/* Release every device buffer and graph of ctx.  Synchronous.  NULL is a no-op. */
void rbsog_free(rbsog_ctx *ctx);

/* ---- Batches of independent systems ------------------------------------------------
 * R systems, each a periodic Yukawa system with its own parameters (box, kappa, Gamma,
 * r_c, P, seed, dt, ensemble), advanced together: every kernel of Algorithm 2's step is
 * one launch over all systems and the step is replayed as one CUDA graph.  The systems'
 * particles are concatenated in the caller's arrays: system r holds particles
 * p_off[r] .. p_off[r+1]-1 (p_off[0] = 0, p_off[r+1] = p_off[r] + N[r]), and its P modes
 * are entries m_off[r] .. m_off[r+1]-1 of the concatenated mode arrays.  Every system
 * uses the FP32 path (precision must be RBSOG_FP32) and the same device.  The step and
 * k-draw counters are shared, so system r draws the same modes and Langevin noise as a
 * single context (rbsog_init) with params[r] after the same calls.  A device error in
 * any system (cell overflow, sampler limit) fails the call for the whole batch. */

/* Create a batch.  params: R parameter blocks; N: R particle counts (each >= 2, total
 * < 2^31); q_host, m_host: host arrays of sum(N) charges and masses, copied.
 * Synchronous.  On failure *out is NULL and rbsog_batch_last_error(NULL) holds the
 * message (naming the first invalid system). */
int rbsog_batch_init(const rbsog_params *params, int32_t R, const int64_t *N, const double *q_host,
                     const double *m_host, rbsog_batch **out);

/* Positions r and optional velocities v ([sum N][3] doubles, host or device) of all
 * systems; as rbsog_set_state for each system.  Asynchronous on stream. */
int rbsog_batch_set_state(rbsog_batch *b, const double *r, const double *v, void *stream);

/* Positions and velocities ([sum N][3], caller order, host or device; either may be
 * NULL) and the shared step counter.  Synchronous. */
int rbsog_batch_get_state(rbsog_batch *b, double *r, double *v, uint64_t *step, void *stream);

/* One force evaluation of every system: total forces ([sum N][3], caller order, host or
 * device, may be NULL) and, if e is not NULL, R energy records.  Synchronous. */
int rbsog_batch_forces(rbsog_batch *b, double *F, rbsog_energy *e, void *stream);

/* Advance every system nsteps >= 0 steps (graph captured once on an internal stream,
 * replayed on stream).  If e is not NULL, R energy records after the last step are
 * written and the call is synchronous; with nsteps = 0 right after
 * rbsog_batch_set_state (no evaluation at the uploaded state yet) that fails with
 * RBSOG_EINVAL. */
int rbsog_batch_step(rbsog_batch *b, int32_t nsteps, rbsog_energy *e, void *stream);

/* Inject the next evaluation's modes for every system: sum(P) triples, host, not
 * (0,0,0).  Synchronous. */
int rbsog_batch_set_ksample(rbsog_batch *b, const int32_t *m_host);

/* Modes (sum(P) triples) and coefficients (sum(P) doubles) of the last evaluation, host
 * arrays, either may be NULL.  Synchronous. */
int rbsog_batch_get_ksample(rbsog_batch *b, int32_t *m_host, double *coef_host);

/* Layout: p_off and m_off (R + 1 entries each) and the structure-factor chunk (particles
 * per block, R entries) of each system; any output may be NULL. */
int rbsog_batch_layout(const rbsog_batch *b, int64_t *p_off, int64_t *m_off, int32_t *rho_chunk);

/* Set the structure-factor chunk of each system (R entries, each >= 64 particles per
 * block).  The chunk fixes the summation order of rho(k), so results are reproducible
 * for a fixed chunk; it changes only the launch shape, not what is computed.  Drops the
 * captured graph.  Synchronous. */
int rbsog_batch_set_rho_chunk(rbsog_batch *b, const int32_t *rho_chunk);

/* Launch shapes of every system: near_target is the number of target particles a
 * near-field brick (one 256-thread CTA: a run of cells in each of up to 2 x 4 rows) aims
 * at, up to 230 (the run length follows from each system's cell occupancy, capped by the
 * brick's shared-memory buffers; default 230), rho_target the particles
 * per structure-factor block (each system's chunk is its N split evenly near that
 * size; default 512).  The near-field shape changes only the order of the near-energy
 * sum; the structure-factor shape the order of rho(k).  Drops the captured graph.
 * Synchronous. */
int rbsog_batch_set_shapes(rbsog_batch *b, double near_target, int32_t rho_target);

/* Autotuner: times the near-field kernel and the structure-factor kernels (median of
 * reps evaluations each) over a fixed set of candidate shapes on the current state,
 * applies the fastest and returns it (either output may be NULL).  The step and draw
 * counters are restored afterwards, so a batch tuned right after
 * rbsog_batch_set_state follows the same trajectory as one given the same shapes
 * with rbsog_batch_set_shapes.  Synchronous. */
int rbsog_batch_tune(rbsog_batch *b, int32_t reps, double *near_target, int32_t *rho_target, void *stream);

/* Advance nsteps >= 1 steps with eager launches and CUDA events around each kernel
 * group (the groups of rbsog_profile_name); ms[RBSOG_NPROF] receives the summed
 * milliseconds per group.  Synchronous. */
int rbsog_batch_profile(rbsog_batch *b, int32_t nsteps, double *ms, void *stream);

/* The form of a step: enable = 0 replays the batched kernels (one launch per kernel over
 * all systems, 11 per step) from a CUDA graph; enable != 0 runs the whole step (or force
 * evaluation) as one persistent cooperative launch, captured in the graph the same way.
 * Its CTAs are all resident and walk the step's phases, meeting at grid barriers between
 * dependent phases; the near-field tiles and the structure-factor blocks of every system
 * form work lists that CTAs take items from as they finish.  Forces and trajectories are
 * bit-identical in both forms (the same per-block arithmetic); the near energies differ
 * in rounding (another grouping of the per-warp partial sums).  Energies of evaluations
 * before a switch cannot be read after it (RBSOG_EINVAL until the next evaluation).
 * rbsog_batch_profile and rbsog_batch_tune time the graph form's kernels.  Every
 * grid-barrier wait is bounded (rbsog_batch_set_wait_limit): a wait that gives up makes
 * the next synchronous call return RBSOG_ETIMEOUT (the pass that timed out is not valid).
 * RBSOG_EUNSUPPORTED if the device has no cooperative launch.  Synchronous. */
int rbsog_batch_set_persistent(rbsog_batch *b, int32_t enable);

/* Polls of one grid-barrier wait of the persistent step before it gives up (>= 1; default
 * 2e7, about a second or more).  Synchronous. */
int rbsog_batch_set_wait_limit(rbsog_batch *b, int64_t polls);

/* Message of the last failed call on b (or of the last failed rbsog_batch_init when b
 * is NULL). */
const char *rbsog_batch_last_error(const rbsog_batch *b);

/* Release every device buffer and graph of b.  Synchronous.  NULL is a no-op. */
void rbsog_batch_free(rbsog_batch *b);

/* ---- Job server with continuous batching ---------------------------------------------
 * MD jobs (each an independent FP32 system as in the batch functions, with its own step
 * count) are submitted with an arrival time.  rbsog_server_run admits arrived jobs in
 * arrival order as soon as the resident arenas have room for them (particles, cells,
 * modes and job slots, fixed at creation; a job that does not fit yet waits and later
 * arrivals may pass it), advances every resident job together in rounds of at most
 * steps_per_round steps (every kernel of a step one launch over all resident jobs, the
 * step a CUDA graph), and retires each job after its last step: its final state and
 * energies are read back to the host and the remaining jobs are compacted.  A job's
 * first pass evaluates its initial forces; a job draws the same modes and Langevin noise,
 * and gives the same result bit for bit, alone and among any other jobs.  A device error
 * of one job (cell overflow, sampler limit) fails that job only.  Times are seconds on
 * the server's clock, which starts at rbsog_server_create.  The server runs on the
 * calling thread; its functions must not be called concurrently. */

#define RBSOG_JOB_QUEUED 0
#define RBSOG_JOB_RESIDENT 1
#define RBSOG_JOB_DONE 2
#define RBSOG_JOB_FAILED 3

typedef struct rbsog_server_config {
    int64_t max_particles;   /* resident particles (sum of N), >= 2 */
    int64_t max_cells;       /* resident cells (sum of the jobs' cell counts) */
    int64_t max_modes;       /* resident modes (sum of P) */
    double near_target;      /* near-field shape (see rbsog_batch_set_shapes); 0 selects 230 */
    int32_t max_jobs;        /* resident jobs at once, 1 .. 65536 */
    int32_t steps_per_round; /* steps between admission points, >= 1 */
    int32_t rho_target;      /* structure-factor shape; 0 selects 512 */
    int32_t device;          /* CUDA device ordinal */
    int32_t reserved[2];     /* must be 0 */
} rbsog_server_config;

typedef struct rbsog_job_info {
    int32_t status;          /* RBSOG_JOB_* */
    int32_t error;           /* RBSOG_* status of a failed job */
    int64_t N;
    int32_t nsteps;
    int32_t steps_done;
    double t_arrival;        /* server clock, seconds */
    double t_admit;          /* -1 until admitted */
    double t_done;           /* -1 until done or failed */
    uint64_t footprint_bytes; /* device memory the job occupied while resident */
    rbsog_energy energy;     /* after the last step */
} rbsog_job_info;

/* Create a server: allocates the arenas on cfg->device.  On failure *out is NULL and
 * rbsog_server_last_error(NULL) holds the message. */
int rbsog_server_create(const rbsog_server_config *cfg, rbsog_server **out);

/* Submit a job: params (precision RBSOG_FP32; device ignored), N particles, host arrays
 * q[N], m[N], r[N][3] and optional v[N][3] (copied), nsteps >= 0 steps, and the arrival
 * time on the server clock (t_arrival < 0: now).  The job becomes eligible for admission
 * once the clock passes t_arrival.  *job_id receives its handle (0, 1, 2, ...).  Host
 * only; invalid parameters are reported when the job is considered for admission (the
 * job then fails), as is a job larger than the arenas (RBSOG_ENOMEM, once nothing else
 * is resident). */
int rbsog_server_submit(rbsog_server *s, const rbsog_params *params, int64_t N, const double *q, const double *m,
                        const double *r, const double *v, int32_t nsteps, double t_arrival, int64_t *job_id);

/* Run the admission / round / retirement loop until every submitted job is done or
 * failed (t_until < 0), or until the server clock passes t_until.  Sleeps while nothing
 * is resident and the next arrival is in the future.  Returns a non-zero status only for
 * errors of the server itself (CUDA failures), not for failed jobs. */
int rbsog_server_run(rbsog_server *s, double t_until);

/* Status and timings of a job; for a done job also its final positions r_out[N][3] and
 * velocities v_out[N][3] (host arrays, either may be NULL).  Returns the job's error for
 * a failed job and RBSOG_EINVAL if a state is asked of a job that is not done. */
int rbsog_server_job(rbsog_server *s, int64_t job_id, rbsog_job_info *info, double *r_out, double *v_out);

/* Counters: rounds, admissions, retirements, seconds the device was busy with rounds,
 * particle-steps of done jobs, peak resident particles, peak resident jobs, seconds of
 * admission set-up (out8[8]). */
int rbsog_server_stats(const rbsog_server *s, double *out8);

/* The server clock (seconds since rbsog_server_create). */
double rbsog_server_clock(const rbsog_server *s);

const char *rbsog_server_last_error(const rbsog_server *s);

/* Release the arenas.  Synchronous.  NULL is a no-op. */
void rbsog_server_free(rbsog_server *s);

#ifdef __cplusplus
}
#endif

#endif /* RBSOG_H */
