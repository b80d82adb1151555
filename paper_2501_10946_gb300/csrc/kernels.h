// Launchers of the RBSOG kernels (internal to the library).
#pragma once

#include "common.cuh"

namespace rbsog {

// ---- cell list and integrator, first half (k_cells.cu) ----
struct BinArgs {
    State in;                 // rest buffer (cell-sorted order of the last build)
    State out;                // work buffer, same index k
    const void *F;            // forces of the rest order, SoA [3][N]: float (FP32) or double (FP64)
    int integrate;            // 0 none, 1 velocity Verlet (kick + drift), 2 BAOAB (B A O A)
    double dt, c1, kT;
    double okT;               // (1 - c1^2) k_B T: the FP32 build's noise variance per unit 1/m
    float dt_f, hdt_f, c1_f, okT_f;   // dt, dt/2, c1, okT rounded to FP32 (set_bin_floats)
    unsigned long long seed;
    DevCounters *ctr;
    uint32_t N;               // particles of this system
    uint32_t stride;          // SoA stride of F (N, or the batch total)
    uint32_t cell_base;       // first global cell of this system (0 for a single system)
    Box box;
    void *rec_w;              // particle records in this (work) order: uint4 (FP32) or Rec64 (FP64)
    void *rec_id;             // the same records at their particle ids (an order the storage does not change)
    uint32_t *cell, *slot, *count;
    double *K_part;           // nullptr, or per-block kinetic energy of the velocities this
                              // kernel leaves (the instantaneous temperature of calF)
};
// Fills the FP32 copies of dt, dt/2, c1 and okT from the doubles.
inline void set_bin_floats(BinArgs &a) {
    a.dt_f = (float)a.dt;
    a.hdt_f = (float)(0.5 * a.dt);
    a.c1_f = (float)a.c1;
    a.okT_f = (float)a.okT;
}
void launch_bin(int prec, const BinArgs &a, cudaStream_t st);
void launch_scan(uint32_t *count, uint32_t *tile_sums, uint32_t *cell_start, int ncell, uint32_t N,
                 cudaStream_t st);
// keys[cell_start[cell[k]] + slot[k]] = (id[k] << 32) | k: each cell's keys, in the order
// the atomics gave the slots
void launch_scatter(const uint32_t *cell, const uint32_t *slot, const uint32_t *cell_start, const uint32_t *id,
                    uint32_t N, unsigned long long *keys, cudaStream_t st);
// Move R systems to a new particle layout: system r's particles old_off[r] + i (rest
// state and forces F, SoA stride `stride`) go to new_off[r] + i of `to` and F_to.
void launch_relayout(State from, State to, const float *F_from, float *F_to, uint32_t stride,
                     const uint32_t *old_off, const uint32_t *new_off, int R, uint32_t Nnew, cudaStream_t st);
// The cell of each key orders it by particle id (rank among the cell's keys); a cell over
// the occupancy limit sets kErrCellOverflow in ctr[0], or, with c_off (R + 1 first cells
// of R systems), in the counter of the system that owns the cell.
struct GatherArgs {
    State in;                 // work buffer
    State out;                // rest buffer (new cell-sorted order)
    const unsigned long long *keys;   // launch_scatter's output
    const uint32_t *cell;     // cell of each work-order particle
    const uint32_t *cell_start;
    DevCounters *ctr;
    const uint32_t *c_off;    // nullptr for one system
    int R;
    const void *rec_w;        // records of the work order (k_bin's)
    void *rec;                // uint4 (FP32) or Rec64 (FP64) records in the new order
    uint32_t N;
};
void launch_gather(int prec, const GatherArgs &g, cudaStream_t st);
// Caller rows [N][3] (r, v, F) in and out of one context.  Each pointer is device memory or
// the mapped address of pinned host memory: the kernels move whole lines either way.
// A state upload: particle k = caller index k, 1/m from the inverse masses invm_user.
void launch_set_state(const double *r, const double *v, const double *q_user, const double *invm_user, State rest,
                      uint32_t N, Box box, DevCounters *ctr, cudaStream_t st);
// pos[caller index] = place in the rest order (the inverse of rest.id), for the reads below
void launch_rest_pos(const uint32_t *id, uint32_t N, uint32_t *pos, cudaStream_t st);
void launch_get_state(State rest, const uint32_t *pos, uint32_t N, double *r_out, double *v_out, cudaStream_t st);
// F_in ([N][3] doubles, caller order = the rest order after a state upload) into the SoA
// force buffer F of the build's precision; sets ctr->fvalid
void launch_set_forces(int prec, const double *F_in, void *F, uint32_t N, DevCounters *ctr, cudaStream_t st);
// the SoA forces of the rest order into F_out ([N][3] doubles, caller order)
void launch_get_forces(int prec, const uint32_t *pos, const void *F, uint32_t N, double *F_out, cudaStream_t st);
void launch_set_forces_f32(const float *F_in, float *F, uint32_t N, DevCounters *ctr, cudaStream_t st);
void launch_get_forces_f32(const uint32_t *pos, const float *F, uint32_t N, float *F_out, cudaStream_t st);

// ---- sampler and normalisation (k_sample.cu) ----
// A mixture of separable components: component c has weight mix and per-axis alias
// tables (ax_off, ax_nmax) over |n| <= nmax.
struct SamplerTables {
    int mtot;                 // number of mixture components
    const unsigned long long *mix_thr; const int *mix_alias;     // [mtot] keep thresholds, aliases
    const int *ax_off;        // [mtot*3] offset into ax_prob/ax_alias
    const int *ax_nmax;       // [mtot*3]
    const unsigned long long *ax_thr; const int *ax_alias;
};
struct SampleArgs {
    SamplerTables tab;
    int P;
    unsigned long long seed;
    double tpl[3];            // 2 pi / L
    double A;                 // k_B T V
    double Q2;                // sum q^2
    Yterms y;                 // psi(k) of the adaptive correction (Eq. 62 with the kernel's transform)
    double S, V;
    // signed far-field transform when it may change sign (EGS): the modes come from the
    // envelope sum |fA_m| exp(-k^2 finv4b_m) and coef carries Fhat / Fhat_env; nfh = 0 otherwise
    int nfh;
    double fA[kMaxGauss], finv4b[kMaxGauss];
    int measure;              // RBSOG_SAMPLING_*: calF of Eq. (62), 1, k^2, Eq. (62) with 4 pi
    double Q2a;               // sum q^2 in the acceptance ratio (4 pi sum q^2 for the Debye form)
    DevCounters *ctr;
    const int *inject_m;      // [P*3]
    int *m_out;               // [P*3]
    double *coef_out;         // [P]
    const double *temp;       // nullptr, or {k_B T V, S} of this evaluation at the instantaneous
                              // temperature (launch_temperature), which replace A and S
    // FP32 pre-test of the acceptance test (calF of Eq. 62 with one Yukawa term): FP32
    // copies of 2 pi / L, lambda^-2 and Q2a, and whether their ranges allow it
    // (sample_set_prefilter); the FP64 test still decides every draw the pre-test leaves open
    float tplf[3], il2f, Q2af;
    int f32pre;
};
void sample_set_prefilter(SampleArgs *a);
void launch_sample(const SampleArgs &a, cudaStream_t st);
// Metropolis-Hastings chains (one per batch slot): state m and proposals made t (t = 0: the
// chain has not started)
struct MHChainArgs {
    int *m;                   // [P*3]
    unsigned long long *t;    // [P]
    int sweeps, burnin;
};
void launch_sample_mh(const SampleArgs &a, const MHChainArgs &c, cudaStream_t st);
// Instantaneous temperature and S at it: k_B T = 2 K / (3 N) from the kinetic-energy
// partials of k_bin, S(T) = sum_j calF(k2_j; T) W_j over the distinct |k|^2 of the mode
// support (W_j: multiplicity times Fhat_env at k2_j).  out = {k_B T V, S, k_B T}.
struct TempArgs {
    const double *K_part;
    int nK;
    double two_3N;            // 2 / (3 N)
    double V, Q2;
    Yterms y;
    int measure;
    const double *k2, *W;
    int n;
    double *part;             // [kTempBlocks]
    unsigned int *done;       // arrival counter (0 between launches)
    double *out;              // [3]
};
constexpr int kTempBlocks = 64;
void launch_temperature(const TempArgs &a, cudaStream_t st);
struct SArgs {
    int mtot;
    double A[kMaxGauss], inv4b[kMaxGauss];   // Fhat(k) = sum_m A_m exp(-k^2 inv4b_m)
    double tpl[3];
    double kmax2;
    int nmax[3];
    double kTV, Q2;
    Yterms y;
    int measure;
};
void launch_S(const SArgs &a, double *partials, cudaStream_t st);   // partials[2*nmax[0]+1]

// ---- forces (k_forces.cu) ----
struct NearArgs {
    NearConsts nc;
    const void *rec;
    const uint32_t *cell_start;
    Box box;
    uint32_t N;                // particles of this system
    uint32_t stride;           // SoA stride of Fn (N, or the batch total)
    void *Fn;                  // near force SoA [3][stride] (float or double), global particle index
    double *U_part;            // near energy partials, one per warp
    DevCounters *ctr;          // error bits: skip the pair loops when the cell build overflowed
};
int launch_near(int prec, const NearArgs &a, cudaStream_t st);   // returns #energy partials (one per warp)
struct RhoArgs {
    const void *rec;
    uint32_t N;
    const int *m;              // [P*3]
    int P;
    double2 *partial;          // [G][P]
    int G;
};
int rho_blocks(int prec, uint32_t N, int P);
void launch_rho(int prec, const RhoArgs &a, cudaStream_t st);
struct RhoFinalArgs {
    const double2 *partial;
    int G, P;
    const int *m;
    const double *coef;
    double tpl[3];
    double2 *rho;              // [P]
    void *gtab;                // gather table: float (FP32) / double (FP64), [P] x {ckx,cky,ckz,Re,Im} + int m
    double *Ufar;              // [P]: coef_l |rho_l|^2 / 2
    DevCounters *ctr;
    int keep_draw;             // 1: the draw counter is not advanced (a reduced rho set from outside)
    // launch_rho_final: the eight warp groups of each 32 modes in blocks of their own, the
    // group sums in wsum [8][P] and the groups' arrivals in wdone [ceil(P/32)] (zero between
    // launches: the last block of each 32 modes resets its counter)
    double2 *wsum;
    unsigned int *wdone;
};
void launch_rho_final(int prec, const RhoFinalArgs &a, cudaStream_t st);
struct FarArgs {
    const void *rec;
    uint32_t N;                // particles of this system
    uint32_t stride;           // SoA stride of Fn and F
    int P;
    const void *gtab;
    const int *m;
    const void *Fn;            // near force (SoA)
    void *F;                   // total force out (SoA, same precision)
    State st;                  // rest state (velocities updated when integrate)
    int integrate;
    double dt;
    double *K_part;            // per-block kinetic energy
    double *F_user;            // optional [N][3] total force in caller order
    double *Fn_user;           // optional near part
    double *Ff_user;           // optional far part
    const DevCounters *ctr;    // integrate only once the forces of the state are valid
};
int launch_far(int prec, const FarArgs &a, cudaStream_t st);     // returns #blocks
struct EnergyArgs {
    const double *U_part; int nU;
    const double *K_part; int nK;
    const double *Ufar; int nUfar;   // per-mode U*_F terms
    double Ufar0;              // k = 0 term
    double Uself;
    double *out;               // [5]: U_near, U_far, U_self, K, total
    DevCounters *ctr;
    double *scratch;           // [3 kEnergyBlocks] per-block sums (single system)
    unsigned int *done;        // arrival counter of the blocks (0 between launches)
};
constexpr int kEnergyBlocks = 32;
// Single system: kEnergyBlocks blocks, the last to finish adds their sums in a fixed order
// (the partials of the last force evaluation; launched when the energies are read).
void launch_energy(const EnergyArgs &a, cudaStream_t st);
// End of a single system's force evaluation: fvalid = 1, step += 1 when advance_step and
// the forces were valid before.
void launch_close_eval(DevCounters *ctr, int advance_step, cudaStream_t st);
void launch_close_eval_batch(DevCounters *ctr, int R, int advance_step, cudaStream_t st);

// ---- batched systems: one launch per kernel over every system --------------------
constexpr size_t kGTab32Bytes = 32;   // one FP32 gather-table entry (int4 + float4)
// items[r] = first block of system r, items[R] = total blocks; argument arrays in device
// memory hold each system's arguments with pointers already offset into the
// concatenated buffers.
void launch_bin_batch(const BinArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st);
void launch_sample_batch(const SampleArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st);
// FP32 pair constants of one system for the near-field bricks, each duplicated into both
// halves of a 64-bit word for packed FP32x2 arithmetic (near_f32_consts builds them).
struct alignas(16) NearF {
    int mtot;
    int two;                                // a second Yukawa term (EGS screening)
    unsigned long long nl2;                 // -log2(e)/lambda
    unsigned long long il2;                 // 1/lambda
    unsigned long long ly1;                 // log2 of the first term's weight
    unsigned long long nl2b, il2b, ly2, sg2;   // second term: -log2(e)/lambda_2, 1/lambda_2, log2|y2|, sign
    unsigned long long nb[kMaxGauss];       // -b_m log2(e)
    unsigned long long naf[kMaxGauss];      // -a_m (the energy's SOG sum is accumulated negated)
    unsigned long long cf[kMaxGauss];       // c_m
};
NearF near_f32_consts(const NearConsts &c);
// Near-field geometry of one system: bricks of W cells along x in each of by x bz rows
// (tiles_x x tiles_y x tiles_z of them), or the per-particle path (tiled = 0: fewer than 3
// cells on an axis; W then holds the system's first global record index in a batch).
struct NearBatchGeom {
    int tiled;
    int W, tiles_x, tiles_y, tiles_z, by, bz;
};
constexpr int kNearBrickThreads = 256;      // threads per near-field brick (CTA)
constexpr double kNearBrickTarget = 230.0;  // targets per brick aimed at by default
// Bricks of one system aiming at `target` targets each (capped by the brick's buffers);
// returns their number (0 when the box has fewer than 3 cells on an axis).
uint32_t near_bricks(const Box &box, uint32_t N, double target, NearBatchGeom *g);
// Row tiles of the FP64 build: staged particles per CTA and the widest tile in cells.
constexpr int kNearCapSingle = 1280;
constexpr int kNearMaxWSingle = 48;
// target: particles per CTA the tile width aims at (capped by the staging buffer `cap`);
// threads: threads per CTA of the per-particle path (boxes under 3 cells per axis);
// max_w: widest tile in cells (tiles span at most n_x - 2 cells)
void near_geometry(const Box &box, uint32_t N, int *tiled, int *W, int *tiles_x, uint32_t *nblocks,
                   double target = 110.0, int cap = kNearCapSingle, int threads = 128,
                   int max_w = kNearMaxWSingle);
// one brick (or per-particle block) per CTA of every system; nf: the systems' pair constants
void launch_near_batch(const NearArgs *args, const NearF *nf, const NearBatchGeom *geom, const uint32_t *items,
                       int R, uint32_t nblocks, cudaStream_t st);
void launch_rho_batch(const RhoArgs *args, const int *chunk, const uint32_t *items, int R, uint32_t nblocks,
                      cudaStream_t st);
void launch_rho_final_batch(const RhoFinalArgs *args, const uint32_t *items, int R, uint32_t nblocks,
                            cudaStream_t st);
void launch_far_batch(const FarArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st);
void launch_energy_batch(const EnergyArgs *args, int R, cudaStream_t st);

// ---- persistent batched step (k_persist.cuh): one cooperative launch per pass ----
// Grid-barrier state and the work counters of the near-field / structure-factor phase.
// count, q_near, q_rho return to 0 after a completed launch; status is sticky (1: a
// barrier wait gave up) until the host clears it.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int q_near, q_rho;
    int status;
    int pad[3];
};
struct PersistArgs {
    const BinArgs *bin; const uint32_t *it_bin; uint32_t nb_bin;
    const SampleArgs *sample; const uint32_t *it_sample; uint32_t nb_sample;   // 4-slot sample blocks
    uint32_t *count, *tile_sums, *cell_start; int ncell, ntiles; uint32_t N;
    const uint32_t *cell, *slot, *id; unsigned long long *keys;
    GatherArgs gather;
    const NearArgs *near; const NearF *nearf; const NearBatchGeom *geom; const uint32_t *it_near; uint32_t nb_near;
    const RhoArgs *rho; const int *chunk; const uint32_t *it_rho; uint32_t nb_rho;
    const RhoFinalArgs *rf; const uint32_t *it_rf; uint32_t nb_rf;
    const FarArgs *far; const uint32_t *it_far; uint32_t nb_far;
    DevCounters *ctr; int R; int advance;
    GridBar *bar; long long wait_limit;   // polls of a barrier wait before it gives up
};
size_t persist_smem_bytes();
// CTAs of the cooperative grid on `device` (all resident); returns a cudaError_t value
int persist_grid(int device, int *grid);
cudaError_t launch_step_persist(const PersistArgs &a, int grid, cudaStream_t st);
// state of system r: rest buffer (offset), its charges and masses, first particle in the
// caller's concatenated arrays
struct SysStateArgs {
    State rest;
    const double *q_user, *m_user;
    uint32_t N, p_off;
    Box box;
};
// also clears the step counter and error bits of ctr[0 .. nctr-1]
void launch_set_state_batch(const SysStateArgs *args, const uint32_t *items, int R, uint32_t nblocks,
                            const double *r, const double *v, DevCounters *ctr, int nctr, cudaStream_t st);
void launch_get_state_batch(const SysStateArgs *args, const uint32_t *items, int R, uint32_t nblocks, double *r_out,
                            double *v_out, cudaStream_t st);
// blocks one system takes in each batched kernel
uint32_t bin_batch_blocks(uint32_t N);           // also set/get state
uint32_t sample_batch_blocks(int P);
uint32_t rho_batch_blocks(int G, int P);         // G particle chunks x ceil(P/256) mode passes
uint32_t rho_final_batch_blocks(int P);
uint32_t far_batch_blocks(uint32_t N);

}  // namespace rbsog
