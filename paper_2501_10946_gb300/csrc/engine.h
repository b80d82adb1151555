// Resident-set engine (internal to the library): any number of independent FP32 systems
// held in fixed-capacity device arenas and advanced together, every kernel of the step
// one launch over all resident systems.  The batch ABI (a fixed set of systems) and the
// job server (systems that join and leave between rounds) are both built on it.
//
// Layout: resident systems are concatenated system-major.  System r owns particles
// p_off[r] .. p_off[r+1]-1 of every per-particle buffer (SoA arrays of three components
// use the particle capacity as their stride, so a system's range never depends on the
// others), cells c_off[r] .. c_off[r+1]-1 of the global cell list and modes
// m_off[r] .. m_off[r+1]-1.  The counting sort runs once over all cells; since cells and
// particles are ordered system-major with no gaps, the sorted order keeps every system
// inside its own particle range.  Kernels map a block to (system, local block) through
// prefix arrays of per-system block counts and read the system's arguments (pointers
// already offset) from device arrays.  Each system owns its step/draw counters, its
// error bits and a forces-valid flag, so it follows the same Philox streams and the same
// arithmetic alone and among others.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "common.cuh"
#include "kernels.h"
#include "system.h"

struct rbsog_batch {
    // capacities (fixed at creation)
    uint32_t capN = 0;
    int capC = 0, capP = 0, capR = 0;
    int device = 0;
    // resident systems
    int R = 0;
    uint32_t Ntot = 0;
    int Ctot = 0, Ptot = 0;
    std::vector<rbsog::HostSystem> sys;
    std::vector<uint32_t> p_off{0}, c_off{0}, m_off{0};   // R + 1 entries
    std::vector<int> rho_chunk;                          // particles per structure-factor block
    double near_target = rbsog::kNearBrickTarget;        // targets per near-field brick
    int rho_target = 512;
    bool dirty = true;                                   // arguments need rebuilding
    bool force_valid = false;                            // batch API: forces of the state evaluated
    std::string err;
    // device arenas
    rbsog::State rest{}, work{};
    double *stage_a = nullptr, *stage_b = nullptr;       // [3 capN] caller-order staging
    double *stage_qm = nullptr;                          // [2 capN]: charges, then masses (admission)
    float *F = nullptr, *Fn = nullptr;                   // SoA [3][capN]
    uint4 *rec_w = nullptr;                              // records in the work order [capN]
    uint4 *rec_id = nullptr;                             // records at system offset + particle id [capN]
    uint4 *rec = nullptr;
    uint32_t *cell = nullptr, *slot = nullptr, *count = nullptr, *tile_sums = nullptr, *cell_start = nullptr;
    unsigned long long *keys = nullptr;
    int *modes = nullptr, *inject_m = nullptr;
    double *coef = nullptr, *Ufar = nullptr, *energy = nullptr;
    double2 *rho = nullptr;
    unsigned char *gtab = nullptr;
    rbsog::DevCounters *ctr = nullptr;                   // [capR]
    // grow-only buffers
    double2 *partial = nullptr;
    double *U_part = nullptr, *K_part = nullptr;
    size_t cap_part = 0, cap_upart = 0, cap_kpart = 0;
    unsigned long long *mix_thr = nullptr, *ax_thr = nullptr;   // alias keep thresholds
    int *mix_alias = nullptr, *ax_off = nullptr, *ax_nmax = nullptr, *ax_alias = nullptr;
    size_t cap_mix = 0, cap_ax = 0;
    // per-system arguments (device arrays of capR entries) and block prefixes
    rbsog::BinArgs *d_bin[2] = {nullptr, nullptr};       // [0] force evaluation only, [1] step
    rbsog::FarArgs *d_far[2] = {nullptr, nullptr};
    rbsog::FarArgs *d_far_user = nullptr;
    rbsog::EnergyArgs *d_energy[2] = {nullptr, nullptr};
    rbsog::SampleArgs *d_sample = nullptr;
    rbsog::NearArgs *d_near = nullptr;
    rbsog::NearF *d_nearf = nullptr;                     // each system's FP32 pair constants
    rbsog::NearBatchGeom *d_geom = nullptr;
    rbsog::RhoArgs *d_rho = nullptr;
    int *d_chunk = nullptr;
    rbsog::RhoFinalArgs *d_rf = nullptr;
    rbsog::SysStateArgs *d_state = nullptr;
    rbsog::SysStateArgs *d_state_sub = nullptr;          // state arguments of a system subset
    std::vector<rbsog::SysStateArgs> h_state;
    uint32_t *d_items = nullptr;                         // 6 prefix arrays of capR + 1 entries
    uint32_t *d_coff = nullptr;                          // c_off on the device (capR + 1)
    uint32_t *d_off2 = nullptr;                          // relayout offsets (2 (capR + 1))
    uint32_t *d_sub_items = nullptr;                     // items of a system subset (capR + 1)
    uint32_t nb[6] = {0, 0, 0, 0, 0, 0};                 // total blocks: bin, sample, near, rho, rho_final, far
    std::vector<uint32_t> h_items;                       // host copy of the bin prefix
    std::vector<rbsog::FarArgs> h_far;                   // host copy of d_far[0]
    std::vector<void *> allocs;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;                  // structure factor beside the near field
    cudaEvent_t ev_fork = nullptr, ev_bin = nullptr, ev_join = nullptr;
    cudaGraphExec_t graph = nullptr;
    // persistent step: one cooperative launch per pass (near-field tiles of 128 threads)
    bool persistent = false;
    bool energies_stale = false;                         // partials written in the other layout
    int pgrid = 0;                                       // CTAs of the cooperative grid
    rbsog::GridBar *bar = nullptr;
    long long wait_limit = 20000000;                     // polls of a grid-barrier wait
};

namespace rbsog {

struct EngineCaps {
    uint32_t particles;
    int cells, modes, systems;
};

// Allocate the arenas.  Returns an RBSOG_* status; the message is in b->err.
int engine_alloc(rbsog_batch *b, const EngineCaps &caps, int device);
void engine_release(rbsog_batch *b);
// Bytes of device memory a system takes in the arenas (particles, cells, modes and
// per-block partials at the engine's shapes).
size_t engine_footprint(const rbsog_batch *b, const HostSystem &h);
// each system's energies of its last force evaluation into energy[5 R]; enqueued on st
int engine_reduce_energies(rbsog_batch *b, cudaStream_t st);
// True if the system fits the remaining capacity.
bool engine_fits(const rbsog_batch *b, const HostSystem &h);
// Append a system (host bookkeeping only; its state is set with engine_set_state).
int engine_append(rbsog_batch *b, HostSystem &&h);
// Keep the systems with keep[r] != 0 (in order), moving their state and forces; their
// counters move with them.  Synchronous.
int engine_retain(rbsog_batch *b, const std::vector<char> &keep, cudaStream_t st);
// Rebuild tables, partial buffers and arguments after membership or shape changes.
int engine_commit(rbsog_batch *b);
// State of systems first .. first+count-1 from caller-order device arrays whose element 0
// is the first particle of system `first`; clears their step counter, error bits and
// forces-valid flag.  With q and m (device, same indexing) the systems are initialised
// (identity order, charges and masses); without, resident particles keep their places,
// charges and masses.  Synchronous with respect to the host arguments.
int engine_set_state(rbsog_batch *b, int first, int count, const double *r, const double *v, const double *q,
                     const double *m, cudaStream_t st);
// Caller-order positions/velocities of systems first .. first+count-1 into device arrays
// (element 0 = first particle of system `first`).  Asynchronous.
int engine_get_state(rbsog_batch *b, int first, int count, double *r, double *v, cudaStream_t st);
// One pass over every resident system: set 0 evaluates forces only, set 1 steps.
int engine_enqueue(rbsog_batch *b, cudaStream_t st, int set, const FarArgs *far = nullptr, cudaEvent_t *ev = nullptr);
// n step passes replayed from a graph captured for the current membership.
int engine_launch_steps(rbsog_batch *b, int n, cudaStream_t st);
// Per-system counters (capR read back, R valid).  Synchronous.
int engine_counters(rbsog_batch *b, std::vector<DevCounters> *out);
// Error bits of every system to an RBSOG_* status (first error found).
int engine_status(rbsog_batch *b, const std::vector<DevCounters> &c, int r);
int engine_fail(rbsog_batch *b, int code, const std::string &msg);
int engine_cuda_fail(rbsog_batch *b, cudaError_t e, const char *where);

}  // namespace rbsog
