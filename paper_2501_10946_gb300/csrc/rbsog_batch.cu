// A batch of independent systems advanced together: every kernel of the step is one
// launch over all systems (FP32 path).
//
// Layout: the systems' particles, cells and modes are concatenated system-major.  System
// r owns particles p_off[r] .. p_off[r+1]-1 of every per-particle buffer, cells
// c_off[r] .. c_off[r+1]-1 of the global cell list and modes m_off[r] .. m_off[r+1]-1.
// The counting sort runs once over all cells; since the cells are ordered system-major,
// the sorted order keeps every system in its own particle range.  Every other kernel
// maps a block to (system, local block) through a prefix array of per-system block
// counts and reads that system's arguments (pointers already offset) from a device
// array, so the step is 12 launches whatever the number of systems, captured once as
// a CUDA graph.  Each system keeps its own box, SOG decomposition, P, seed, time step,
// ensemble and step/draw counters, so system r of a batch follows the same Philox
// streams as a single context built with the same parameters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rbsog.h"
#include "common.cuh"
#include "kernels.h"
#include "system.h"

using namespace rbsog;

struct rbsog_batch {
    int R = 0;
    uint32_t Ntot = 0;
    int Ctot = 0, Ptot = 0;
    int device = 0;
    std::string err;
    std::vector<HostSystem> sys;
    std::vector<uint32_t> p_off, c_off, m_off;         // R + 1 entries
    std::vector<int> rho_chunk;                        // particles per structure-factor block
    double near_target = 110.0;                        // particles per near-field CTA the tiles aim at
    size_t cap_part = 0, cap_upart = 0;                // allocated partial buffer entries
    // device buffers
    State rest{}, work{};
    double *q_user = nullptr, *m_user = nullptr, *stage_a = nullptr, *stage_b = nullptr;
    float *F = nullptr, *Fn = nullptr;
    uint32_t *s = nullptr;
    uint4 *rec = nullptr;
    uint32_t *cell = nullptr, *slot = nullptr, *count = nullptr, *tile_sums = nullptr, *cell_start = nullptr,
             *perm_src = nullptr;
    unsigned long long *keys = nullptr;
    int *modes = nullptr, *inject_m = nullptr;
    double *coef = nullptr, *Ufar = nullptr, *U_part = nullptr, *K_part = nullptr, *energy = nullptr;
    double2 *partial = nullptr, *rho = nullptr;
    unsigned char *gtab = nullptr;
    double *mix_prob = nullptr, *ax_prob = nullptr;
    int *mix_alias = nullptr, *ax_off = nullptr, *ax_nmax = nullptr, *ax_alias = nullptr;
    DevCounters *ctr = nullptr;                        // [R + 1]: systems, then the cell-list status
    // per-system kernel arguments (device arrays) and block prefixes
    BinArgs *d_bin[2] = {nullptr, nullptr};            // [0] force evaluation only, [1] step
    FarArgs *d_far[2] = {nullptr, nullptr};
    FarArgs *d_far_user = nullptr;                     // force evaluation with caller outputs
    EnergyArgs *d_energy[2] = {nullptr, nullptr};
    SampleArgs *d_sample = nullptr;
    NearArgs *d_near = nullptr;
    NearBatchGeom *d_geom = nullptr;
    RhoArgs *d_rho = nullptr;
    int *d_chunk = nullptr;
    RhoFinalArgs *d_rf = nullptr;
    SysStateArgs *d_state = nullptr;
    uint32_t *d_items = nullptr;                       // 6 prefix arrays of R + 1 entries
    uint32_t nb[6] = {0, 0, 0, 0, 0, 0};               // total blocks: bin, sample, near, rho, rho_final, far
    std::vector<FarArgs> h_far;                        // host copy of d_far[0]
    std::vector<void *> allocs;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool force_valid = false;
};

namespace {

enum { kItBin = 0, kItSample, kItNear, kItRho, kItRhoFinal, kItFar };

std::string g_batch_init_error;

int bfail(rbsog_batch *b, int code, const std::string &msg) {
    if (b) b->err = msg;
    else g_batch_init_error = msg;
    return code;
}

int bcuda_fail(rbsog_batch *b, cudaError_t e, const char *where) {
    return bfail(b, e == cudaErrorMemoryAllocation ? RBSOG_ENOMEM : RBSOG_ECUDA,
                 std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}

#define BCK(call, where)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return bcuda_fail(b, e_, where);   \
    } while (0)

template <typename T>
cudaError_t balloc(rbsog_batch *b, T **ptr, size_t count) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e == cudaSuccess) {
        b->allocs.push_back(p);
        *ptr = (T *)p;
    }
    return e;
}

// Copy a host vector to a device array, allocating the array on first use (the size of
// each array is fixed for the lifetime of the batch).
template <typename T>
cudaError_t upload(rbsog_batch *b, T **dst, const std::vector<T> &src) {
    if (*dst == nullptr) {
        cudaError_t e = balloc(b, dst, src.size());
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool dev_ptr(const void *ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

State offset_state(const State &s, size_t o) {
    State t;
    t.rx = s.rx + o; t.ry = s.ry + o; t.rz = s.rz + o;
    t.vx = s.vx + o; t.vy = s.vy + o; t.vz = s.vz + o;
    t.invm = s.invm + o; t.q = s.q + o; t.id = s.id + o;
    return t;
}

// Structure-factor chunking: about `target` particles per block (at least 64).
int chunk_for(uint32_t N, int target) {
    const uint32_t t = (uint32_t)std::max(64, target);
    const uint32_t G = (N + t - 1) / t;
    return (int)((N + G - 1) / G);
}

// Sizes of the per-block partial buffers: structure factor (double2), near energy, kinetic energy.
void partial_sizes(const rbsog_batch *b, size_t *part, size_t *upart, size_t *kpart) {
    *part = *upart = *kpart = 0;
    for (int r = 0; r < b->R; ++r) {
        const HostSystem &h = b->sys[r];
        const uint32_t c = (uint32_t)b->rho_chunk[r];
        *part += (size_t)((h.N + c - 1) / c) * 8 * (size_t)h.p.P;
        int tiled, W, tiles_x;
        uint32_t nbn;
        near_geometry(h.box, h.N, &tiled, &W, &tiles_x, &nbn, b->near_target);
        *upart += 4 * (size_t)nbn;
        *kpart += far_batch_blocks(h.N);
    }
}

// Grow the partial buffers to the current shapes (old buffers stay allocated until free).
int ensure_partials(rbsog_batch *b) {
    size_t part, upart, kpart;
    partial_sizes(b, &part, &upart, &kpart);
    if (part > b->cap_part) {
        BCK(balloc(b, &b->partial, part), "alloc partials");
        b->cap_part = part;
    }
    if (upart + 4 > b->cap_upart) {
        BCK(balloc(b, &b->U_part, upart + 4), "alloc partials");
        b->cap_upart = upart + 4;
    }
    if (b->K_part == nullptr) BCK(balloc(b, &b->K_part, kpart + 1), "alloc partials");
    return RBSOG_OK;
}

int check_errors(rbsog_batch *b) {
    std::vector<DevCounters> hc(b->R + 1);
    BCK(cudaMemcpy(hc.data(), b->ctr, hc.size() * sizeof(DevCounters), cudaMemcpyDeviceToHost), "read device status");
    DevCounters h{};
    for (const DevCounters &x : hc) h.err |= x.err;
    if (h.err & kErrCellOverflow) return bfail(b, RBSOG_EOVERFLOW, "a cell holds more than 4096 particles");
    if (h.err & kErrSampler) return bfail(b, RBSOG_ETIMEOUT, "k-sampler exceeded its attempt limit");
    if (h.err & kErrNearStage) return bfail(b, RBSOG_ETIMEOUT, "near-field staging wait exceeded its limit");
    return RBSOG_OK;
}

int read_energies(rbsog_batch *b, rbsog_energy *e, cudaStream_t st) {
    std::vector<double> h(5 * (size_t)b->R);
    std::vector<DevCounters> hc(b->R);
    BCK(cudaMemcpyAsync(h.data(), b->energy, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "read energy");
    BCK(cudaMemcpyAsync(hc.data(), b->ctr, hc.size() * sizeof(DevCounters), cudaMemcpyDeviceToHost, st),
        "read counters");
    BCK(cudaStreamSynchronize(st), "synchronize");
    for (int r = 0; r < b->R; ++r) {
        const double *x = &h[5 * (size_t)r];
        e[r].U_near = x[0]; e[r].U_far = x[1]; e[r].U_self = x[2]; e[r].kinetic = x[3]; e[r].total = x[4];
        e[r].step = hc[r].step;
    }
    return check_errors(b);
}

// Per-system argument arrays (device), rebuilt when the structure-factor chunking changes.
int build_args(rbsog_batch *b) {
    const int R = b->R;
    std::vector<BinArgs> bin[2];
    std::vector<FarArgs> far[2];
    std::vector<EnergyArgs> en[2];
    std::vector<SampleArgs> sa(R);
    std::vector<NearArgs> na(R);
    std::vector<NearBatchGeom> geom(R);
    std::vector<RhoArgs> ra(R);
    std::vector<RhoFinalArgs> rf(R);
    std::vector<SysStateArgs> ss(R);
    std::vector<uint32_t> items(6 * (size_t)(R + 1), 0u);
    for (int k = 0; k < 2; ++k) {
        bin[k].resize(R);
        far[k].resize(R);
        en[k].resize(R);
    }
    size_t part_off = 0, u_off = 0, k_off = 0, ax_base = 0;
    uint32_t it[6] = {0, 0, 0, 0, 0, 0};
    for (int r = 0; r < R; ++r) {
        const HostSystem &h = b->sys[r];
        const rbsog_params &p = h.p;
        const size_t po = b->p_off[r], mo = b->m_off[r];
        const uint32_t N = h.N;
        const int P = p.P;
        const int mode = p.ensemble == RBSOG_LANGEVIN ? 2 : 1;
        // cell list + opening half of the integrator
        for (int k = 0; k < 2; ++k) {
            BinArgs &a = bin[k][r];
            a.in = offset_state(b->rest, po);
            a.out = offset_state(b->work, po);
            a.F = b->F + po;
            a.integrate = k ? mode : 0;
            a.dt = p.dt;
            a.c1 = std::exp(-p.langevin_gamma * p.dt);
            a.kT = h.kT;
            a.seed = p.seed;
            a.ctr = b->ctr + r;
            a.N = N;
            a.stride = b->Ntot;
            a.cell_base = b->c_off[r];
            a.box = h.box;
            a.s = b->s + po;
            a.cell = b->cell + po;
            a.slot = b->slot + po;
            a.count = b->count;
        }
        // sampler: this system's tables inside the concatenated ones
        {
            SampleArgs &a = sa[r];
            const int mt = h.sog.mtot();
            size_t mix_base = 0;
            for (int q = 0; q < r; ++q) mix_base += (size_t)b->sys[q].sog.mtot();
            a.tab = SamplerTables{mt, b->mix_prob + mix_base, b->mix_alias + mix_base, b->ax_off + 3 * mix_base,
                                  b->ax_nmax + 3 * mix_base, b->ax_prob + ax_base, b->ax_alias + ax_base};
            ax_base += h.ax_prob.size();
            a.P = P;
            a.seed = p.seed;
            for (int d = 0; d < 3; ++d) a.tpl[d] = h.box.tpl[d];
            a.A = h.kT * h.V;
            a.Q2 = h.Q2;
            a.inv_lam2 = 1.0 / (h.lam * h.lam);
            a.S = h.S;
            a.V = h.V;
            a.ctr = b->ctr + r;
            a.inject_m = b->inject_m + 3 * mo;
            a.m_out = b->modes + 3 * mo;
            a.coef_out = b->coef + mo;
        }
        // near field: global records and forces, this system's cell range
        int tiled, W, tiles_x;
        uint32_t nbn;
        near_geometry(h.box, N, &tiled, &W, &tiles_x, &nbn, b->near_target);
        geom[r] = NearBatchGeom{tiled, tiled ? W : (int)po, tiles_x};
        {
            NearArgs &a = na[r];
            a.nc = h.nconsts;
            a.rec = b->rec;
            a.cell_start = b->cell_start + b->c_off[r];
            a.box = h.box;
            a.N = N;
            a.stride = b->Ntot;
            a.Fn = b->Fn;
            a.U_part = b->U_part + u_off;
            a.ctr = b->ctr + b->R;   // cell-list status (overflow is detected by the global sort)
        }
        // structure factor and its reduction
        const int chunk = b->rho_chunk[r];
        const int G = (int)((N + (uint32_t)chunk - 1) / (uint32_t)chunk);
        {
            RhoArgs &a = ra[r];
            a.rec = b->rec + po;
            a.N = N;
            a.m = b->modes + 3 * mo;
            a.P = P;
            a.partial = b->partial + part_off;
            a.G = G;
        }
        {
            RhoFinalArgs &a = rf[r];
            a.partial = b->partial + part_off;
            a.G = G;
            a.P = P;
            a.m = b->modes + 3 * mo;
            a.coef = b->coef + mo;
            for (int d = 0; d < 3; ++d) a.tpl[d] = h.box.tpl[d];
            a.rho = b->rho + mo;
            a.gtab = b->gtab + kGTab32Bytes * mo;
            a.Ufar = b->Ufar + mo;
            a.ctr = b->ctr + r;
        }
        const uint32_t nbf = far_batch_blocks(N);
        for (int k = 0; k < 2; ++k) {
            FarArgs &a = far[k][r];
            a.rec = b->rec + po;
            a.N = N;
            a.stride = b->Ntot;
            a.P = P;
            a.gtab = b->gtab + kGTab32Bytes * mo;
            a.m = b->modes + 3 * mo;
            a.Fn = b->Fn + po;
            a.F = b->F + po;
            a.st = offset_state(b->rest, po);
            a.integrate = k;
            a.dt = p.dt;
            a.K_part = b->K_part + k_off;
            a.F_user = a.Fn_user = a.Ff_user = nullptr;
            EnergyArgs &e = en[k][r];
            e.U_part = b->U_part + u_off;
            e.nU = 4 * (int)nbn;
            e.K_part = b->K_part + k_off;
            e.nK = (int)nbf;
            e.Ufar = b->Ufar + mo;
            e.nUfar = P;
            e.Ufar0 = h.Ufar0;
            e.Uself = h.Uself;
            e.out = b->energy + 5 * (size_t)r;
            e.ctr = b->ctr + r;
            e.advance_step = k;
        }
        ss[r] = SysStateArgs{offset_state(b->rest, po), b->q_user + po, b->m_user + po, N, (uint32_t)po, h.box};
        const uint32_t cnt[6] = {bin_batch_blocks(N), sample_batch_blocks(P), nbn, rho_batch_blocks(G, P),
                                 rho_final_batch_blocks(P), nbf};
        for (int j = 0; j < 6; ++j) {
            items[(size_t)j * (R + 1) + r] = it[j];
            it[j] += cnt[j];
        }
        part_off += (size_t)G * 8 * P;
        u_off += 4 * (size_t)nbn;
        k_off += nbf;
    }
    for (int j = 0; j < 6; ++j) {
        items[(size_t)j * (R + 1) + R] = it[j];
        b->nb[j] = it[j];
    }
    BCK(upload(b, &b->d_bin[0], bin[0]), "upload arguments");
    BCK(upload(b, &b->d_bin[1], bin[1]), "upload arguments");
    BCK(upload(b, &b->d_far[0], far[0]), "upload arguments");
    BCK(upload(b, &b->d_far[1], far[1]), "upload arguments");
    BCK(upload(b, &b->d_far_user, far[0]), "upload arguments");
    BCK(upload(b, &b->d_energy[0], en[0]), "upload arguments");
    BCK(upload(b, &b->d_energy[1], en[1]), "upload arguments");
    BCK(upload(b, &b->d_sample, sa), "upload arguments");
    BCK(upload(b, &b->d_near, na), "upload arguments");
    BCK(upload(b, &b->d_geom, geom), "upload arguments");
    BCK(upload(b, &b->d_rho, ra), "upload arguments");
    BCK(upload(b, &b->d_chunk, b->rho_chunk), "upload arguments");
    BCK(upload(b, &b->d_rf, rf), "upload arguments");
    BCK(upload(b, &b->d_state, ss), "upload arguments");
    BCK(upload(b, &b->d_items, items), "upload arguments");
    b->h_far = far[0];
    return RBSOG_OK;
}

const uint32_t *items_of(const rbsog_batch *b, int j) { return b->d_items + (size_t)j * (b->R + 1); }

// One force evaluation (set 0) or one step (set 1) of every system.  With ev (11 events)
// the kernel groups bin, scan, sort, gather, sample, near, rho, rho_final, far, energy
// are bracketed by ev[g] and ev[g + 1].
int enqueue(rbsog_batch *b, cudaStream_t st, int set, const FarArgs *far, cudaEvent_t *ev = nullptr) {
    const int R = b->R;
    auto mark = [&](int g) {
        if (ev) cudaEventRecord(ev[g], st);
    };
    mark(0);
    launch_bin_batch(b->d_bin[set], items_of(b, kItBin), R, b->nb[kItBin], st);
    mark(1);
    launch_scan(b->count, b->tile_sums, b->cell_start, b->Ctot, b->Ntot, st);
    mark(2);
    launch_scatter_sort(b->cell, b->slot, b->cell_start, b->work.id, b->Ntot, b->Ctot, b->keys, b->perm_src,
                        b->ctr + R, st);
    mark(3);
    GatherArgs g{};
    g.in = b->work; g.out = b->rest; g.perm_src = b->perm_src; g.s = b->s; g.rec = b->rec; g.N = b->Ntot;
    launch_gather(RBSOG_FP32, g, st);
    mark(4);
    launch_sample_batch(b->d_sample, items_of(b, kItSample), R, b->nb[kItSample], st);
    mark(5);
    launch_near_batch(b->d_near, b->d_geom, items_of(b, kItNear), R, b->nb[kItNear], st);
    mark(6);
    launch_rho_batch(b->d_rho, b->d_chunk, items_of(b, kItRho), R, b->nb[kItRho], st);
    mark(7);
    launch_rho_final_batch(b->d_rf, items_of(b, kItRhoFinal), R, b->nb[kItRhoFinal], st);
    mark(8);
    launch_far_batch(far ? far : b->d_far[set], items_of(b, kItFar), R, b->nb[kItFar], st);
    mark(9);
    launch_energy_batch(b->d_energy[set], R, st);
    mark(10);
    BCK(cudaGetLastError(), "kernel launch");
    return RBSOG_OK;
}

struct EventSet {
    cudaEvent_t ev[11] = {};
    bool ok = true;
    EventSet() {
        for (auto &e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    }
    ~EventSet() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    float ms(int g0, int g1) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[g0], ev[g1]);
        return t;
    }
};

// Apply a near tile target and a structure-factor target to every system.
int apply_shapes(rbsog_batch *b, double near_target, int rho_target) {
    b->near_target = near_target;
    for (int r = 0; r < b->R; ++r) b->rho_chunk[r] = chunk_for(b->sys[r].N, rho_target);
    if (int c = ensure_partials(b)) return c;
    if (int c = build_args(b)) return c;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return RBSOG_OK;
}

}  // namespace

extern "C" {

int rbsog_batch_init(const rbsog_params *params, int32_t R, const int64_t *N, const double *q_host,
                     const double *m_host, rbsog_batch **out) {
    if (!out) return bfail(nullptr, RBSOG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !N || !q_host || !m_host) return bfail(nullptr, RBSOG_EINVAL, "params, N, q or m is NULL");
    if (R < 1 || R > (1 << 20)) return bfail(nullptr, RBSOG_EINVAL, "R must be in [1, 2^20]");
    std::vector<HostSystem> sys(R);
    std::vector<uint32_t> p_off(R + 1, 0), c_off(R + 1, 0), m_off(R + 1, 0);
    long long nt = 0, ct = 0, pt = 0;
    for (int r = 0; r < R; ++r) {
        if (params[r].precision != RBSOG_FP32)
            return bfail(nullptr, RBSOG_EUNSUPPORTED, "batched systems run the FP32 path only");
        if (params[r].device != params[0].device)
            return bfail(nullptr, RBSOG_EINVAL, "every system of a batch uses the same device");
        std::string err;
        const int code = setup_system(params[r], N[r], q_host + nt, m_host + nt, &sys[r], &err);
        if (code != RBSOG_OK) return bfail(nullptr, code, "system " + std::to_string(r) + ": " + err);
        nt += N[r];
        ct += sys[r].box.ncell;
        pt += params[r].P;
        if (nt >= 0x7fffffffLL || ct > (1LL << 28) || pt > (1LL << 26))
            return bfail(nullptr, RBSOG_EINVAL, "batch too large (particles, cells or modes)");
        p_off[r + 1] = (uint32_t)nt;
        c_off[r + 1] = (uint32_t)ct;
        m_off[r + 1] = (uint32_t)pt;
    }
    if (cudaSetDevice(params[0].device) != cudaSuccess) {
        cudaGetLastError();
        return bfail(nullptr, RBSOG_ECUDA, "cudaSetDevice failed (no usable CUDA device)");
    }
    rbsog_batch *b = new rbsog_batch();
    b->R = R;
    b->Ntot = (uint32_t)nt;
    b->Ctot = (int)ct;
    b->Ptot = (int)pt;
    b->device = params[0].device;
    b->sys = std::move(sys);
    b->p_off = p_off;
    b->c_off = c_off;
    b->m_off = m_off;
    b->rho_chunk.resize(R);
    for (int r = 0; r < R; ++r) b->rho_chunk[r] = chunk_for(b->sys[r].N, 512);
    auto bail = [&](int code, const std::string &msg) {
        g_batch_init_error = msg.empty() ? b->err : msg;
        rbsog_batch_free(b);
        return code;
    };
    const size_t n = b->Ntot, n3 = 3 * n;
    State *sts[2] = {&b->rest, &b->work};
    for (State *s : sts)
        if (balloc(b, &s->rx, n) || balloc(b, &s->ry, n) || balloc(b, &s->rz, n) || balloc(b, &s->vx, n) ||
            balloc(b, &s->vy, n) || balloc(b, &s->vz, n) || balloc(b, &s->invm, n) || balloc(b, &s->q, n) ||
            balloc(b, &s->id, n))
            return bail(RBSOG_ENOMEM, "device allocation failed (state)");
    const size_t ntiles = ((size_t)b->Ctot + kScanTile - 1) / kScanTile;
    const size_t P = (size_t)b->Ptot;
    if (balloc(b, &b->q_user, n) || balloc(b, &b->m_user, n) || balloc(b, &b->stage_a, n3) ||
        balloc(b, &b->stage_b, n3) || balloc(b, &b->F, n3) || balloc(b, &b->Fn, n3) || balloc(b, &b->s, n3) ||
        balloc(b, &b->rec, n) || balloc(b, &b->cell, n) || balloc(b, &b->slot, n) ||
        balloc(b, &b->count, (size_t)b->Ctot) || balloc(b, &b->tile_sums, ntiles) ||
        balloc(b, &b->cell_start, (size_t)b->Ctot + 1) || balloc(b, &b->perm_src, n) || balloc(b, &b->keys, n) ||
        balloc(b, &b->modes, 3 * P) || balloc(b, &b->inject_m, 3 * P) || balloc(b, &b->coef, P) ||
        balloc(b, &b->rho, P) || balloc(b, &b->gtab, kGTab32Bytes * P) || balloc(b, &b->Ufar, P) ||
        balloc(b, &b->energy, 5 * (size_t)R + 3) || balloc(b, &b->ctr, (size_t)R + 1))
        return bail(RBSOG_ENOMEM, "device allocation failed");
    // sampling tables, concatenated system by system
    std::vector<double> mp, axp;
    std::vector<int> ma, off, nmax, axa;
    for (const HostSystem &h : b->sys) {
        mp.insert(mp.end(), h.mix_prob.begin(), h.mix_prob.end());
        ma.insert(ma.end(), h.mix_alias.begin(), h.mix_alias.end());
        off.insert(off.end(), h.ax_off.begin(), h.ax_off.end());
        nmax.insert(nmax.end(), h.ax_nmax.begin(), h.ax_nmax.end());
        axp.insert(axp.end(), h.ax_prob.begin(), h.ax_prob.end());
        axa.insert(axa.end(), h.ax_alias.begin(), h.ax_alias.end());
    }
    std::vector<double> qv(q_host, q_host + n), mv(m_host, m_host + n);
    if (upload(b, &b->mix_prob, mp) || upload(b, &b->mix_alias, ma) || upload(b, &b->ax_off, off) ||
        upload(b, &b->ax_nmax, nmax) || upload(b, &b->ax_prob, axp) || upload(b, &b->ax_alias, axa) ||
        cudaMemcpy(b->q_user, qv.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->m_user, mv.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->count, 0, sizeof(uint32_t) * (size_t)b->Ctot) != cudaSuccess ||
        cudaMemset(b->ctr, 0, sizeof(DevCounters) * ((size_t)R + 1)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(RBSOG_ECUDA, "device initialisation failed");
    for (int r = 0; r < R; ++r) {
        std::string err;
        const int code = system_S(&b->sys[r], &err);
        if (code != RBSOG_OK) return bail(code, err);
    }
    if (ensure_partials(b) != RBSOG_OK) return bail(RBSOG_ENOMEM, "device allocation failed (partials)");
    const int code = build_args(b);
    if (code != RBSOG_OK) return bail(code, "");
    // a valid (zero) state so every call is defined before rbsog_batch_set_state
    if (cudaMemset(b->stage_a, 0, n3 * sizeof(double)) != cudaSuccess) return bail(RBSOG_ECUDA, "device initialisation failed");
    launch_set_state_batch(b->d_state, items_of(b, kItBin), R, b->nb[kItBin], b->stage_a, nullptr, b->ctr, R + 1, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(RBSOG_ECUDA, "device initialisation failed");
    *out = b;
    return RBSOG_OK;
}

int rbsog_batch_set_state(rbsog_batch *b, const double *r, const double *v, void *stream) {
    if (!b || !r) return bfail(b, RBSOG_EINVAL, "batch or r is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)b->Ntot * sizeof(double);
    const double *rd = r, *vd = v;
    if (!dev_ptr(r)) {
        BCK(cudaMemcpyAsync(b->stage_a, r, bytes, cudaMemcpyDefault, st), "copy r");
        rd = b->stage_a;
    }
    if (v && !dev_ptr(v)) {
        BCK(cudaMemcpyAsync(b->stage_b, v, bytes, cudaMemcpyDefault, st), "copy v");
        vd = b->stage_b;
    }
    launch_set_state_batch(b->d_state, items_of(b, kItBin), b->R, b->nb[kItBin], rd, vd, b->ctr, b->R + 1, st);
    BCK(cudaGetLastError(), "set_state");
    b->force_valid = false;
    return RBSOG_OK;
}

int rbsog_batch_get_state(rbsog_batch *b, double *r, double *v, uint64_t *step, void *stream) {
    if (!b) return bfail(b, RBSOG_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)b->Ntot * sizeof(double);
    double *rd = r && dev_ptr(r) ? r : (r ? b->stage_a : nullptr);
    double *vd = v && dev_ptr(v) ? v : (v ? b->stage_b : nullptr);
    launch_get_state_batch(b->d_state, items_of(b, kItBin), b->R, b->nb[kItBin], rd, vd, st);
    BCK(cudaGetLastError(), "get_state");
    if (r && rd != r) BCK(cudaMemcpyAsync(r, rd, bytes, cudaMemcpyDefault, st), "copy r out");
    if (v && vd != v) BCK(cudaMemcpyAsync(v, vd, bytes, cudaMemcpyDefault, st), "copy v out");
    DevCounters hc;
    BCK(cudaMemcpyAsync(&hc, b->ctr, sizeof hc, cudaMemcpyDeviceToHost, st), "read counters");
    BCK(cudaStreamSynchronize(st), "synchronize");
    if (step) *step = hc.step;
    return check_errors(b);
}

int rbsog_batch_forces(rbsog_batch *b, double *F, rbsog_energy *e, void *stream) {
    if (!b) return bfail(b, RBSOG_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const FarArgs *far = nullptr;
    double *Fd = nullptr;
    if (F) {
        Fd = dev_ptr(F) ? F : b->stage_a;
        // caller-order outputs: system r's forces at 3 p_off[r] of F
        std::vector<FarArgs> fa = b->h_far;
        for (int r = 0; r < b->R; ++r) fa[r].F_user = Fd + 3 * (size_t)b->p_off[r];
        BCK(cudaMemcpyAsync(b->d_far_user, fa.data(), fa.size() * sizeof(FarArgs), cudaMemcpyHostToDevice, st),
            "upload arguments");
        BCK(cudaStreamSynchronize(st), "synchronize");
        far = b->d_far_user;
    }
    int code = enqueue(b, st, 0, far);
    if (code) return code;
    b->force_valid = true;
    if (F && Fd != F)
        BCK(cudaMemcpyAsync(F, Fd, 3 * (size_t)b->Ntot * sizeof(double), cudaMemcpyDefault, st), "copy forces out");
    if (e) return read_energies(b, e, st);
    BCK(cudaStreamSynchronize(st), "synchronize");
    return check_errors(b);
}

int rbsog_batch_step(rbsog_batch *b, int32_t nsteps, rbsog_energy *e, void *stream) {
    if (!b) return bfail(b, RBSOG_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(b, RBSOG_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->force_valid && nsteps > 0) {
        int code = enqueue(b, st, 0, nullptr);
        if (code) return code;
        b->force_valid = true;
    }
    if (nsteps > 0 && !b->graph) {
        cudaGraph_t g;
        BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int code = enqueue(b, b->cap_stream, 1, nullptr);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (code) return code;
        BCK(e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e3, "graph instantiate");
    }
    for (int i = 0; i < nsteps; ++i) BCK(cudaGraphLaunch(b->graph, st), "graph launch");
    if (e) return read_energies(b, e, st);
    return RBSOG_OK;
}

int rbsog_batch_set_ksample(rbsog_batch *b, const int32_t *m_host) {
    if (!b || !m_host) return bfail(b, RBSOG_EINVAL, "batch or m is NULL");
    for (int l = 0; l < b->Ptot; ++l)
        if (m_host[3 * l] == 0 && m_host[3 * l + 1] == 0 && m_host[3 * l + 2] == 0)
            return bfail(b, RBSOG_EINVAL, "mode (0,0,0) is not in the sampled support");
    BCK(cudaDeviceSynchronize(), "synchronize");
    BCK(cudaMemcpy(b->inject_m, m_host, 3 * sizeof(int32_t) * (size_t)b->Ptot, cudaMemcpyHostToDevice), "copy modes");
    int one = 1;
    for (int r = 0; r < b->R; ++r)
        BCK(cudaMemcpy(&b->ctr[r].inject, &one, sizeof(int), cudaMemcpyHostToDevice), "set inject flag");
    return RBSOG_OK;
}

int rbsog_batch_get_ksample(rbsog_batch *b, int32_t *m_host, double *coef_host) {
    if (!b) return bfail(b, RBSOG_EINVAL, "batch is NULL");
    BCK(cudaDeviceSynchronize(), "synchronize");
    if (m_host)
        BCK(cudaMemcpy(m_host, b->modes, 3 * sizeof(int32_t) * (size_t)b->Ptot, cudaMemcpyDeviceToHost), "copy modes");
    if (coef_host)
        BCK(cudaMemcpy(coef_host, b->coef, sizeof(double) * (size_t)b->Ptot, cudaMemcpyDeviceToHost), "copy coef");
    return check_errors(b);
}

int rbsog_batch_layout(const rbsog_batch *b, int64_t *p_off, int64_t *m_off, int32_t *rho_chunk) {
    if (!b) return bfail(nullptr, RBSOG_EINVAL, "batch is NULL");
    for (int r = 0; r <= b->R; ++r) {
        if (p_off) p_off[r] = b->p_off[r];
        if (m_off) m_off[r] = b->m_off[r];
        if (rho_chunk && r < b->R) rho_chunk[r] = b->rho_chunk[r];
    }
    return RBSOG_OK;
}

int rbsog_batch_set_rho_chunk(rbsog_batch *b, const int32_t *rho_chunk) {
    if (!b || !rho_chunk) return bfail(b, RBSOG_EINVAL, "batch or rho_chunk is NULL");
    for (int r = 0; r < b->R; ++r)
        if (rho_chunk[r] < 64) return bfail(b, RBSOG_EINVAL, "rho_chunk must be >= 64");
    BCK(cudaDeviceSynchronize(), "synchronize");
    for (int r = 0; r < b->R; ++r) b->rho_chunk[r] = rho_chunk[r];
    if (int c = ensure_partials(b)) return c;
    int code = build_args(b);
    if (code != RBSOG_OK) return code;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return RBSOG_OK;
}

int rbsog_batch_profile(rbsog_batch *b, int32_t nsteps, double *ms, void *stream) {
    if (!b || !ms || nsteps < 1) return bfail(b, RBSOG_EINVAL, "batch or ms is NULL, or nsteps < 1");
    cudaStream_t st = (cudaStream_t)stream;
    EventSet es;
    if (!es.ok) return bfail(b, RBSOG_ECUDA, "event creation failed");
    for (int g = 0; g < RBSOG_NPROF; ++g) ms[g] = 0.0;
    if (!b->force_valid) {
        if (int c = enqueue(b, st, 0, nullptr)) return c;
        b->force_valid = true;
    }
    for (int i = 0; i < nsteps; ++i) {
        if (int c = enqueue(b, st, 1, nullptr, es.ev)) return c;
        BCK(cudaStreamSynchronize(st), "synchronize");
        for (int g = 0; g < RBSOG_NPROF; ++g) ms[g] += es.ms(g, g + 1);
    }
    return check_errors(b);
}

int rbsog_batch_set_shapes(rbsog_batch *b, double near_target, int32_t rho_target) {
    if (!b) return bfail(b, RBSOG_EINVAL, "batch is NULL");
    if (!(near_target >= 8.0 && near_target <= 4096.0) || rho_target < 64)
        return bfail(b, RBSOG_EINVAL, "need 8 <= near_target <= 4096 and rho_target >= 64");
    BCK(cudaDeviceSynchronize(), "synchronize");
    return apply_shapes(b, near_target, rho_target);
}

int rbsog_batch_tune(rbsog_batch *b, int32_t reps, double *near_target, int32_t *rho_target, void *stream) {
    if (!b || reps < 1) return bfail(b, RBSOG_EINVAL, "batch is NULL or reps < 1");
    cudaStream_t st = (cudaStream_t)stream;
    EventSet es;
    if (!es.ok) return bfail(b, RBSOG_EINVAL, "event creation failed");
    // the counters are restored afterwards, so the tuning evaluations leave no trace in
    // the draws; the next step re-evaluates the forces
    std::vector<DevCounters> saved(b->R + 1);
    BCK(cudaStreamSynchronize(st), "synchronize");
    BCK(cudaMemcpy(saved.data(), b->ctr, saved.size() * sizeof(DevCounters), cudaMemcpyDeviceToHost), "save counters");
    const double near_c[] = {48.0, 80.0, 110.0, 160.0};
    const int rho_c[] = {256, 512, 1024, 2048};
    double best_near = b->near_target, best_near_ms = 1e30;
    int best_rho = 512;
    double best_rho_ms = 1e30;
    int code = RBSOG_OK;
    for (int ci = 0; ci < 4 && code == RBSOG_OK; ++ci) {
        // near field and structure factor are independent: tune both from one sweep
        if ((code = apply_shapes(b, near_c[ci], rho_c[ci])) != RBSOG_OK) break;
        std::vector<double> tn, tr;
        for (int i = 0; i <= reps && code == RBSOG_OK; ++i) {
            if ((code = enqueue(b, st, 0, nullptr, es.ev)) != RBSOG_OK) break;
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                code = bcuda_fail(b, cudaGetLastError(), "synchronize");
                break;
            }
            if (i == 0) continue;   // first run after a shape change: warm-up
            tn.push_back(es.ms(5, 6));
            tr.push_back(es.ms(6, 8));
        }
        if (code != RBSOG_OK) break;
        std::sort(tn.begin(), tn.end());
        std::sort(tr.begin(), tr.end());
        if (tn[tn.size() / 2] < best_near_ms) { best_near_ms = tn[tn.size() / 2]; best_near = near_c[ci]; }
        if (tr[tr.size() / 2] < best_rho_ms) { best_rho_ms = tr[tr.size() / 2]; best_rho = rho_c[ci]; }
    }
    if (code == RBSOG_OK) code = apply_shapes(b, best_near, best_rho);
    cudaError_t e = cudaMemcpy(b->ctr, saved.data(), saved.size() * sizeof(DevCounters), cudaMemcpyHostToDevice);
    b->force_valid = false;
    if (code != RBSOG_OK) return code;
    BCK(e, "restore counters");
    if (near_target) *near_target = best_near;
    if (rho_target) *rho_target = best_rho;
    return check_errors(b);
}

const char *rbsog_batch_last_error(const rbsog_batch *b) { return b ? b->err.c_str() : g_batch_init_error.c_str(); }

void rbsog_batch_free(rbsog_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
}

}  // extern "C"
