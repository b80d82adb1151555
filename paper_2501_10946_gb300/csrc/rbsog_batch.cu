// Resident-set engine (the layout is described in engine.h) and the batch ABI: a fixed
// set of systems advanced together, every kernel of the step one launch over all of
// them, replayed from one CUDA graph per step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

using namespace rbsog;

namespace {

enum { kItBin = 0, kItSample, kItNear, kItRho, kItRhoFinal, kItFar };

std::string g_batch_init_error;

#define BCK(call, where)                                                \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return engine_cuda_fail(b, e_, where);   \
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

// Replace a grow-only buffer by a larger one (the device is idle when this is called).
template <typename T>
cudaError_t regrow(rbsog_batch *b, T **ptr, size_t *cap, size_t need) {
    if (need <= *cap && *ptr) return cudaSuccess;
    if (*ptr) {
        auto it = std::find(b->allocs.begin(), b->allocs.end(), (void *)*ptr);
        if (it != b->allocs.end()) b->allocs.erase(it);
        cudaFree(*ptr);
        *ptr = nullptr;
    }
    const size_t n = std::max<size_t>(need, 1) + need / 4;   // headroom against frequent regrowth
    cudaError_t e = balloc(b, ptr, n);
    if (e == cudaSuccess) *cap = n;
    return e;
}

template <typename T>
cudaError_t upload(T *dst, const std::vector<T> &src) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
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

struct SysShape {
    NearBatchGeom ng;          // near-field bricks (or the per-particle path)
    uint32_t near_blocks;
    int G;
};

// Threads of one near-field block: a brick of the batched kernel or of the persistent step.
int near_threads(const rbsog_batch *) { return kNearBrickThreads; }

SysShape shape_of(const HostSystem &h, double near_target, int chunk, int nthreads) {
    SysShape s{};
    s.near_blocks = near_bricks(h.box, h.N, near_target, &s.ng);
    if (!s.ng.tiled) s.near_blocks = (h.N + (uint32_t)nthreads - 1) / (uint32_t)nthreads;
    s.G = (int)((h.N + (uint32_t)chunk - 1) / (uint32_t)chunk);
    return s;
}

const uint32_t *items_of(const rbsog_batch *b, int j) { return b->d_items + (size_t)j * (b->capR + 1); }

// Per-system argument arrays and block prefixes for the current membership and shapes.
int build_args(rbsog_batch *b) {
    const int R = b->R;
    std::vector<BinArgs> bin[2];
    std::vector<FarArgs> far[2];
    std::vector<EnergyArgs> en[2];
    for (int k = 0; k < 2; ++k) {
        bin[k].resize(R);
        far[k].resize(R);
        en[k].resize(R);
    }
    std::vector<SampleArgs> sa(R);
    std::vector<NearArgs> na(R);
    std::vector<NearF> nfs(R);
    std::vector<NearBatchGeom> geom(R);
    std::vector<RhoArgs> ra(R);
    std::vector<RhoFinalArgs> rf(R);
    std::vector<SysStateArgs> ss(R);
    std::vector<uint32_t> items(6 * (size_t)(b->capR + 1), 0u);
    size_t part_off = 0, u_off = 0, k_off = 0, ax_base = 0, mix_base = 0;
    uint32_t it[6] = {0, 0, 0, 0, 0, 0};
    for (int r = 0; r < R; ++r) {
        const HostSystem &h = b->sys[r];
        const rbsog_params &p = h.p;
        const size_t po = b->p_off[r], mo = b->m_off[r];
        const uint32_t N = h.N;
        const int P = p.P;
        const int mode = p.ensemble == RBSOG_LANGEVIN ? 2 : 1;
        DevCounters *ctr = b->ctr + r;
        const SysShape sh = shape_of(h, b->near_target, b->rho_chunk[r], near_threads(b));
        for (int k = 0; k < 2; ++k) {
            BinArgs &a = bin[k][r];
            a.in = offset_state(b->rest, po);
            a.out = offset_state(b->work, po);
            a.F = b->F + po;
            a.integrate = k ? mode : 0;
            a.dt = p.dt;
            a.c1 = std::exp(-p.langevin_gamma * p.dt);
            a.kT = h.kT;
            a.okT = (1.0 - a.c1 * a.c1) * a.kT;
            set_bin_floats(a);
            a.seed = p.seed;
            a.ctr = ctr;
            a.N = N;
            a.stride = b->capN;
            a.cell_base = b->c_off[r];
            a.box = h.box;
            a.rec_w = b->rec_w + po;
            a.rec_id = b->rec_id + po;
            a.cell = b->cell + po;
            a.slot = b->slot + po;
            a.count = b->count;
        }
        {
            SampleArgs &a = sa[r];
            const int mt = (int)h.mix_prob.size();   // mixture components
            a.tab = SamplerTables{mt, b->mix_thr + mix_base, b->mix_alias + mix_base, b->ax_off + 3 * mix_base,
                                  b->ax_nmax + 3 * mix_base, b->ax_thr + ax_base, b->ax_alias + ax_base};
            mix_base += (size_t)mt;
            ax_base += h.ax_prob.size();
            a.P = P;
            a.seed = p.seed;
            for (int d = 0; d < 3; ++d) a.tpl[d] = h.box.tpl[d];
            a.A = h.kT * h.V;
            a.Q2 = h.Q2;
            a.y = h.y;
            fill_signed_fhat(h.y, h.sA, h.sb, &a);
            a.S = h.S;
            a.V = h.V;
            a.measure = h.p.sampling;
            a.Q2a = h.p.sampling == RBSOG_SAMPLING_DEBYE ? (4.0 * 3.14159265358979323846) * h.Q2 : h.Q2;
            sample_set_prefilter(&a);
            a.ctr = ctr;
            a.inject_m = b->inject_m + 3 * mo;
            a.m_out = b->modes + 3 * mo;
            a.coef_out = b->coef + mo;
        }
        // near field: global record and force indices, this system's cell range
        geom[r] = sh.ng;
        if (!sh.ng.tiled) geom[r].W = (int)po;
        nfs[r] = near_f32_consts(h.nconsts);
        {
            NearArgs &a = na[r];
            a.nc = h.nconsts;
            a.rec = b->rec;
            a.cell_start = b->cell_start + b->c_off[r];
            a.box = h.box;
            a.N = N;
            a.stride = b->capN;
            a.Fn = b->Fn;
            a.U_part = b->U_part + u_off;
            a.ctr = ctr;
        }
        {
            RhoArgs &a = ra[r];
            a.rec = b->rec_id + po;    // id order: no cell list needed
            a.N = N;
            a.m = b->modes + 3 * mo;
            a.P = P;
            a.partial = b->partial + part_off;
            a.G = sh.G;
        }
        {
            RhoFinalArgs &a = rf[r];
            a.partial = b->partial + part_off;
            a.G = sh.G;
            a.P = P;
            a.m = b->modes + 3 * mo;
            a.coef = b->coef + mo;
            for (int d = 0; d < 3; ++d) a.tpl[d] = h.box.tpl[d];
            a.rho = b->rho + mo;
            a.gtab = b->gtab + kGTab32Bytes * mo;
            a.Ufar = b->Ufar + mo;
            a.ctr = ctr;
        }
        const uint32_t nbf = far_batch_blocks(N);
        for (int k = 0; k < 2; ++k) {
            FarArgs &a = far[k][r];
            a.rec = b->rec + po;
            a.N = N;
            a.stride = b->capN;
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
            a.ctr = ctr;
            EnergyArgs &e = en[k][r];
            e.U_part = b->U_part + u_off;
            e.nU = near_threads(b) / 32 * (int)sh.near_blocks;
            e.K_part = b->K_part + k_off;
            e.nK = (int)nbf;
            e.Ufar = b->Ufar + mo;
            e.nUfar = P;
            e.Ufar0 = h.Ufar0;
            e.Uself = h.Uself;
            e.out = b->energy + 5 * (size_t)r;
            e.ctr = ctr;
        }
        ss[r] = SysStateArgs{offset_state(b->rest, po), nullptr, nullptr, N, (uint32_t)po, h.box};
        const uint32_t cnt[6] = {bin_batch_blocks(N), sample_batch_blocks(P), sh.near_blocks,
                                 rho_batch_blocks(sh.G, P), rho_final_batch_blocks(P), nbf};
        for (int j = 0; j < 6; ++j) {
            items[(size_t)j * (b->capR + 1) + r] = it[j];
            it[j] += cnt[j];
        }
        part_off += (size_t)sh.G * 8 * P;
        u_off += (size_t)(near_threads(b) / 32) * sh.near_blocks;
        k_off += nbf;
    }
    b->h_items.assign(R + 1, 0u);
    for (int j = 0; j < 6; ++j) {
        items[(size_t)j * (b->capR + 1) + R] = it[j];
        b->nb[j] = it[j];
    }
    for (int r = 0; r <= R; ++r) b->h_items[r] = items[r];
    BCK(upload(b->d_bin[0], bin[0]), "upload arguments");
    BCK(upload(b->d_bin[1], bin[1]), "upload arguments");
    BCK(upload(b->d_far[0], far[0]), "upload arguments");
    BCK(upload(b->d_far[1], far[1]), "upload arguments");
    BCK(upload(b->d_far_user, far[0]), "upload arguments");
    BCK(upload(b->d_energy[0], en[0]), "upload arguments");
    BCK(upload(b->d_energy[1], en[1]), "upload arguments");
    BCK(upload(b->d_sample, sa), "upload arguments");
    BCK(upload(b->d_near, na), "upload arguments");
    BCK(upload(b->d_nearf, nfs), "upload arguments");
    BCK(upload(b->d_geom, geom), "upload arguments");
    BCK(upload(b->d_rho, ra), "upload arguments");
    BCK(upload(b->d_chunk, std::vector<int>(b->rho_chunk.begin(), b->rho_chunk.begin() + R)), "upload arguments");
    BCK(upload(b->d_rf, rf), "upload arguments");
    BCK(upload(b->d_state, ss), "upload arguments");
    b->h_state = ss;
    BCK(upload(b->d_items, items), "upload arguments");
    BCK(upload(b->d_coff, std::vector<uint32_t>(b->c_off.begin(), b->c_off.end())), "upload arguments");
    b->h_far = far[0];
    return RBSOG_OK;
}

// Switch between the graph of batched kernels and the persistent step; the arguments are
// rebuilt for the form's near-field block size (energy partials written before the switch
// are no longer readable).
int set_form(rbsog_batch *b, bool persistent) {
    if (b->persistent == persistent) return RBSOG_OK;
    BCK(cudaDeviceSynchronize(), "synchronize");
    b->persistent = persistent;
    b->dirty = true;
    b->energies_stale = true;
    return engine_commit(b);
}

// Per-kernel timing (profiling, tuning) runs the graph form's kernels one by one.
struct GraphFormScope {
    rbsog_batch *b;
    bool was;
    int code = RBSOG_OK;
    explicit GraphFormScope(rbsog_batch *b_) : b(b_), was(b_->persistent) {
        if (was) code = set_form(b, false);
    }
    ~GraphFormScope() {
        if (was) set_form(b, true);
    }
};

// A persistent step whose barrier wait gave up: report it and clear the barrier state
// (the state of that pass is not valid).
int check_barrier(rbsog_batch *b) {
    GridBar h{};
    BCK(cudaMemcpy(&h, b->bar, sizeof h, cudaMemcpyDeviceToHost), "read barrier state");
    if (h.status) {
        // the pass stopped between phases: barrier state, work counters and the cell counts
        // (incremented by binning, cleared by the scan) start again from zero
        BCK(cudaMemset(b->bar, 0, sizeof(GridBar)), "reset barrier state");
        if (b->Ctot) BCK(cudaMemset(b->count, 0, sizeof(uint32_t) * (size_t)b->Ctot), "reset cell counts");
        return engine_fail(b, RBSOG_ETIMEOUT, "a grid-barrier wait of the persistent step exceeded its limit");
    }
    return RBSOG_OK;
}

int check_all(rbsog_batch *b) {
    if (int code = check_barrier(b)) return code;
    std::vector<DevCounters> c;
    if (int code = engine_counters(b, &c)) return code;
    for (int r = 0; r < b->R; ++r)
        if (int code = engine_status(b, c, r)) return code;
    return RBSOG_OK;
}

int read_energies(rbsog_batch *b, rbsog_energy *e, cudaStream_t st) {
    if (b->energies_stale)
        return engine_fail(b, RBSOG_EINVAL, "the form changed since the last force evaluation: no energies to read");
    if (int code = check_barrier(b)) return code;
    if (int code = engine_reduce_energies(b, st)) return code;
    std::vector<double> h(5 * (size_t)b->R);
    if (b->R) BCK(cudaMemcpyAsync(h.data(), b->energy, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
                  "read energy");
    BCK(cudaStreamSynchronize(st), "synchronize");
    std::vector<DevCounters> c;
    if (int code = engine_counters(b, &c)) return code;
    for (int r = 0; r < b->R; ++r) {
        const double *x = &h[5 * (size_t)r];
        e[r].U_near = x[0]; e[r].U_far = x[1]; e[r].U_self = x[2]; e[r].kinetic = x[3]; e[r].total = x[4];
        e[r].step = c[r].step;
    }
    for (int r = 0; r < b->R; ++r)
        if (int code = engine_status(b, c, r)) return code;
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
    b->rho_target = rho_target;
    for (int r = 0; r < b->R; ++r) b->rho_chunk[r] = chunk_for(b->sys[r].N, rho_target);
    b->dirty = true;
    return engine_commit(b);
}

// Items of the bin kernel restricted to systems first .. first+count-1 (relative block
// numbers), uploaded to d_sub_items.
int sub_items(rbsog_batch *b, int first, int count, uint32_t *nblocks, cudaStream_t st) {
    std::vector<uint32_t> it(count + 1);
    for (int k = 0; k <= count; ++k) it[k] = b->h_items[first + k] - b->h_items[first];
    *nblocks = it[count];
    BCK(cudaMemcpyAsync(b->d_sub_items, it.data(), it.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st),
        "upload items");
    // the host vector dies at return: wait for the copy
    BCK(cudaStreamSynchronize(st), "synchronize");
    return RBSOG_OK;
}

}  // namespace

namespace rbsog {

int engine_fail(rbsog_batch *b, int code, const std::string &msg) {
    if (b) b->err = msg;
    else g_batch_init_error = msg;
    return code;
}

int engine_cuda_fail(rbsog_batch *b, cudaError_t e, const char *where) {
    return engine_fail(b, e == cudaErrorMemoryAllocation ? RBSOG_ENOMEM : RBSOG_ECUDA,
                       std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}

int engine_alloc(rbsog_batch *b, const EngineCaps &caps, int device) {
    if (caps.particles < 2 || caps.particles >= 0x7fffffffu || caps.cells < 1 || caps.cells > (1 << 28) ||
        caps.modes < 1 || caps.modes > (1 << 26) || caps.systems < 1 || caps.systems > (1 << 20))
        return engine_fail(b, RBSOG_EINVAL, "engine capacities out of range");
    b->capN = caps.particles;
    b->capC = caps.cells;
    b->capP = caps.modes;
    b->capR = caps.systems;
    b->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return engine_fail(b, RBSOG_ECUDA, "cudaSetDevice failed (no usable CUDA device)");
    }
    const size_t n = b->capN, n3 = 3 * n, C = (size_t)b->capC, P = (size_t)b->capP, R = (size_t)b->capR;
    State *sts[2] = {&b->rest, &b->work};
    for (State *s : sts)
        if (balloc(b, &s->rx, n) || balloc(b, &s->ry, n) || balloc(b, &s->rz, n) || balloc(b, &s->vx, n) ||
            balloc(b, &s->vy, n) || balloc(b, &s->vz, n) || balloc(b, &s->invm, n) || balloc(b, &s->q, n) ||
            balloc(b, &s->id, n))
            return engine_fail(b, RBSOG_ENOMEM, "device allocation failed (state)");
    const size_t ntiles = (C + kScanTile - 1) / kScanTile;
    if (balloc(b, &b->stage_a, n3) || balloc(b, &b->stage_b, n3) || balloc(b, &b->stage_qm, 2 * n) ||
        balloc(b, &b->d_state_sub, R) || balloc(b, &b->F, n3) || balloc(b, &b->Fn, n3) ||
        balloc(b, &b->rec_w, n) || balloc(b, &b->rec_id, n) || balloc(b, &b->rec, n) || balloc(b, &b->cell, n) || balloc(b, &b->slot, n) ||
        balloc(b, &b->count, C) || balloc(b, &b->tile_sums, ntiles) || balloc(b, &b->cell_start, C + 1) ||
        balloc(b, &b->keys, n) || balloc(b, &b->modes, 3 * P) ||
        balloc(b, &b->inject_m, 3 * P) || balloc(b, &b->coef, P) || balloc(b, &b->rho, P) ||
        balloc(b, &b->gtab, kGTab32Bytes * P) || balloc(b, &b->Ufar, P) || balloc(b, &b->energy, 5 * R) ||
        balloc(b, &b->ctr, R) || balloc(b, &b->d_bin[0], R) || balloc(b, &b->d_bin[1], R) ||
        balloc(b, &b->d_far[0], R) || balloc(b, &b->d_far[1], R) || balloc(b, &b->d_far_user, R) ||
        balloc(b, &b->d_energy[0], R) || balloc(b, &b->d_energy[1], R) || balloc(b, &b->d_sample, R) ||
        balloc(b, &b->d_near, R) || balloc(b, &b->d_nearf, R) || balloc(b, &b->d_geom, R) || balloc(b, &b->d_rho, R) ||
        balloc(b, &b->d_chunk, R) || balloc(b, &b->d_rf, R) || balloc(b, &b->d_state, R) ||
        balloc(b, &b->d_items, 6 * (R + 1)) || balloc(b, &b->d_coff, R + 1) || balloc(b, &b->d_off2, 2 * (R + 1)) ||
        balloc(b, &b->d_sub_items, R + 1) || balloc(b, &b->bar, 1))
        return engine_fail(b, RBSOG_ENOMEM, "device allocation failed");
    if (cudaMemset(b->count, 0, sizeof(uint32_t) * C) != cudaSuccess ||
        cudaMemset(b->bar, 0, sizeof(GridBar)) != cudaSuccess ||
        cudaMemset(b->ctr, 0, sizeof(DevCounters) * R) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_bin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return engine_fail(b, RBSOG_ECUDA, "device initialisation failed");
    return RBSOG_OK;
}

void engine_release(rbsog_batch *b) {
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->cap_stream = nullptr;
    if (b->side_stream) cudaStreamDestroy(b->side_stream);
    b->side_stream = nullptr;
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_bin) cudaEventDestroy(b->ev_bin);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    b->ev_fork = b->ev_bin = b->ev_join = nullptr;
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
}

// Each system's energies from the partials of its last force evaluation (fixed order),
// into b->energy.  Enqueued on st.
int engine_reduce_energies(rbsog_batch *b, cudaStream_t st) {
    if (b->R) launch_energy_batch(b->d_energy[0], b->R, st);
    BCK(cudaGetLastError(), "energy reduction");
    return RBSOG_OK;
}

size_t engine_footprint(const rbsog_batch *b, const HostSystem &h) {
    const SysShape sh = shape_of(h, b->near_target, chunk_for(h.N, b->rho_target), near_threads(b));
    const size_t per_particle = 2 * 9 * 8 - 2 * 4   // rest + work state (id is 4 bytes)
                                + 2 * 3 * 8          // caller-order staging
                                + 2 * 3 * 4 + 2 * 16 // F, Fn, work-order and id-order records
                                + 16 + 2 * 4 + 8;    // record, cell/slot, sort key
    const size_t per_mode = 3 * 4 * 2 + 8 + 16 + kGTab32Bytes + 8;
    return (size_t)h.N * per_particle + (size_t)h.box.ncell * 12 + (size_t)h.p.P * per_mode +
           (size_t)sh.G * 8 * h.p.P * 16 + (size_t)(near_threads(b) / 32) * sh.near_blocks * 8 + far_batch_blocks(h.N) * 8;
}

bool engine_fits(const rbsog_batch *b, const HostSystem &h) {
    return b->R < b->capR && (uint64_t)b->Ntot + h.N <= b->capN && (int64_t)b->Ctot + h.box.ncell <= b->capC &&
           (int64_t)b->Ptot + h.p.P <= b->capP;
}

int engine_append(rbsog_batch *b, HostSystem &&h) {
    if (h.p.precision != RBSOG_FP32) return engine_fail(b, RBSOG_EUNSUPPORTED, "resident systems run the FP32 path");
    if (!engine_fits(b, h)) return engine_fail(b, RBSOG_ENOMEM, "system does not fit the engine's capacity");
    const uint32_t N = h.N;
    const int cells = h.box.ncell, P = h.p.P;
    b->rho_chunk.push_back(chunk_for(N, b->rho_target));
    b->sys.push_back(std::move(h));
    b->R += 1;
    b->Ntot += N;
    b->Ctot += cells;
    b->Ptot += P;
    b->p_off.push_back(b->Ntot);
    b->c_off.push_back((uint32_t)b->Ctot);
    b->m_off.push_back((uint32_t)b->Ptot);
    b->dirty = true;
    return RBSOG_OK;
}

int engine_retain(rbsog_batch *b, const std::vector<char> &keep, cudaStream_t st) {
    std::vector<int> idx;
    for (int r = 0; r < b->R; ++r)
        if (keep[r]) idx.push_back(r);
    if ((int)idx.size() == b->R) return RBSOG_OK;
    const int Rn = (int)idx.size();
    std::vector<uint32_t> old_off(Rn + 1, 0), new_off(Rn + 1, 0), c_new{0}, m_new{0};
    std::vector<HostSystem> sys;
    std::vector<int> chunk;
    for (int k = 0; k < Rn; ++k) {
        const int r = idx[k];
        old_off[k] = b->p_off[r];
        new_off[k + 1] = new_off[k] + b->sys[r].N;
        c_new.push_back(c_new.back() + (uint32_t)b->sys[r].box.ncell);
        m_new.push_back(m_new.back() + (uint32_t)b->sys[r].p.P);
        chunk.push_back(b->rho_chunk[r]);
    }
    // counters move with their systems
    std::vector<DevCounters> c;
    if (int code = engine_counters(b, &c)) return code;
    std::vector<DevCounters> cn(Rn);
    for (int k = 0; k < Rn; ++k) cn[k] = c[idx[k]];
    if (Rn) {
        std::vector<uint32_t> offs(2 * (size_t)(Rn + 1));
        std::copy(old_off.begin(), old_off.end(), offs.begin());
        std::copy(new_off.begin(), new_off.end(), offs.begin() + Rn + 1);
        BCK(cudaMemcpyAsync(b->d_off2, offs.data(), offs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st),
            "upload relayout offsets");
        launch_relayout(b->rest, b->work, b->F, b->Fn, b->capN, b->d_off2, b->d_off2 + Rn + 1, Rn, new_off[Rn], st);
        BCK(cudaGetLastError(), "relayout");
        BCK(cudaMemcpyAsync(b->ctr, cn.data(), Rn * sizeof(DevCounters), cudaMemcpyHostToDevice, st),
            "move counters");
        BCK(cudaStreamSynchronize(st), "synchronize");
        std::swap(b->rest, b->work);
        std::swap(b->F, b->Fn);
    }
    for (int k = 0; k < Rn; ++k) sys.push_back(std::move(b->sys[idx[k]]));
    b->sys = std::move(sys);
    b->rho_chunk = chunk;
    b->R = Rn;
    b->p_off = new_off;
    b->c_off = c_new;
    b->m_off = m_new;
    b->Ntot = new_off[Rn];
    b->Ctot = (int)c_new.back();
    b->Ptot = (int)m_new.back();
    b->dirty = true;
    return RBSOG_OK;
}

int engine_commit(rbsog_batch *b) {
    if (!b->dirty) return RBSOG_OK;
    BCK(cudaDeviceSynchronize(), "synchronize");
    // sampling tables, concatenated system by system
    std::vector<unsigned long long> mp, axp;
    std::vector<int> ma, off, nmax, axa;
    for (const HostSystem &h : b->sys) {
        const std::vector<unsigned long long> mt = alias_thresholds(h.mix_prob), at = alias_thresholds(h.ax_prob);
        mp.insert(mp.end(), mt.begin(), mt.end());
        ma.insert(ma.end(), h.mix_alias.begin(), h.mix_alias.end());
        off.insert(off.end(), h.ax_off.begin(), h.ax_off.end());
        nmax.insert(nmax.end(), h.ax_nmax.begin(), h.ax_nmax.end());
        axp.insert(axp.end(), at.begin(), at.end());
        axa.insert(axa.end(), h.ax_alias.begin(), h.ax_alias.end());
    }
    if (mp.size() > b->cap_mix || !b->mix_thr) {
        size_t cm = 0, c1 = 0, c2 = 0, c3 = 0;
        BCK(regrow(b, &b->mix_thr, &cm, mp.size()), "alloc sampler");
        BCK(regrow(b, &b->mix_alias, &c1, mp.size()), "alloc sampler");
        BCK(regrow(b, &b->ax_off, &c2, 3 * cm), "alloc sampler");
        BCK(regrow(b, &b->ax_nmax, &c3, 3 * cm), "alloc sampler");
        b->cap_mix = std::min(cm, c1);
    }
    if (axp.size() > b->cap_ax || !b->ax_thr) {
        size_t ca = 0, c1 = 0;
        BCK(regrow(b, &b->ax_thr, &ca, axp.size()), "alloc sampler");
        BCK(regrow(b, &b->ax_alias, &c1, axp.size()), "alloc sampler");
        b->cap_ax = std::min(ca, c1);
    }
    BCK(upload(b->mix_thr, mp), "upload sampler");
    BCK(upload(b->mix_alias, ma), "upload sampler");
    BCK(upload(b->ax_off, off), "upload sampler");
    BCK(upload(b->ax_nmax, nmax), "upload sampler");
    BCK(upload(b->ax_thr, axp), "upload sampler");
    BCK(upload(b->ax_alias, axa), "upload sampler");
    // per-block partial buffers at the current shapes
    size_t part = 0, upart = 4, kpart = 1;
    for (int r = 0; r < b->R; ++r) {
        const HostSystem &h = b->sys[r];
        const SysShape sh = shape_of(h, b->near_target, b->rho_chunk[r], near_threads(b));
        part += (size_t)sh.G * 8 * (size_t)h.p.P;
        upart += (size_t)(near_threads(b) / 32) * sh.near_blocks;
        kpart += far_batch_blocks(h.N);
    }
    BCK(regrow(b, &b->partial, &b->cap_part, part), "alloc partials");
    BCK(regrow(b, &b->U_part, &b->cap_upart, upart), "alloc partials");
    BCK(regrow(b, &b->K_part, &b->cap_kpart, kpart), "alloc partials");
    if (int code = build_args(b)) return code;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->dirty = false;
    return RBSOG_OK;
}

int engine_set_state(rbsog_batch *b, int first, int count, const double *r, const double *v, const double *q,
                     const double *m, cudaStream_t st) {
    if (first < 0 || count < 1 || first + count > b->R) return engine_fail(b, RBSOG_EINVAL, "bad system range");
    if (int code = engine_commit(b)) return code;
    uint32_t nbk = 0;
    if (int code = sub_items(b, first, count, &nbk, st)) return code;
    // arguments of the subset; caller charges and masses when initialising
    std::vector<SysStateArgs> ss(b->h_state.begin() + first, b->h_state.begin() + first + count);
    for (int k = 0; k < count; ++k) {
        const size_t o = (size_t)b->p_off[first + k] - b->p_off[first];
        ss[k].q_user = q ? q + o : nullptr;
        ss[k].m_user = q ? m + o : nullptr;
    }
    BCK(cudaMemcpyAsync(b->d_state_sub, ss.data(), ss.size() * sizeof(SysStateArgs), cudaMemcpyHostToDevice, st),
        "upload state arguments");
    // the kernel offsets r and v by 3 p_off of each system; shift the base so that
    // element 0 is the first particle of system `first` (pointer arithmetic only)
    const size_t shift = 3 * (size_t)b->p_off[first];
    launch_set_state_batch(b->d_state_sub, b->d_sub_items, count, nbk, r - shift, v ? v - shift : nullptr,
                           b->ctr + first, count, st);
    BCK(cudaGetLastError(), "set_state");
    BCK(cudaStreamSynchronize(st), "synchronize");
    return RBSOG_OK;
}

int engine_get_state(rbsog_batch *b, int first, int count, double *r, double *v, cudaStream_t st) {
    if (first < 0 || count < 1 || first + count > b->R) return engine_fail(b, RBSOG_EINVAL, "bad system range");
    if (int code = engine_commit(b)) return code;
    uint32_t nbk = 0;
    if (int code = sub_items(b, first, count, &nbk, st)) return code;
    const size_t shift = 3 * (size_t)b->p_off[first];
    launch_get_state_batch(b->d_state + first, b->d_sub_items, count, nbk, r ? r - shift : nullptr,
                           v ? v - shift : nullptr, st);
    BCK(cudaGetLastError(), "get_state");
    return RBSOG_OK;
}

// The persistent form of one pass: every phase in one cooperative launch.
int enqueue_persistent(rbsog_batch *b, cudaStream_t st, int set, const FarArgs *far) {
    if (!b->pgrid) {
        int grid = 0;
        const int e = persist_grid(b->device, &grid);
        if (e) return engine_cuda_fail(b, (cudaError_t)e, "persistent grid size");
        b->pgrid = grid;
    }
    const int R = b->R;
    PersistArgs a{};
    a.bin = b->d_bin[set]; a.it_bin = items_of(b, kItBin); a.nb_bin = b->nb[kItBin];
    a.sample = b->d_sample; a.it_sample = items_of(b, kItSample); a.nb_sample = b->nb[kItSample];
    a.count = b->count; a.tile_sums = b->tile_sums; a.cell_start = b->cell_start; a.ncell = b->Ctot;
    a.ntiles = (b->Ctot + kScanTile - 1) / kScanTile; a.N = b->Ntot;
    a.cell = b->cell; a.slot = b->slot; a.id = b->work.id; a.keys = b->keys;
    GatherArgs &g = a.gather;
    g.in = b->work; g.out = b->rest; g.keys = b->keys; g.cell = b->cell; g.cell_start = b->cell_start; g.ctr = b->ctr;
    g.c_off = b->d_coff; g.R = R; g.rec_w = b->rec_w; g.rec = b->rec; g.N = b->Ntot;
    a.near = b->d_near; a.nearf = b->d_nearf; a.geom = b->d_geom; a.it_near = items_of(b, kItNear); a.nb_near = b->nb[kItNear];
    a.rho = b->d_rho; a.chunk = b->d_chunk; a.it_rho = items_of(b, kItRho); a.nb_rho = b->nb[kItRho];
    a.rf = b->d_rf; a.it_rf = items_of(b, kItRhoFinal); a.nb_rf = b->nb[kItRhoFinal];
    a.far = far ? far : b->d_far[set]; a.it_far = items_of(b, kItFar); a.nb_far = b->nb[kItFar];
    a.ctr = b->ctr; a.R = R; a.advance = set;
    a.bar = b->bar; a.wait_limit = b->wait_limit;
    BCK(launch_step_persist(a, b->pgrid, st), "persistent step launch");
    b->energies_stale = false;
    return RBSOG_OK;
}

int engine_enqueue(rbsog_batch *b, cudaStream_t st, int set, const FarArgs *far, cudaEvent_t *ev) {
    if (int code = engine_commit(b)) return code;
    const int R = b->R;
    if (R == 0) return RBSOG_OK;
    if (b->persistent && !ev) return enqueue_persistent(b, st, set, far);
    if (b->persistent) return engine_fail(b, RBSOG_EINVAL, "per-kernel timing needs the graph form");
    b->energies_stale = false;
    auto mark = [&](int g) {
        if (ev) cudaEventRecord(ev[g], st);
    };
    // Outside profiling (ev == nullptr) the k-sample runs on a side stream from the start
    // of the step, and the structure factor follows there as soon as binning has written
    // the work-order records, beside the rest of the cell list and the near field; far
    // waits for both streams.  Profiling keeps one stream, so each group's events time that
    // group alone.
    const bool fork = !ev;
    cudaStream_t sr = fork ? b->side_stream : st;
    if (fork) {
        BCK(cudaEventRecord(b->ev_fork, st), "fork the structure-factor stream");
        BCK(cudaStreamWaitEvent(sr, b->ev_fork, 0), "fork the structure-factor stream");
        launch_sample_batch(b->d_sample, items_of(b, kItSample), R, b->nb[kItSample], sr);
    }
    mark(0);
    launch_bin_batch(b->d_bin[set], items_of(b, kItBin), R, b->nb[kItBin], st);
    mark(1);
    if (fork) {
        BCK(cudaEventRecord(b->ev_bin, st), "hand the records to the structure-factor stream");
        BCK(cudaStreamWaitEvent(sr, b->ev_bin, 0), "hand the records to the structure-factor stream");
        launch_rho_batch(b->d_rho, b->d_chunk, items_of(b, kItRho), R, b->nb[kItRho], sr);
        launch_rho_final_batch(b->d_rf, items_of(b, kItRhoFinal), R, b->nb[kItRhoFinal], sr);
    }
    launch_scan(b->count, b->tile_sums, b->cell_start, b->Ctot, b->Ntot, st);
    mark(2);
    launch_scatter(b->cell, b->slot, b->cell_start, b->work.id, b->Ntot, b->keys, st);
    mark(3);
    GatherArgs g{};
    g.in = b->work; g.out = b->rest; g.keys = b->keys; g.cell = b->cell; g.cell_start = b->cell_start; g.ctr = b->ctr;
    g.c_off = b->d_coff; g.R = R; g.rec_w = b->rec_w; g.rec = b->rec;
    g.N = b->Ntot;
    launch_gather(RBSOG_FP32, g, st);
    mark(4);
    if (!fork) launch_sample_batch(b->d_sample, items_of(b, kItSample), R, b->nb[kItSample], st);
    mark(5);
    launch_near_batch(b->d_near, b->d_nearf, b->d_geom, items_of(b, kItNear), R, b->nb[kItNear], st);
    mark(6);
    if (fork) {
        BCK(cudaEventRecord(b->ev_join, sr), "join the structure-factor stream");
        BCK(cudaStreamWaitEvent(st, b->ev_join, 0), "join the structure-factor stream");
    } else {
        launch_rho_batch(b->d_rho, b->d_chunk, items_of(b, kItRho), R, b->nb[kItRho], st);
        mark(7);
        launch_rho_final_batch(b->d_rf, items_of(b, kItRhoFinal), R, b->nb[kItRhoFinal], st);
    }
    mark(8);
    launch_far_batch(far ? far : b->d_far[set], items_of(b, kItFar), R, b->nb[kItFar], st);
    mark(9);
    launch_close_eval_batch(b->ctr, R, set, st);   // the energies are reduced when read
    mark(10);
    BCK(cudaGetLastError(), "kernel launch");
    return RBSOG_OK;
}

int engine_launch_steps(rbsog_batch *b, int n, cudaStream_t st) {
    if (int code = engine_commit(b)) return code;
    if (n <= 0 || b->R == 0) return RBSOG_OK;
    if (!b->graph) {
        cudaGraph_t g;
        BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int code = engine_enqueue(b, b->cap_stream, 1);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (code) return code;
        BCK(e2, "end capture");
        cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e3, "graph instantiate");
    }
    for (int i = 0; i < n; ++i) BCK(cudaGraphLaunch(b->graph, st), "graph launch");
    return RBSOG_OK;
}

int engine_counters(rbsog_batch *b, std::vector<DevCounters> *out) {
    out->assign(b->capR, DevCounters{});
    BCK(cudaMemcpy(out->data(), b->ctr, b->capR * sizeof(DevCounters), cudaMemcpyDeviceToHost), "read counters");
    return RBSOG_OK;
}

int engine_status(rbsog_batch *b, const std::vector<DevCounters> &c, int r) {
    const int e = c[r].err;
    const std::string who = "system " + std::to_string(r) + ": ";
    if (e & kErrCellOverflow) return engine_fail(b, RBSOG_EOVERFLOW, who + "a cell holds more than 4096 particles");
    if (e & kErrSampler) return engine_fail(b, RBSOG_ETIMEOUT, who + "k-sampler exceeded its attempt limit");
    if (e & kErrNearStage) return engine_fail(b, RBSOG_ETIMEOUT, who + "near-field staging wait exceeded its limit");
    return RBSOG_OK;
}

}  // namespace rbsog

extern "C" {

int rbsog_batch_init(const rbsog_params *params, int32_t R, const int64_t *N, const double *q_host,
                     const double *m_host, rbsog_batch **out) {
    if (!out) return engine_fail(nullptr, RBSOG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !N || !q_host || !m_host) return engine_fail(nullptr, RBSOG_EINVAL, "params, N, q or m is NULL");
    if (R < 1 || R > (1 << 20)) return engine_fail(nullptr, RBSOG_EINVAL, "R must be in [1, 2^20]");
    std::vector<HostSystem> sys(R);
    long long nt = 0, ct = 0, pt = 0;
    for (int r = 0; r < R; ++r) {
        if (params[r].precision != RBSOG_FP32)
            return engine_fail(nullptr, RBSOG_EUNSUPPORTED, "batched systems run the FP32 path only");
        if (params[r].q2_total != 0.0)
            return engine_fail(nullptr, RBSOG_EUNSUPPORTED, "batched systems are whole systems (q2_total = 0)");
        if (params[r].sampler != RBSOG_SAMPLER_IID || params[r].temperature != RBSOG_KT_TARGET)
            return engine_fail(nullptr, RBSOG_EUNSUPPORTED,
                               "batched systems draw i.i.d. modes at the target temperature");
        if (params[r].device != params[0].device)
            return engine_fail(nullptr, RBSOG_EINVAL, "every system of a batch uses the same device");
        std::string err;
        const int code = setup_system(params[r], N[r], q_host + nt, m_host + nt, &sys[r], &err);
        if (code != RBSOG_OK) return engine_fail(nullptr, code, "system " + std::to_string(r) + ": " + err);
        nt += N[r];
        ct += sys[r].box.ncell;
        pt += params[r].P;
        if (nt >= 0x7fffffffLL || ct > (1LL << 28) || pt > (1LL << 26))
            return engine_fail(nullptr, RBSOG_EINVAL, "batch too large (particles, cells or modes)");
    }
    rbsog_batch *b = new rbsog_batch();
    auto bail = [&](int code) {
        g_batch_init_error = b->err;
        rbsog_batch_free(b);
        return code;
    };
    int code = engine_alloc(b, EngineCaps{(uint32_t)nt, (int)ct, (int)pt, R}, params[0].device);
    if (code) return bail(code);
    for (int r = 0; r < R; ++r) {
        std::string err;
        if ((code = system_S(&sys[r], &err)) != RBSOG_OK) {
            b->err = err;
            return bail(code);
        }
        if ((code = engine_append(b, std::move(sys[r]))) != RBSOG_OK) return bail(code);
    }
    if ((code = engine_commit(b)) != RBSOG_OK) return bail(code);
    // charges and masses into the rest state, positions zero: every call is defined
    // before rbsog_batch_set_state
    if (cudaMemcpy(b->stage_qm, q_host, nt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->stage_qm + b->capN, m_host, nt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->stage_a, 0, 3 * (size_t)nt * sizeof(double)) != cudaSuccess) {
        b->err = "device initialisation failed";
        return bail(RBSOG_ECUDA);
    }
    if ((code = engine_set_state(b, 0, R, b->stage_a, nullptr, b->stage_qm, b->stage_qm + b->capN, 0)) != RBSOG_OK)
        return bail(code);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        b->err = "device initialisation failed";
        return bail(RBSOG_ECUDA);
    }
    *out = b;
    return RBSOG_OK;
}

int rbsog_batch_set_state(rbsog_batch *b, const double *r, const double *v, void *stream) {
    if (!b || !r) return engine_fail(b, RBSOG_EINVAL, "batch or r is NULL");
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
    if (int code = engine_set_state(b, 0, b->R, rd, vd, nullptr, nullptr, st)) return code;
    b->force_valid = false;
    return RBSOG_OK;
}

int rbsog_batch_get_state(rbsog_batch *b, double *r, double *v, uint64_t *step, void *stream) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 3 * (size_t)b->Ntot * sizeof(double);
    double *rd = r && dev_ptr(r) ? r : (r ? b->stage_a : nullptr);
    double *vd = v && dev_ptr(v) ? v : (v ? b->stage_b : nullptr);
    if (rd || vd)
        if (int code = engine_get_state(b, 0, b->R, rd, vd, st)) return code;
    if (r && rd != r) BCK(cudaMemcpyAsync(r, rd, bytes, cudaMemcpyDefault, st), "copy r out");
    if (v && vd != v) BCK(cudaMemcpyAsync(v, vd, bytes, cudaMemcpyDefault, st), "copy v out");
    BCK(cudaStreamSynchronize(st), "synchronize");
    std::vector<DevCounters> c;
    if (int code = engine_counters(b, &c)) return code;
    if (step) *step = c[0].step;
    return check_all(b);
}

int rbsog_batch_forces(rbsog_batch *b, double *F, rbsog_energy *e, void *stream) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (int code = engine_commit(b)) return code;
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
    int code = engine_enqueue(b, st, 0, far);
    if (code) return code;
    b->force_valid = true;
    if (F && Fd != F)
        BCK(cudaMemcpyAsync(F, Fd, 3 * (size_t)b->Ntot * sizeof(double), cudaMemcpyDefault, st), "copy forces out");
    if (e) return read_energies(b, e, st);
    BCK(cudaStreamSynchronize(st), "synchronize");
    return check_all(b);
}

int rbsog_batch_step(rbsog_batch *b, int32_t nsteps, rbsog_energy *e, void *stream) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    if (nsteps < 0) return engine_fail(b, RBSOG_EINVAL, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->force_valid && nsteps > 0) {
        if (int code = engine_enqueue(b, st, 0)) return code;
        b->force_valid = true;
    }
    if (int code = engine_launch_steps(b, nsteps, st)) return code;
    if (e && !b->force_valid)
        return engine_fail(b, RBSOG_EINVAL, "no force evaluation since the last state upload: no energies to read");
    if (e) return read_energies(b, e, st);
    return RBSOG_OK;
}

int rbsog_batch_set_ksample(rbsog_batch *b, const int32_t *m_host) {
    if (!b || !m_host) return engine_fail(b, RBSOG_EINVAL, "batch or m is NULL");
    for (int l = 0; l < b->Ptot; ++l)
        if (m_host[3 * l] == 0 && m_host[3 * l + 1] == 0 && m_host[3 * l + 2] == 0)
            return engine_fail(b, RBSOG_EINVAL, "mode (0,0,0) is not in the sampled support");
    BCK(cudaDeviceSynchronize(), "synchronize");
    BCK(cudaMemcpy(b->inject_m, m_host, 3 * sizeof(int32_t) * (size_t)b->Ptot, cudaMemcpyHostToDevice), "copy modes");
    int one = 1;
    for (int r = 0; r < b->R; ++r)
        BCK(cudaMemcpy(&b->ctr[r].inject, &one, sizeof(int), cudaMemcpyHostToDevice), "set inject flag");
    return RBSOG_OK;
}

int rbsog_batch_get_ksample(rbsog_batch *b, int32_t *m_host, double *coef_host) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    BCK(cudaDeviceSynchronize(), "synchronize");
    if (m_host)
        BCK(cudaMemcpy(m_host, b->modes, 3 * sizeof(int32_t) * (size_t)b->Ptot, cudaMemcpyDeviceToHost), "copy modes");
    if (coef_host)
        BCK(cudaMemcpy(coef_host, b->coef, sizeof(double) * (size_t)b->Ptot, cudaMemcpyDeviceToHost), "copy coef");
    return check_all(b);
}

int rbsog_batch_layout(const rbsog_batch *b, int64_t *p_off, int64_t *m_off, int32_t *rho_chunk) {
    if (!b) return engine_fail(nullptr, RBSOG_EINVAL, "batch is NULL");
    for (int r = 0; r <= b->R; ++r) {
        if (p_off) p_off[r] = b->p_off[r];
        if (m_off) m_off[r] = b->m_off[r];
        if (rho_chunk && r < b->R) rho_chunk[r] = b->rho_chunk[r];
    }
    return RBSOG_OK;
}

int rbsog_batch_set_rho_chunk(rbsog_batch *b, const int32_t *rho_chunk) {
    if (!b || !rho_chunk) return engine_fail(b, RBSOG_EINVAL, "batch or rho_chunk is NULL");
    for (int r = 0; r < b->R; ++r)
        if (rho_chunk[r] < 64) return engine_fail(b, RBSOG_EINVAL, "rho_chunk must be >= 64");
    for (int r = 0; r < b->R; ++r) b->rho_chunk[r] = rho_chunk[r];
    b->dirty = true;
    return engine_commit(b);
}

int rbsog_batch_profile(rbsog_batch *b, int32_t nsteps, double *ms, void *stream) {
    if (!b || !ms || nsteps < 1) return engine_fail(b, RBSOG_EINVAL, "batch or ms is NULL, or nsteps < 1");
    GraphFormScope form(b);
    if (form.code) return form.code;
    cudaStream_t st = (cudaStream_t)stream;
    EventSet es;
    if (!es.ok) return engine_fail(b, RBSOG_ECUDA, "event creation failed");
    for (int g = 0; g < RBSOG_NPROF; ++g) ms[g] = 0.0;
    if (!b->force_valid) {
        if (int c = engine_enqueue(b, st, 0)) return c;
        b->force_valid = true;
    }
    for (int i = 0; i < nsteps; ++i) {
        if (int c = engine_enqueue(b, st, 1, nullptr, es.ev)) return c;
        BCK(cudaStreamSynchronize(st), "synchronize");
        for (int g = 0; g < RBSOG_NPROF; ++g) ms[g] += es.ms(g, g + 1);
    }
    return check_all(b);
}

int rbsog_batch_set_persistent(rbsog_batch *b, int32_t enable) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    if (enable) {
        int coop = 0;
        BCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device), "device attribute");
        if (!coop) return engine_fail(b, RBSOG_EUNSUPPORTED, "the device has no cooperative launch");
    }
    return set_form(b, enable != 0);
}

int rbsog_batch_set_wait_limit(rbsog_batch *b, int64_t polls) {
    if (!b || polls < 1) return engine_fail(b, RBSOG_EINVAL, "batch is NULL or polls < 1");
    BCK(cudaDeviceSynchronize(), "synchronize");
    b->wait_limit = polls;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return RBSOG_OK;
}

int rbsog_batch_set_shapes(rbsog_batch *b, double near_target, int32_t rho_target) {
    if (!b) return engine_fail(b, RBSOG_EINVAL, "batch is NULL");
    if (!(near_target >= 8.0 && near_target <= 4096.0) || rho_target < 64)
        return engine_fail(b, RBSOG_EINVAL, "need 8 <= near_target <= 4096 and rho_target >= 64");
    return apply_shapes(b, near_target, rho_target);
}

int rbsog_batch_tune(rbsog_batch *b, int32_t reps, double *near_target, int32_t *rho_target, void *stream) {
    if (!b || reps < 1) return engine_fail(b, RBSOG_EINVAL, "batch is NULL or reps < 1");
    GraphFormScope form(b);
    if (form.code) return form.code;
    cudaStream_t st = (cudaStream_t)stream;
    EventSet es;
    if (!es.ok) return engine_fail(b, RBSOG_EINVAL, "event creation failed");
    // the counters are restored afterwards, so the tuning evaluations leave no trace in
    // the draws; the next step re-evaluates the forces
    BCK(cudaStreamSynchronize(st), "synchronize");
    std::vector<DevCounters> saved;
    if (int code = engine_counters(b, &saved)) return code;
    const double near_c[] = {128.0, 160.0, 192.0, 230.0};
    const int rho_c[] = {256, 512, 1024, 2048};
    double best_near = b->near_target, best_near_ms = 1e30;
    int best_rho = b->rho_target;
    double best_rho_ms = 1e30;
    int code = RBSOG_OK;
    for (int ci = 0; ci < 4 && code == RBSOG_OK; ++ci) {
        // near field and structure factor are independent: tune both from one sweep
        if ((code = apply_shapes(b, near_c[ci], rho_c[ci])) != RBSOG_OK) break;
        std::vector<double> tn, tr;
        for (int i = 0; i <= reps && code == RBSOG_OK; ++i) {
            if ((code = engine_enqueue(b, st, 0, nullptr, es.ev)) != RBSOG_OK) break;
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                code = engine_cuda_fail(b, e, "synchronize");
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
    return check_all(b);
}

const char *rbsog_batch_last_error(const rbsog_batch *b) { return b ? b->err.c_str() : g_batch_init_error.c_str(); }

void rbsog_batch_free(rbsog_batch *b) {
    if (!b) return;
    engine_release(b);
    delete b;
}

}  // extern "C"
