// Job server with continuous batching: MD jobs (each an independent system with its own
// N, box, screening, coupling, P, seed and step count) arrive over time, wait until the
// resident arenas have room for them, then advance together with every other resident
// job, every kernel of a step one launch over all of them (engine.h).  Admission and
// retirement happen between rounds of a few steps; a retiring job's state is read back
// and the survivors are compacted.  A job's arithmetic and random streams depend only on
// the job (its own counters, chunking fixed by its N and the server's shapes), so its
// result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

using namespace rbsog;

namespace {

enum { kQueued = 0, kResident = 1, kDone = 2, kFailed = 3 };

struct Job {
    int64_t id = 0;
    rbsog_params p{};
    int64_t N = 0;
    std::vector<double> q, m, r, v;     // inputs, then (r, v) the final state
    int32_t nsteps = 0, steps_done = 0;
    bool evaluated = false;              // initial force evaluation done
    double t_arrival = 0, t_admit = -1, t_done = -1;
    int status = kQueued, error = RBSOG_OK;
    std::string message;
    size_t footprint = 0;
    rbsog_energy energy{};
    std::shared_ptr<HostSystem> hs;      // set up on its first admission attempt, kept while it waits
};

std::string g_server_init_error;

}  // namespace

struct rbsog_server {
    rbsog_server_config cfg{};
    rbsog_batch eng;
    std::vector<Job> jobs;
    std::vector<int64_t> resident;       // job ids in engine order
    std::deque<int64_t> waiting;         // submitted, not yet resident, in arrival order
    std::chrono::steady_clock::time_point t0;
    cudaStream_t st = nullptr;
    std::string err;
    double stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // rounds, admissions, retirements, busy s, particle-steps,
                                                  // peak resident particles, peak resident jobs, prep s
};

namespace {

int sfail(rbsog_server *s, int code, const std::string &msg) {
    if (s) s->err = msg;
    else g_server_init_error = msg;
    return code;
}

double now_s(const rbsog_server *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

#define SCK(call, where)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return sfail(s, RBSOG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Read back and retire the jobs that are done or failed; compact the rest.
int retire(rbsog_server *s, const std::vector<DevCounters> &ctr) {
    rbsog_batch *b = &s->eng;
    std::vector<char> keep(b->R, 1);
    std::vector<double> e5(5 * (size_t)b->R);
    if (b->R) {
        if (int c = engine_reduce_energies(b, s->st)) return sfail(s, c, b->err);
        SCK(cudaStreamSynchronize(s->st), "energy reduction");
        SCK(cudaMemcpy(e5.data(), b->energy, e5.size() * sizeof(double), cudaMemcpyDeviceToHost), "read energy");
    }
    for (int r = 0; r < b->R; ++r) {
        Job &j = s->jobs[s->resident[r]];
        const int code = engine_status(b, ctr, r);
        const bool failed = code != RBSOG_OK;
        if (!failed && j.steps_done < j.nsteps) continue;
        keep[r] = 0;
        const double *x = &e5[5 * (size_t)r];
        j.energy.U_near = x[0]; j.energy.U_far = x[1]; j.energy.U_self = x[2];
        j.energy.kinetic = x[3]; j.energy.total = x[4]; j.energy.step = ctr[r].step;
        if (failed) {
            j.status = kFailed;
            j.error = code;
            j.message = b->err;
        } else {
            const size_t n3 = 3 * (size_t)j.N;
            if (int c2 = engine_get_state(b, r, 1, b->stage_a, b->stage_b, s->st)) return sfail(s, c2, b->err);
            j.r.resize(n3);
            j.v.resize(n3);
            SCK(cudaMemcpyAsync(j.r.data(), b->stage_a, n3 * sizeof(double), cudaMemcpyDeviceToHost, s->st), "copy r out");
            SCK(cudaMemcpyAsync(j.v.data(), b->stage_b, n3 * sizeof(double), cudaMemcpyDeviceToHost, s->st), "copy v out");
            SCK(cudaStreamSynchronize(s->st), "synchronize");
            j.status = kDone;
            s->stats[4] += (double)j.N * (double)j.nsteps;
        }
        j.t_done = now_s(s);
        std::vector<double>().swap(j.q);
        std::vector<double>().swap(j.m);
        s->stats[2] += 1;
    }
    if (int c = engine_retain(b, keep, s->st)) return sfail(s, c, b->err);
    std::vector<int64_t> res;
    for (int r = 0; r < (int)keep.size(); ++r)
        if (keep[r]) res.push_back(s->resident[r]);
    s->resident = res;
    return RBSOG_OK;
}

// Admit arrived jobs in arrival order while they fit (a job that does not fit yet is
// skipped, later arrivals may pass it).
int admit(rbsog_server *s) {
    rbsog_batch *b = &s->eng;
    const double t = now_s(s);
    std::vector<int64_t> admitted;
    for (auto it = s->waiting.begin(); it != s->waiting.end();) {
        Job &j = s->jobs[*it];
        if (j.t_arrival > t) break;
        auto tp = std::chrono::steady_clock::now();
        std::string err;
        int code = RBSOG_OK;
        if (!j.hs) {
            // the host setup (SOG, sampler tables) once per job: a job that does not fit yet
            // keeps it until it does
            auto hs = std::make_shared<HostSystem>();
            code = setup_system(j.p, j.N, j.q.data(), j.m.data(), hs.get(), &err);
            if (code == RBSOG_OK && hs->p.precision != RBSOG_FP32) {
                code = RBSOG_EUNSUPPORTED;
                err = "served jobs run the FP32 path";
            }
            if (code == RBSOG_OK && (hs->p.sampler != RBSOG_SAMPLER_IID || hs->p.temperature != RBSOG_KT_TARGET ||
                                     hs->p.q2_total != 0.0)) {
                code = RBSOG_EUNSUPPORTED;
                err = "served jobs draw i.i.d. modes at the target temperature";
            }
            if (code == RBSOG_OK) j.hs = hs;
            s->stats[7] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
        }
        if (code == RBSOG_OK && !engine_fits(b, *j.hs) && b->R == 0) {
            code = RBSOG_ENOMEM;
            err = "job larger than the server's arenas";
        }
        if (code != RBSOG_OK) {
            j.status = kFailed;
            j.error = code;
            j.message = err;
            j.t_done = now_s(s);
            j.hs.reset();
            it = s->waiting.erase(it);
            continue;
        }
        if (!engine_fits(b, *j.hs)) {
            ++it;
            continue;
        }
        tp = std::chrono::steady_clock::now();
        HostSystem &hs = *j.hs;
        if ((code = system_S(&hs, &err)) != RBSOG_OK) return sfail(s, code, err);
        j.footprint = engine_footprint(b, hs);
        if ((code = engine_append(b, std::move(hs))) != RBSOG_OK) return sfail(s, code, b->err);
        j.hs.reset();
        s->stats[7] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
        s->resident.push_back(j.id);
        admitted.push_back(j.id);
        it = s->waiting.erase(it);
    }
    if (admitted.empty()) return RBSOG_OK;
    if (int c = engine_commit(b)) return sfail(s, c, b->err);
    for (int64_t id : admitted) {
        Job &j = s->jobs[id];
        const int r = (int)(std::find(s->resident.begin(), s->resident.end(), id) - s->resident.begin());
        const size_t n = (size_t)j.N;
        DevCounters zero{};
        SCK(cudaMemcpyAsync(b->ctr + r, &zero, sizeof zero, cudaMemcpyHostToDevice, s->st), "reset counters");
        SCK(cudaMemcpyAsync(b->stage_a, j.r.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s->st), "copy r");
        SCK(cudaMemcpyAsync(b->stage_b, j.v.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s->st), "copy v");
        SCK(cudaMemcpyAsync(b->stage_qm, j.q.data(), n * sizeof(double), cudaMemcpyHostToDevice, s->st), "copy q");
        SCK(cudaMemcpyAsync(b->stage_qm + b->capN, j.m.data(), n * sizeof(double), cudaMemcpyHostToDevice, s->st),
            "copy m");
        if (int c = engine_set_state(b, r, 1, b->stage_a, b->stage_b, b->stage_qm, b->stage_qm + b->capN, s->st))
            return sfail(s, c, b->err);
        j.status = kResident;
        j.t_admit = now_s(s);
        j.evaluated = false;
        s->stats[1] += 1;
    }
    s->stats[5] = std::max(s->stats[5], (double)b->Ntot);
    s->stats[6] = std::max(s->stats[6], (double)b->R);
    return RBSOG_OK;
}

// One round: as many passes as the next job to finish needs (capped by steps_per_round).
int round_once(rbsog_server *s) {
    rbsog_batch *b = &s->eng;
    int K = std::max(1, s->cfg.steps_per_round);
    for (int64_t id : s->resident) {
        const Job &j = s->jobs[id];
        const int need = (j.nsteps - j.steps_done) + (j.evaluated ? 0 : 1);
        K = std::min(K, std::max(need, 1));
    }
    const auto tb = std::chrono::steady_clock::now();
    if (int c = engine_launch_steps(b, K, s->st)) return sfail(s, c, b->err);
    SCK(cudaStreamSynchronize(s->st), "synchronize");
    s->stats[3] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
    s->stats[0] += 1;
    for (int64_t id : s->resident) {
        Job &j = s->jobs[id];
        const int passes = K - (j.evaluated ? 0 : 1);
        j.evaluated = true;
        j.steps_done += passes;
    }
    std::vector<DevCounters> ctr;
    if (int c = engine_counters(b, &ctr)) return sfail(s, c, b->err);
    for (int r = 0; r < b->R; ++r) {
        const Job &j = s->jobs[s->resident[r]];
        if (ctr[r].err == 0 && (int64_t)ctr[r].step != j.steps_done)
            return sfail(s, RBSOG_ECUDA, "step counter of a resident job disagrees with the schedule");
    }
    return retire(s, ctr);
}

}  // namespace

extern "C" {

int rbsog_server_create(const rbsog_server_config *cfg, rbsog_server **out) {
    if (!out) return sfail(nullptr, RBSOG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return sfail(nullptr, RBSOG_EINVAL, "cfg is NULL");
    if (cfg->max_particles < 2 || cfg->max_particles >= 0x7fffffffLL || cfg->max_cells < 1 ||
        cfg->max_cells > (1LL << 28) || cfg->max_modes < 1 || cfg->max_modes > (1LL << 26) || cfg->max_jobs < 1 ||
        cfg->max_jobs > 65536 || cfg->steps_per_round < 1 || cfg->near_target < 0 || cfg->rho_target < 0 ||
        cfg->reserved[0] != 0 || cfg->reserved[1] != 0)
        return sfail(nullptr, RBSOG_EINVAL, "server configuration out of range");
    rbsog_server *s = new rbsog_server();
    s->cfg = *cfg;
    rbsog_batch *b = &s->eng;
    if (cfg->near_target > 0) b->near_target = std::max(8.0, cfg->near_target);
    if (cfg->rho_target > 0) b->rho_target = std::max(64, (int)cfg->rho_target);
    int code = engine_alloc(b, EngineCaps{(uint32_t)cfg->max_particles, (int)cfg->max_cells, (int)cfg->max_modes,
                                          (int)cfg->max_jobs},
                            cfg->device);
    if (code == RBSOG_OK && cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess)
        code = engine_fail(b, RBSOG_ECUDA, "stream creation failed");
    if (code != RBSOG_OK) {
        g_server_init_error = b->err;
        rbsog_server_free(s);
        return code;
    }
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return RBSOG_OK;
}

int rbsog_server_submit(rbsog_server *s, const rbsog_params *p, int64_t N, const double *q, const double *m,
                        const double *r, const double *v, int32_t nsteps, double t_arrival, int64_t *job_id) {
    if (!s || !p || !q || !m || !r) return sfail(s, RBSOG_EINVAL, "server, params, q, m or r is NULL");
    if (N < 2 || N >= 0x7fffffffLL) return sfail(s, RBSOG_EINVAL, "N must be in [2, 2^31)");
    if (nsteps < 0) return sfail(s, RBSOG_EINVAL, "nsteps < 0");
    Job j;
    j.id = (int64_t)s->jobs.size();
    j.p = *p;
    j.N = N;
    j.q.assign(q, q + N);
    j.m.assign(m, m + N);
    j.r.assign(r, r + 3 * N);
    if (v) j.v.assign(v, v + 3 * N);
    else j.v.assign(3 * N, 0.0);
    j.nsteps = nsteps;
    const double t = now_s(s);
    j.t_arrival = t_arrival >= 0 ? t_arrival : t;
    // waiting list in arrival order
    auto it = s->waiting.begin();
    while (it != s->waiting.end() && s->jobs[*it].t_arrival <= j.t_arrival) ++it;
    s->waiting.insert(it, j.id);
    if (job_id) *job_id = j.id;
    s->jobs.push_back(std::move(j));
    return RBSOG_OK;
}

int rbsog_server_run(rbsog_server *s, double t_until) {
    if (!s) return sfail(s, RBSOG_EINVAL, "server is NULL");
    for (;;) {
        if (t_until >= 0 && now_s(s) >= t_until) return RBSOG_OK;
        if (int c = admit(s)) return c;
        if (!s->resident.empty()) {
            if (int c = round_once(s)) return c;
            continue;
        }
        if (s->waiting.empty()) return RBSOG_OK;
        // idle: wait for the next arrival
        const double next = s->jobs[s->waiting.front()].t_arrival;
        const double wait = next - now_s(s);
        if (wait > 0) {
            const double cap = t_until >= 0 ? std::min(wait, t_until - now_s(s)) : wait;
            if (cap > 0) std::this_thread::sleep_for(std::chrono::duration<double>(cap));
        } else if (s->resident.empty()) {
            // the head has arrived and does not fit an empty server: admit() failed it
            continue;
        }
    }
}

int rbsog_server_job(rbsog_server *s, int64_t job_id, rbsog_job_info *info, double *r_out, double *v_out) {
    if (!s || job_id < 0 || job_id >= (int64_t)s->jobs.size()) return sfail(s, RBSOG_EINVAL, "unknown job");
    const Job &j = s->jobs[job_id];
    if (info) {
        info->status = j.status;
        info->error = j.error;
        info->N = j.N;
        info->nsteps = j.nsteps;
        info->steps_done = j.steps_done;
        info->t_arrival = j.t_arrival;
        info->t_admit = j.t_admit;
        info->t_done = j.t_done;
        info->footprint_bytes = j.footprint;
        info->energy = j.energy;
    }
    if ((r_out || v_out) && j.status != kDone) return sfail(s, RBSOG_EINVAL, "job has no result yet");
    if (r_out) std::copy(j.r.begin(), j.r.end(), r_out);
    if (v_out) std::copy(j.v.begin(), j.v.end(), v_out);
    if (j.status == kFailed) return sfail(s, j.error, j.message);
    return RBSOG_OK;
}

int rbsog_server_stats(const rbsog_server *s, double *out8) {
    if (!s || !out8) return sfail(nullptr, RBSOG_EINVAL, "server or out is NULL");
    for (int i = 0; i < 8; ++i) out8[i] = s->stats[i];
    return RBSOG_OK;
}

double rbsog_server_clock(const rbsog_server *s) { return s ? now_s(s) : -1.0; }

const char *rbsog_server_last_error(const rbsog_server *s) { return s ? s->err.c_str() : g_server_init_error.c_str(); }

void rbsog_server_free(rbsog_server *s) {
    if (!s) return;
    engine_release(&s->eng);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

}  // extern "C"
