// Structure factor for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed, pre-reserved
// memory budget owned by another allocator (for example a caching allocator that
// would have to give memory back first), and latency-critical loops that must not
// pay for an allocation that may synchronise the whole device.  For them this file
// offers rbsog_rho_noalloc: the FP32 structure-factor computation of the force step,
// with its per-block partial sums kept in a fixed, statically sized device array
// instead of a buffer from cudaMalloc.  The caller still passes inputs and outputs.
//
// The array g_noalloc_partials lives in every GPU that loads this library until the
// process exits (4 MiB).  Host code cannot use the array's name as a device address,
// so the address is fetched once per device with cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rbsog.h"
#include "common.cuh"
#include "devmath.cuh"

namespace rbsog {
void set_global_error(const std::string &msg);   // rbsog.cu
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaTile = 512;              // particles staged in shared memory per tile
constexpr int kNaMaxBlocks = 152;         // one block per SM
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaSlots = 262144;       // double2 partial sums: 4 MiB

static __device__ __align__(256) double2 g_noalloc_partials[kNaSlots];

std::mutex g_na_mutex;
double2 *g_na_addr[kNaMaxDevices] = {nullptr};

int na_fail(int code, const std::string &msg) {
    set_global_error(msg);      // reported by rbsog_last_error(NULL)
    return code;
}

// Mode groups and particle subsets of one pass.  Subsets (warps sharing a mode group over
// different particles) are used only with a single pass (P <= 256), so the scratch needs
// G x P slots whenever P > 128.
__host__ __device__ inline void na_split(int P, int pass_base, int ML, int &ngroups, int &nsub) {
    const int left = P - pass_base;
    ngroups = (left + 32 * ML - 1) / (32 * ML);
    if (ngroups > 8) ngroups = 8;
    nsub = (ML == 1) ? 8 / ngroups : 1;
}

inline int na_ml(int P) { return P <= 256 ? 1 : (P <= 512 ? 2 : 4); }

// Per block: partial rho over a contiguous particle chunk.  Positions are turned into the
// 2^32 fixed point s = floor(frac(r/L) 2^32) while staging, so no record buffer is needed.
template <int ML>
__global__ void __launch_bounds__(kNaThreads)
    k_rho_noalloc(const double *r, const double *q, uint32_t N, double L0, double L1, double L2, const int *m,
                  int P, int chunk, int nsub_stride, double2 *partial) {
    __shared__ uint4 sp[kNaTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pass_base = blockIdx.y * 256 * ML;
    int ngroups, nsub;
    na_split(P, pass_base, ML, ngroups, nsub);
    const int g = warp % ngroups, sub = warp / ngroups;
    const bool active = sub < nsub;
    int mm[ML][3], lidx[ML];
#pragma unroll
    for (int j = 0; j < ML; ++j) {
        lidx[j] = pass_base + g * 32 * ML + j * 32 + lane;
        const bool ok = active && lidx[j] < P;
        mm[j][0] = ok ? m[3 * lidx[j]] : 0;
        mm[j][1] = ok ? m[3 * lidx[j] + 1] : 0;
        mm[j][2] = ok ? m[3 * lidx[j] + 2] : 0;
    }
    float sre[ML], cre[ML], sim[ML], cim[ML];
#pragma unroll
    for (int j = 0; j < ML; ++j) sre[j] = cre[j] = sim[j] = cim[j] = 0.f;
    const uint32_t begin = (uint32_t)blockIdx.x * (uint32_t)chunk;
    uint32_t end = begin + (uint32_t)chunk;
    if (end > N) end = N;
    const double Ls[3] = {L0, L1, L2};
    for (uint32_t base = begin; base < end; base += kNaTile) {
        const int tn = (int)min((uint32_t)kNaTile, end - base);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) {
            const size_t i = (size_t)(base + t);
            uint32_t s[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double u = __ddiv_rn(r[3 * i + d], Ls[d]);
                double f = __dsub_rn(u, floor(u));
                if (f >= 1.0) f = 0.0;
                s[d] = (uint32_t)__double2ull_rz(f * 4294967296.0);
            }
            sp[t] = make_uint4(s[0], s[1], s[2], __float_as_uint((float)q[i]));
        }
        __syncthreads();
        if (!active) continue;
        float tre[ML], tim[ML];
#pragma unroll
        for (int j = 0; j < ML; ++j) tre[j] = tim[j] = 0.f;
        for (int i = sub; i < tn; i += nsub) {
            const uint4 rr = sp[i];
            const float qq = __uint_as_float(rr.w);
#pragma unroll
            for (int j = 0; j < ML; ++j) {
                const uint32_t th = (uint32_t)mm[j][0] * rr.x + (uint32_t)mm[j][1] * rr.y + (uint32_t)mm[j][2] * rr.z;
                float sn, cs;
                const float qs = flip(qq, half_turn_sincos(th, sn, cs));
                tre[j] = fmaf(qs, cs, tre[j]);
                tim[j] = fmaf(qs, sn, tim[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < ML; ++j) {
            kahan_add(sre[j], cre[j], tre[j]);
            kahan_add(sim[j], cim[j], tim[j]);
        }
    }
    if (!active) return;
#pragma unroll
    for (int j = 0; j < ML; ++j)
        if (lidx[j] < P)
            partial[((size_t)blockIdx.x * nsub_stride + sub) * P + lidx[j]] =
                make_double2((double)sre[j] - (double)cre[j], (double)sim[j] - (double)cim[j]);
}

// Fixed-order sum of the partials of every block into rho (P complex values, FP64).
__global__ void __launch_bounds__(1024) k_rho_noalloc_final(const double2 *partial, int G, int P, int ML,
                                                           int nsub_stride, double *rho) {
    for (int l = threadIdx.x; l < P; l += blockDim.x) {
        int ngroups, nsub;
        na_split(P, (l / (256 * ML)) * 256 * ML, ML, ngroups, nsub);
        double re = 0.0, im = 0.0;
        for (int b = 0; b < G; ++b)
            for (int s = 0; s < nsub; ++s) {
                const double2 v = partial[((size_t)b * nsub_stride + s) * P + l];
                re += v.x;
                im += v.y;
            }
        rho[2 * l] = re;
        rho[2 * l + 1] = im;
    }
}

// Device address of g_noalloc_partials on the current device (looked up once per device).
int na_scratch(double2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(RBSOG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return na_fail(RBSOG_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return na_fail(RBSOG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_addr[dev] = (double2 *)p;
    }
    *out = g_na_addr[dev];
    return RBSOG_OK;
}

}  // namespace
}  // namespace rbsog

using namespace rbsog;

extern "C" int rbsog_rho_noalloc(const double *r_dev, const double *q_dev, int64_t N, const double *box_host,
                                 const int32_t *m_dev, int32_t P, double *rho_dev, void *stream) {
    if (!r_dev || !q_dev || !box_host || !m_dev || !rho_dev)
        return na_fail(RBSOG_EINVAL, "rbsog_rho_noalloc: a pointer argument is NULL");
    if (N < 1 || N > 0x7fffffffLL) return na_fail(RBSOG_EINVAL, "rbsog_rho_noalloc: N must be in [1, 2^31)");
    if (P < 1 || P > 4096) return na_fail(RBSOG_EINVAL, "rbsog_rho_noalloc: P must be in [1, 4096]");
    for (int d = 0; d < 3; ++d)
        if (!(box_host[d] > 0)) return na_fail(RBSOG_EINVAL, "rbsog_rho_noalloc: box lengths must be > 0");
    const int ML = na_ml(P);
    int nsub_stride = 1;
    for (int base = 0; base < P; base += 256 * ML) {
        int ng, ns;
        na_split(P, base, ML, ng, ns);
        if (ns > nsub_stride) nsub_stride = ns;
    }
    const uint32_t n = (uint32_t)N;
    int G = (int)((n + 63) / 64);
    if (G > kNaMaxBlocks) G = kNaMaxBlocks;
    const size_t need = (size_t)G * nsub_stride * P;
    if (need > kNaSlots) {
        return na_fail(RBSOG_EINVAL, "rbsog_rho_noalloc: blocks x particle subsets x P = " + std::to_string(need) +
                                         " partial sums exceed the fixed scratch of " + std::to_string(kNaSlots) +
                                         " (4 MiB); use a smaller P (at most 1724 for N >= 9728)");
    }
    double2 *scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc != RBSOG_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int chunk = (int)((n + (uint32_t)G - 1) / (uint32_t)G);
    dim3 grid(G, (P + 256 * ML - 1) / (256 * ML));
    if (ML == 1)
        k_rho_noalloc<1><<<grid, kNaThreads, 0, st>>>(r_dev, q_dev, n, box_host[0], box_host[1], box_host[2], m_dev,
                                                      P, chunk, nsub_stride, scratch);
    else if (ML == 2)
        k_rho_noalloc<2><<<grid, kNaThreads, 0, st>>>(r_dev, q_dev, n, box_host[0], box_host[1], box_host[2], m_dev,
                                                      P, chunk, nsub_stride, scratch);
    else
        k_rho_noalloc<4><<<grid, kNaThreads, 0, st>>>(r_dev, q_dev, n, box_host[0], box_host[1], box_host[2], m_dev,
                                                      P, chunk, nsub_stride, scratch);
    k_rho_noalloc_final<<<1, 1024, 0, st>>>(scratch, G, P, ML, nsub_stride, rho_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RBSOG_ECUDA, std::string("rbsog_rho_noalloc launch: ") + cudaGetErrorString(e));
    return RBSOG_OK;
}
