// Importance sampling of Fourier modes from P(k) = calF(k) Fhat(k) / S (Eq. 59),
// and the normalisation S = sum_{k != 0} calF(k) Fhat(k).
//
// Fhat is a sum of Gaussians (Eq. 54) that factorises per axis, so one attempt is:
//   mixture component     alias table (for calF of Eq. 62 and calF = 1 the Gaussian m,
//                         weights A_m prod_a theta_{m,a}; for calF = k^2 the pair (m, a)
//                         of k^2 Fhat = sum_m sum_a k_a^2 (...), weights A_m sigma_{m,a}
//                         prod_{b != a} theta_{m,b})
//   n_a per axis          the component's alias tables over |n| <= nmax_{m,a}: the
//                         discrete Gaussian exp(-(2 pi n/L_a)^2 / (4 b_m)), or on axis a of
//                         a k^2 component that Gaussian times (2 pi n/L_a)^2
//   reject n = 0; for calF of Eq. 62 accept with probability calF(k)/sum q^2 (increasing
//   in |k| with supremum sum q^2); the other measures accept every nonzero draw.
// For the EGS screening the mixture weights are |A_m| (the envelope of a transform that
// may change sign), psi(k) of Eq. 62 is that of its two Yukawa terms, and coef carries
// Fhat(k)/Fhat_env(k).
// which yields i.i.d. draws from P(k).  Random words: Philox4x32-10, key = seed,
// counter = (slot, 8 attempt + j, draw lo, draw hi): j = 0 Gaussian, 1..3 axes,
// 4 acceptance.  An alias draw from words (x0..x3) takes index floor((x0 2^32 + x1)
// n / 2^64) and keeps it when u53(x2, x3) < prob, else takes the alias.
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace rbsog {

namespace {

// psi(k) = sum_i c_i / (k^2 + lambda_i^-2) of the kernel's Yukawa terms
__device__ __forceinline__ double psi_of(const Yterms &y, double k2) {
    double p = y.c[0] / (k2 + y.inv_lam2[0]);
    if (y.n > 1) p += y.c[1] / (k2 + y.inv_lam2[1]);
    return p;
}

// calF of the measure (Eq. 62 and its variants) at k^2; A = k_B T V.  One Yukawa term of
// weight 1 keeps the form s / (k^2 + lambda^-2).
__device__ __forceinline__ double calF_of(int measure, double k2, double A, double Q2, const Yterms &y) {
    if (measure == 1) return 1.0;
    if (measure == 2) return k2;
    const double s = measure == 3 ? 4.0 * CUDART_PI : 1.0;
    const double t = y.n == 1 ? s / (k2 + y.inv_lam2[0]) : s * psi_of(y, k2);
    return A / (A / Q2 + t);
}

// keep index i when u53(z, w) < prob_i, i.e. when its 53-bit integer is below the
// precomputed threshold ceil(prob_i 2^53)
__device__ __forceinline__ int alias_draw(U4 w, const unsigned long long *thr, const int *alias, int n) {
    unsigned long long u = ((unsigned long long)w.x << 32) | (unsigned long long)w.y;
    int i = (int)__umul64hi(u, (unsigned long long)n);
    const unsigned long long U = ((unsigned long long)(w.z >> 11) << 32) | (unsigned long long)w.w;
    return (U < thr[i]) ? i : alias[i];
}

// coef = S / (P V calF(k)) (Eqs. 60, 62), calF of the measure at A = k_B T V; with a
// far-field transform that may change sign, times Fhat(k) / Fhat_env(k) (draws from the
// envelope)
__device__ __forceinline__ double mode_coef(const SampleArgs &a, const int m[3], double A, double S) {
    double kx = a.tpl[0] * m[0], ky = a.tpl[1] * m[1], kz = a.tpl[2] * m[2];
    double k2 = kx * kx + ky * ky + kz * kz;
    const double calF = calF_of(a.measure, k2, A, a.Q2, a.y);
    double coef = S / ((double)a.P * a.V * calF);
    if (a.nfh > 0) {
        double fh = 0.0, fe = 0.0;
        for (int g = 0; g < a.nfh; ++g) {
            const double e = a.fA[g] * exp(-k2 * a.finv4b[g]);
            fh += e;
            fe += fabs(e);
        }
        coef = coef * (fh / fe);
    }
    return coef;
}

// |k|^2 of mode n in IEEE operations without contraction: (kx^2 + ky^2) + kz^2
__device__ __forceinline__ double k2_rn(const SampleArgs &a, const int n[3]) {
    const double kx = __dmul_rn(a.tpl[0], (double)n[0]);
    const double ky = __dmul_rn(a.tpl[1], (double)n[1]);
    const double kz = __dmul_rn(a.tpl[2], (double)n[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky)), __dmul_rn(kz, kz));
}

// A t of the acceptance tests: A (k^2 + lambda^-2) for one Yukawa term, A / psi(k) otherwise
__device__ __forceinline__ double At_of(const SampleArgs &a, double A, double k2) {
    return a.y.n == 1 ? __dmul_rn(A, __dadd_rn(k2, a.y.inv_lam2[0])) : __ddiv_rn(A, psi_of(a.y, k2));
}

// FP32 pre-test of the acceptance test u (A t + Q2a) < A t, A t = A (k^2 + lambda^-2).
// With D = A t - u (A t + Q2a) in real arithmetic on the FP64 operands, the FP64 test
// accepts when D > 2^-52 (A t + Q2a) and rejects when D < -2^-52 (A t + Q2a) (two
// roundings of the product).  The FP32 value D32 = fma(-u32, den, At32) differs from D by
// at most 2e-6 (A t + Q2a): 2 pi / L, lambda^-2, Q2a and A each rounded to FP32 (2^-24
// relative), k^2 in three roundings, A t in two more, den = At32 + Q2a32 in one, u
// truncated to its leading 24 bits (u - u32 in [0, 2^-24)) and the fused product and
// difference in one, with every operand normal (the range checks here and in
// sample_set_prefilter).  So |D32| > 1e-5 den decides as the FP64 test does; the rest
// (about 2e-5 of the draws) take the FP64 test.  Returns 1 accept, 0 reject, -1 open.
__device__ __forceinline__ int accept_pretest(const SampleArgs &a, float Af, const int n[3], U4 wa) {
    const float u32 = (float)(((wa.x >> 11) << 3) | (wa.y >> 29)) * 5.9604644775390625e-8f;
    const float kx = a.tplf[0] * (float)n[0], ky = a.tplf[1] * (float)n[1], kz = a.tplf[2] * (float)n[2];
    const float k2 = fmaf(kz, kz, fmaf(ky, ky, kx * kx));
    const float At = Af * (k2 + a.il2f);
    const float den = At + a.Q2af;
    if (!(At >= 1e-25f && den <= 1e30f)) return -1;
    const float D = fmaf(-u32, den, At), m = 1e-5f * den;
    return D > m ? 1 : (D < -m ? 0 : -1);
}

// One slot l per warp: lane j tries attempt att0 + j, so 32 consecutive attempts run at
// once and the slot takes the accepted attempt with the smallest index, exactly the draw
// a sequential loop over attempts returns (the random words depend only on the counter).
__device__ __forceinline__ void sample_warp(const SampleArgs &a, int l) {
    const int lane = threadIdx.x & 31;
    const double A = a.temp ? a.temp[0] : a.A;
    const double S = a.temp ? a.temp[1] : a.S;
    const bool pre = a.f32pre && A >= 1e-30 && A <= 1e30;
    const float Af = (float)A;
    int m[3] = {1, 0, 0};
    if (a.ctr->inject) {
        m[0] = a.inject_m[3 * l]; m[1] = a.inject_m[3 * l + 1]; m[2] = a.inject_m[3 * l + 2];
    } else {
        const unsigned long long d = a.ctr->draw;
        const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
        const uint32_t d0 = (uint32_t)d, d1 = (uint32_t)(d >> 32);
        bool done = false;
        for (int att0 = 0; att0 < kMaxAttempts && !done; att0 += 32) {
            const uint32_t cb = 8u * (uint32_t)(att0 + lane);
            const int g = alias_draw(philox10((uint32_t)l, cb, d0, d1, k0, k1), a.tab.mix_thr, a.tab.mix_alias,
                                     a.tab.mtot);
            int n[3];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const int off = a.tab.ax_off[3 * g + ax], nm = a.tab.ax_nmax[3 * g + ax];
                n[ax] = alias_draw(philox10((uint32_t)l, cb + 1u + ax, d0, d1, k0, k1), a.tab.ax_thr + off,
                                   a.tab.ax_alias + off, 2 * nm + 1) - nm;
            }
            bool ok = !(n[0] == 0 && n[1] == 0 && n[2] == 0);
            if (ok && (a.measure == 0 || a.measure == 3)) {
                U4 wa = philox10((uint32_t)l, cb + 4u, d0, d1, k0, k1);
                const int t = pre ? accept_pretest(a, Af, n, wa) : -1;
                if (t >= 0) {
                    ok = t != 0;
                } else {
                    double u = u53_of(wa.x, wa.y);
                    // u < A / (A + Q2 psi), evaluated without division as u (A t + Q2) < A t
                    // with t = 1/psi = k^2 + lambda^-2 for one Yukawa term
                    const double At = At_of(a, A, k2_rn(a, n));
                    ok = __dmul_rn(u, __dadd_rn(At, a.Q2a)) < At;
                }
            }
            const unsigned acc = __ballot_sync(0xffffffffu, ok);
            if (acc) {
                const int src = __ffs(acc) - 1;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) m[ax] = __shfl_sync(0xffffffffu, n[ax], src);
                done = true;
            }
        }
        if (!done && lane == 0) atomicOr(&a.ctr->err, kErrSampler);
    }
    if (lane == 0) {
        a.m_out[3 * l] = m[0]; a.m_out[3 * l + 1] = m[1]; a.m_out[3 * l + 2] = m[2];
        a.coef_out[l] = mode_coef(a, m, A, S);
    }
}

// Metropolis-Hastings chains (RBSOG_SAMPLER_MH), one thread per chain l.  The proposal is
// the mixture draw of the i.i.d. sampler (component and per-axis alias tables) with Philox
// counter (l, 8 (t mod 2^29) + j, t >> 29, 2^31), t the chain's proposal index, key = seed:
// j = 0 component, 1..3 axes, 4 the uniform u.  A proposal n = 0 is rejected; otherwise n
// replaces the state m when (u At_m)(At_n + Q2) < At_n (At_m + Q2), i.e. u < a(n)/a(m) with
// a = calF / sum q^2 (for calF = 1 and k^2, a = 1 and every nonzero proposal is taken).  A
// chain with t = 0 starts at its first nonzero proposal and makes `burnin` more; later
// evaluations make `sweeps`.  The batch of the evaluation is the P chain states.
__device__ __forceinline__ void mh_propose(const SampleArgs &a, int l, unsigned long long &t, int n[3], double &u) {
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint32_t c1 = 8u * (uint32_t)(t & ((1ull << 29) - 1ull));
    const uint32_t c2 = (uint32_t)(t >> 29);
    const int g = alias_draw(philox10((uint32_t)l, c1, c2, 0x80000000u, k0, k1), a.tab.mix_thr, a.tab.mix_alias,
                             a.tab.mtot);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int off = a.tab.ax_off[3 * g + ax], nm = a.tab.ax_nmax[3 * g + ax];
        n[ax] = alias_draw(philox10((uint32_t)l, c1 + 1u + ax, c2, 0x80000000u, k0, k1), a.tab.ax_thr + off,
                           a.tab.ax_alias + off, 2 * nm + 1) - nm;
    }
    const U4 wa = philox10((uint32_t)l, c1 + 4u, c2, 0x80000000u, k0, k1);
    u = u53_of(wa.x, wa.y);
    t += 1ull;
}

__global__ void __launch_bounds__(128) k_sample_mh(SampleArgs a, MHChainArgs c) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.P) return;
    const double A = a.temp ? a.temp[0] : a.A;
    const double S = a.temp ? a.temp[1] : a.S;
    int m[3];
    if (a.ctr->inject) {
        m[0] = a.inject_m[3 * l]; m[1] = a.inject_m[3 * l + 1]; m[2] = a.inject_m[3 * l + 2];
    } else {
        const bool adaptive = a.measure == 0 || a.measure == 3;
        unsigned long long t = c.t[l];
        int cur[3] = {c.m[3 * l], c.m[3 * l + 1], c.m[3 * l + 2]};
        int nprop = c.sweeps;
        if (t == 0ull) {
            bool found = false;
            for (int tries = 0; tries < kMaxAttempts && !found; ++tries) {
                int n[3];
                double u;
                mh_propose(a, l, t, n, u);
                if (!(n[0] == 0 && n[1] == 0 && n[2] == 0)) {
                    cur[0] = n[0]; cur[1] = n[1]; cur[2] = n[2];
                    found = true;
                }
            }
            if (!found) {
                atomicOr(&a.ctr->err, kErrSampler);
                cur[0] = 1; cur[1] = 0; cur[2] = 0;
            }
            nprop = c.burnin;
        }
        double At_cur = adaptive ? At_of(a, A, k2_rn(a, cur)) : 0.0;
        for (int s = 0; s < nprop; ++s) {
            int n[3];
            double u;
            mh_propose(a, l, t, n, u);
            if (n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
            bool ok = true;
            double At_new = 0.0;
            if (adaptive) {
                At_new = At_of(a, A, k2_rn(a, n));
                ok = __dmul_rn(__dmul_rn(u, At_cur), __dadd_rn(At_new, a.Q2a)) <
                     __dmul_rn(At_new, __dadd_rn(At_cur, a.Q2a));
            }
            if (ok) {
                cur[0] = n[0]; cur[1] = n[1]; cur[2] = n[2];
                At_cur = At_new;
            }
        }
        c.t[l] = t;
        c.m[3 * l] = cur[0]; c.m[3 * l + 1] = cur[1]; c.m[3 * l + 2] = cur[2];
        m[0] = cur[0]; m[1] = cur[1]; m[2] = cur[2];
    }
    a.m_out[3 * l] = m[0]; a.m_out[3 * l + 1] = m[1]; a.m_out[3 * l + 2] = m[2];
    a.coef_out[l] = mode_coef(a, m, A, S);
}

// Instantaneous temperature and the normalisation S at it (RBSOG_KT_INSTANT).  Every block
// sums the kinetic-energy partials in the same fixed order (so all agree on k_B T), then its
// share of the table; the last block to arrive adds the block sums in block order.
__device__ __forceinline__ double block_sum_256(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;     // valid in thread 0
}

__global__ void __launch_bounds__(256) k_temperature(TempArgs a) {
    __shared__ double sh[8];
    __shared__ double kTV_sh;
    double k = 0.0;
    for (int i = threadIdx.x; i < a.nK; i += blockDim.x) k += a.K_part[i];
    k = block_sum_256(k, sh);
    if (threadIdx.x == 0) kTV_sh = (a.two_3N * k) * a.V;
    __syncthreads();
    const double A = kTV_sh;
    double s = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += gridDim.x * blockDim.x)
        s += calF_of(a.measure, a.k2[j], A, a.Q2, a.y) * a.W[j];
    s = block_sum_256(s, sh);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.part[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double S = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) S += ((volatile double *)a.part)[b];
        a.out[0] = A;
        a.out[1] = S;
        a.out[2] = A / a.V;
        *a.done = 0u;
    }
}

constexpr int kSampleWarps = 4;   // slots per 128-thread block

__global__ void __launch_bounds__(128) k_sample(SampleArgs a) {
    const int l = blockIdx.x * kSampleWarps + (threadIdx.x >> 5);
    if (l < a.P) sample_warp(a, l);
}

__global__ void __launch_bounds__(128) k_sample_batch(const SampleArgs *args, const uint32_t *items, int R) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const SampleArgs &a = args[lo];
    const int l = (int)(blockIdx.x - items[lo]) * kSampleWarps + (threadIdx.x >> 5);
    if (l < a.P) sample_warp(a, l);
}

// S over the ball |k|^2 <= kmax2: block x = m_x slab; fixed-order reduction.
__global__ void __launch_bounds__(256) k_S(SArgs a, double *partials) {
    __shared__ double sh[256];
    const int mx = (int)blockIdx.x - a.nmax[0];
    const double kx = a.tpl[0] * mx;
    const int ny = 2 * a.nmax[1] + 1, nz = 2 * a.nmax[2] + 1;
    double acc = 0.0;
    for (long long t = threadIdx.x; t < (long long)ny * nz; t += blockDim.x) {
        const int my = (int)(t / nz) - a.nmax[1];
        const int mz = (int)(t % nz) - a.nmax[2];
        if (mx == 0 && my == 0 && mz == 0) continue;
        const double ky = a.tpl[1] * my, kz = a.tpl[2] * mz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 > a.kmax2) continue;
        double fh = 0.0;
        for (int g = 0; g < a.mtot; ++g) fh += a.A[g] * exp(-k2 * a.inv4b[g]);
        acc += calF_of(a.measure, k2, a.kTV, a.Q2, a.y) * fh;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

}  // namespace

// The FP32 pre-test needs calF of Eq. 62 with one Yukawa term and FP32 copies of 2 pi / L,
// lambda^-2 and Q2a that are normal (or zero) and far from the FP32 overflow, so that
// every rounding in it is relative; A is checked on the device (it may be the
// instantaneous temperature's).
void sample_set_prefilter(SampleArgs *a) {
    auto normal = [](double x) { return x >= 1e-30 && x <= 1e30; };
    bool ok = (a->measure == 0 || a->measure == 3) && a->y.n == 1 && a->nfh == 0;
    for (int d = 0; d < 3; ++d) ok = ok && a->tpl[d] >= 1e-15 && a->tpl[d] <= 1e15;
    const double il2 = a->y.inv_lam2[0];
    ok = ok && (il2 == 0.0 || normal(il2)) && (a->Q2a == 0.0 || normal(a->Q2a));
    a->f32pre = ok ? 1 : 0;
    for (int d = 0; d < 3; ++d) a->tplf[d] = (float)a->tpl[d];
    a->il2f = (float)il2;
    a->Q2af = (float)a->Q2a;
}

void launch_sample(const SampleArgs &a, cudaStream_t st) {
    k_sample<<<(a.P + kSampleWarps - 1) / kSampleWarps, 128, 0, st>>>(a);
}

void launch_sample_mh(const SampleArgs &a, const MHChainArgs &c, cudaStream_t st) {
    k_sample_mh<<<(a.P + 127) / 128, 128, 0, st>>>(a, c);
}

void launch_temperature(const TempArgs &a, cudaStream_t st) {
    k_temperature<<<kTempBlocks, 256, 0, st>>>(a);
}

uint32_t sample_batch_blocks(int P) { return (uint32_t)((P + kSampleWarps - 1) / kSampleWarps); }

void launch_sample_batch(const SampleArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st) {
    k_sample_batch<<<nblocks, 128, 0, st>>>(args, items, R);
}

void launch_S(const SArgs &a, double *partials, cudaStream_t st) {
    k_S<<<2 * a.nmax[0] + 1, 256, 0, st>>>(a, partials);
}

}  // namespace rbsog
