// Far-field kernels of one RBSOG step (the near field is in k_near.cu).
//
//   k_rho     structure factor rho(k_l) = sum_j q_j exp(i k_l.r_j) (Sec. 2): per block,
//             lane <-> mode, particles broadcast from shared memory; phases are exact
//             integer products m.s modulo 2^32 (2^64), so sin/cos see [-pi, pi).
//   k_rho_fin fixed-order grid reduction, U*_F of Eq. (60) and the gather table.
//   k_far32/64 F*_i = -q_i sum_l coef_l k_l Im(exp(-i k_l.r_i) rho_l) (Eq. 60), added to
//             the near force, fused with the closing half kick v += F dt/(2m).
//   k_energy  fixed-order reduction of the energy partials.
#include <math_constants.h>

#include "common.cuh"
#include "devmath.cuh"
#include "devutil.cuh"
#include "kernels.h"

namespace rbsog {

namespace {

constexpr int kRhoThreads = 256;
constexpr int kRhoTile = 512;       // particles staged per tile (FP32: 8 KB, FP64: 16 KB)
constexpr int kFarThreads = 256;
constexpr int kFarTile = 512;       // modes staged per tile

template <typename T>
__device__ __forceinline__ T block_reduce_sum(T v, T *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    T out = sh[0];
    __syncthreads();
    return out;
}

// ------------------------------------------------------------------ structure factor
// Work split of one block: warp w serves mode group g = w % ngroups (32*ML modes of the
// pass) and particle subset sub = w / ngroups (stride nsub through each tile).
__device__ __forceinline__ void rho_split(int P, int pass_base, int ML, int &ngroups, int &nsub) {
    int left = P - pass_base;
    ngroups = (left + 32 * ML - 1) / (32 * ML);
    if (ngroups > 8) ngroups = 8;
    nsub = 8 / ngroups;
}

template <int ML>
__device__ __forceinline__ void rho32_body(const RhoArgs &a, int chunk, unsigned bx, unsigned by, uint4 *sp) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pass_base = (int)by * 256 * ML;
    int ngroups, nsub;
    rho_split(a.P, pass_base, ML, ngroups, nsub);
    const int g = warp % ngroups, sub = warp / ngroups;
    const bool active = sub < nsub;
    int mm[ML][3];
    int lidx[ML];
#pragma unroll
    for (int j = 0; j < ML; ++j) {
        lidx[j] = pass_base + g * 32 * ML + j * 32 + lane;
        const bool ok = active && lidx[j] < a.P;
        mm[j][0] = ok ? a.m[3 * lidx[j]] : 0;
        mm[j][1] = ok ? a.m[3 * lidx[j] + 1] : 0;
        mm[j][2] = ok ? a.m[3 * lidx[j] + 2] : 0;
    }
    float sre[ML], cre[ML], sim[ML], cim[ML];
#pragma unroll
    for (int j = 0; j < ML; ++j) sre[j] = cre[j] = sim[j] = cim[j] = 0.f;
    const uint32_t begin = (uint32_t)bx * (uint32_t)chunk;
    uint32_t end = begin + (uint32_t)chunk;
    if (end > a.N) end = a.N;
    const uint4 *rec = (const uint4 *)a.rec;
    for (uint32_t base = begin; base < end; base += kRhoTile) {
        const int tn = (int)min((uint32_t)kRhoTile, end - base);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) sp[t] = rec[base + t];
        __syncthreads();
        if (!active) continue;
        float tre[ML], tim[ML];
#pragma unroll
        for (int j = 0; j < ML; ++j) tre[j] = tim[j] = 0.f;
        if constexpr (ML == 1) {
            for (int i = sub; i < tn; i += nsub) {
                const uint4 r = sp[i];
                const float q = __uint_as_float(r.w);
                const uint32_t th = (uint32_t)mm[0][0] * r.x + (uint32_t)mm[0][1] * r.y + (uint32_t)mm[0][2] * r.z;
                float sn, cs;
                const float qs = flip(q, half_turn_sincos(th, sn, cs));
                tre[0] = fmaf(qs, cs, tre[0]);
                tim[0] = fmaf(qs, sn, tim[0]);
            }
        } else {
            // two modes per packed FP32x2 operation
            unsigned long long re2[ML / 2], im2[ML / 2];
#pragma unroll
            for (int h = 0; h < ML / 2; ++h) re2[h] = im2[h] = 0ull;
            const unsigned long long K2 = pk2(kTwoPiOver2p32, kTwoPiOver2p32);
            for (int i = sub; i < tn; i += nsub) {
                const uint4 r = sp[i];
                const float q = __uint_as_float(r.w);
#pragma unroll
                for (int h = 0; h < ML / 2; ++h) {
                    const int j0 = 2 * h, j1 = 2 * h + 1;
                    const uint32_t t0 = (uint32_t)mm[j0][0] * r.x + (uint32_t)mm[j0][1] * r.y + (uint32_t)mm[j0][2] * r.z;
                    const uint32_t t1 = (uint32_t)mm[j1][0] * r.x + (uint32_t)mm[j1][1] * r.y + (uint32_t)mm[j1][2] * r.z;
                    const uint32_t g0 = (t0 ^ (t0 << 1)) & 0x80000000u, g1 = (t1 ^ (t1 << 1)) & 0x80000000u;
                    float x0, x1;
                    upk2(mul2(pk2((float)(int)(t0 ^ g0), (float)(int)(t1 ^ g1)), K2), x0, x1);
                    float s0, c0, s1, c1;
                    __sincosf(x0, &s0, &c0);
                    __sincosf(x1, &s1, &c1);
                    const unsigned long long qs = pk2(flip(q, g0), flip(q, g1));
                    re2[h] = fma2(qs, pk2(c0, c1), re2[h]);
                    im2[h] = fma2(qs, pk2(s0, s1), im2[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < ML / 2; ++h) {
                upk2(re2[h], tre[2 * h], tre[2 * h + 1]);
                upk2(im2[h], tim[2 * h], tim[2 * h + 1]);
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
        if (lidx[j] < a.P)
            a.partial[((size_t)bx * 8 + sub) * a.P + lidx[j]] =
                make_double2((double)sre[j] - (double)cre[j], (double)sim[j] - (double)cim[j]);
}

// at most 64 registers (four blocks' worth per SM): beside rho's three blocks per SM the
// near field then keeps two CTAs instead of one (72 registers measured 1% slower per step)
template <int ML>
__global__ void __launch_bounds__(kRhoThreads, 4) k_rho32(RhoArgs a, int chunk) {
    __shared__ uint4 sp[kRhoTile];
    rho32_body<ML>(a, chunk, blockIdx.x, blockIdx.y, sp);
}


// Batched systems: block -> (system, particle chunk, pass of 256 modes); a system has
// G chunks x ceil(P/256) passes.
__global__ void __launch_bounds__(kRhoThreads) k_rho_batch(const RhoArgs *args, const int *chunk,
                                                           const uint32_t *items, int R) {
    __shared__ uint4 sp[kRhoTile];
    const int r = item_system(items, R, blockIdx.x);
    const RhoArgs &a = args[r];
    const unsigned local = blockIdx.x - items[r];
    rho32_body<1>(a, chunk[r], local % (unsigned)a.G, local / (unsigned)a.G, sp);
}

__global__ void __launch_bounds__(kRhoThreads) k_rho64(RhoArgs a, int chunk) {
    __shared__ Rec64 sp[kRhoTile / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pass_base = blockIdx.y * 256;
    int ngroups, nsub;
    rho_split(a.P, pass_base, 1, ngroups, nsub);
    const int g = warp % ngroups, sub = warp / ngroups;
    const bool active = sub < nsub;
    const int l = pass_base + g * 32 + lane;
    const bool ok = active && l < a.P;
    const unsigned long long m0 = (unsigned long long)(long long)(ok ? a.m[3 * l] : 0);
    const unsigned long long m1 = (unsigned long long)(long long)(ok ? a.m[3 * l + 1] : 0);
    const unsigned long long m2 = (unsigned long long)(long long)(ok ? a.m[3 * l + 2] : 0);
    double re = 0.0, im = 0.0;
    const uint32_t begin = (uint32_t)blockIdx.x * (uint32_t)chunk;
    uint32_t end = begin + (uint32_t)chunk;
    if (end > a.N) end = a.N;
    const Rec64 *rec = (const Rec64 *)a.rec;
    for (uint32_t base = begin; base < end; base += kRhoTile / 2) {
        const int tn = (int)min((uint32_t)(kRhoTile / 2), end - base);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) sp[t] = rec[base + t];
        __syncthreads();
        if (!active) continue;
        for (int i = sub; i < tn; i += nsub) {
            const Rec64 r = sp[i];
            const unsigned long long th = m0 * r.s[0] + m1 * r.s[1] + m2 * r.s[2];
            const double f = (double)(long long)th * 5.421010862427522e-20;   // 2^-64
            double sn, cs;
            sincospi(2.0 * f, &sn, &cs);
            re += r.q * cs;
            im += r.q * sn;
        }
    }
    if (ok) a.partial[((size_t)blockIdx.x * 8 + sub) * a.P + l] = make_double2(re, im);
}

// ------------------------------------------------------------------ final reduction
struct GTab32 {
    int4 m;      // m_x, m_y, m_z, Im(rho) as float bits
    float4 f;    // coef k_x, coef k_y, coef k_z, Re(rho)
};
static_assert(sizeof(GTab32) == kGTab32Bytes, "gather table entry size");
struct GTab64 {
    int4 m;
    double ck[3];
    double re, im;
};

// rho, the U*_F term and the gather-table entry of mode l from its summed rho
template <int PREC>
__device__ __forceinline__ void rho_final_write(const RhoFinalArgs &a, int l, double re, double im) {
    a.rho[l] = make_double2(re, im);
    const double coef = a.coef[l];
    a.Ufar[l] = 0.5 * coef * (re * re + im * im);
    const int mx = a.m[3 * l], my = a.m[3 * l + 1], mz = a.m[3 * l + 2];
    const double kx = a.tpl[0] * mx, ky = a.tpl[1] * my, kz = a.tpl[2] * mz;
    if (PREC == 1) {
        GTab32 t;
        t.m = make_int4(mx, my, mz, __float_as_int((float)im));
        t.f = make_float4((float)(coef * kx), (float)(coef * ky), (float)(coef * kz), (float)re);
        ((GTab32 *)a.gtab)[l] = t;
    } else {
        GTab64 t;
        t.m = make_int4(mx, my, mz, 0);
        t.ck[0] = coef * kx; t.ck[1] = coef * ky; t.ck[2] = coef * kz;
        t.re = re; t.im = im;
        ((GTab64 *)a.gtab)[l] = t;
    }
}

// Block b sums modes 32b .. 32b+31: warp w adds the partials of blocks w, w+8, ... in
// order, then warp 0 adds the 8 warp sums in order (fixed, deterministic).  Writes rho,
// the gather table and u_l = coef_l |rho_l|^2 / 2 (summed by k_energy).
template <int PREC>
__device__ __forceinline__ void rho_final_body(const RhoFinalArgs &a, int ML, unsigned bx, bool bump,
                                               double2 (*sh)[32]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l = (int)bx * 32 + lane;
    double re = 0.0, im = 0.0;
    if (l < a.P) {
        const int pass_base = (l / (256 * ML)) * 256 * ML;
        int ngroups, nsub;
        rho_split(a.P, pass_base, ML, ngroups, nsub);
        // eight independent partial sums (blocks b0 + 8u of each stride of 64) keep eight
        // loads in flight; combined in a fixed order
        double r8[8], i8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r8[u] = i8[u] = 0.0;
        for (int b0 = warp; b0 < a.G; b0 += 64) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = b0 + 8 * u;
                if (b < a.G)
                    for (int s = 0; s < nsub; ++s) {
                        const double2 v = a.partial[((size_t)b * 8 + s) * a.P + l];
                        r8[u] += v.x;
                        i8[u] += v.y;
                    }
            }
        }
        re = ((r8[0] + r8[1]) + (r8[2] + r8[3])) + ((r8[4] + r8[5]) + (r8[6] + r8[7]));
        im = ((i8[0] + i8[1]) + (i8[2] + i8[3])) + ((i8[4] + i8[5]) + (i8[6] + i8[7]));
    }
    sh[warp][lane] = make_double2(re, im);
    __syncthreads();
    if (warp == 0 && l < a.P) {
        re = 0.0;
        im = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            re += sh[w][lane].x;
            im += sh[w][lane].y;
        }
        rho_final_write<PREC>(a, l, re, im);
    }
    if (bump && threadIdx.x == 0) {
        a.ctr->draw += 1ull;
        a.ctr->inject = 0;
    }
}

// rho_final_body with the eight warps' sums of each 32 modes in eight blocks: block
// (x, w) holds warp w's eight accumulators in its warps u = 0..7 (each the same sequence
// of additions), adds them in the same tree, and stores the group sum; the last of the
// eight blocks to arrive adds the group sums in order w = 0..7.  Every addition is the
// one-block form's, in its order, so rho is bit-identical; the FP64 additions of a
// mode's G nsub partials spread over eight SMs instead of one.
template <int PREC>
__device__ __forceinline__ void rho_final_split_body(const RhoFinalArgs &a, int ML, double2 (*sh)[32]) {
    __shared__ int last;
    const int u = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = (int)blockIdx.y;
    const int l = (int)blockIdx.x * 32 + lane;
    double re = 0.0, im = 0.0;
    if (l < a.P) {
        const int pass_base = (l / (256 * ML)) * 256 * ML;
        int ngroups, nsub;
        rho_split(a.P, pass_base, ML, ngroups, nsub);
        for (int b0 = w; b0 < a.G; b0 += 64) {
            const int b = b0 + 8 * u;
            if (b < a.G)
                for (int s = 0; s < nsub; ++s) {
                    const double2 v = a.partial[((size_t)b * 8 + s) * a.P + l];
                    re += v.x;
                    im += v.y;
                }
        }
    }
    sh[u][lane] = make_double2(re, im);
    __syncthreads();
    if (u == 0) {
        if (l < a.P) {
            re = ((sh[0][lane].x + sh[1][lane].x) + (sh[2][lane].x + sh[3][lane].x)) +
                 ((sh[4][lane].x + sh[5][lane].x) + (sh[6][lane].x + sh[7][lane].x));
            im = ((sh[0][lane].y + sh[1][lane].y) + (sh[2][lane].y + sh[3][lane].y)) +
                 ((sh[4][lane].y + sh[5][lane].y) + (sh[6][lane].y + sh[7][lane].y));
            a.wsum[(size_t)w * a.P + l] = make_double2(re, im);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) last = atomicAdd(&a.wdone[blockIdx.x], 1u) == 7u;
        __syncwarp();
        if (last) {
            __threadfence();
            if (l < a.P) {
                re = 0.0;
                im = 0.0;
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const double2 g = __ldcg(&a.wsum[(size_t)v * a.P + l]);
                    re += g.x;
                    im += g.y;
                }
                rho_final_write<PREC>(a, l, re, im);
            }
            if (lane == 0) a.wdone[blockIdx.x] = 0u;
            if (blockIdx.x == 0 && lane == 0 && !a.keep_draw) {
                a.ctr->draw += 1ull;
                a.ctr->inject = 0;
            }
        }
    }
}


template <int PREC>
__global__ void __launch_bounds__(256) k_rho_final(RhoFinalArgs a, int ML) {
    __shared__ double2 sh[8][32];
    rho_final_split_body<PREC>(a, ML, sh);
}

__global__ void __launch_bounds__(256) k_rho_final_batch(const RhoFinalArgs *args, const uint32_t *items, int R) {
    __shared__ double2 sh[8][32];
    const int r = item_system(items, R, blockIdx.x);
    // each system advances its own draw counter (first block of the system)
    rho_final_body<1>(args[r], 1, blockIdx.x - items[r], blockIdx.x == items[r], sh);
}

// ------------------------------------------------------------------ far gather + kick
// Closing part of a step for one particle: total force, optional half kick, kinetic
// energy, caller-order outputs.
template <int PREC>
__device__ __forceinline__ double finish_particle(const FarArgs &a, uint32_t p, const double *Ff) {
    const uint32_t N = a.stride;
    double Fn[3], Ft[3];
    if (PREC == 1) {
        const float *fn = (const float *)a.Fn;
        Fn[0] = fn[p]; Fn[1] = fn[N + p]; Fn[2] = fn[2 * (size_t)N + p];
    } else {
        const double *fn = (const double *)a.Fn;
        Fn[0] = fn[p]; Fn[1] = fn[N + p]; Fn[2] = fn[2 * (size_t)N + p];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Ft[d] = Fn[d] + Ff[d];
    if (PREC == 1) {
        float *F = (float *)a.F;
        F[p] = (float)Ft[0]; F[N + p] = (float)Ft[1]; F[2 * (size_t)N + p] = (float)Ft[2];
    } else {
        double *F = (double *)a.F;
        F[p] = Ft[0]; F[N + p] = Ft[1]; F[2 * (size_t)N + p] = Ft[2];
    }
    double v[3] = {a.st.vx[p], a.st.vy[p], a.st.vz[p]};
    const double invm = a.st.invm[p];
    if (a.integrate && a.ctr->fvalid) {
        const double hk = 0.5 * a.dt * invm;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] += hk * Ft[d];
        a.st.vx[p] = v[0]; a.st.vy[p] = v[1]; a.st.vz[p] = v[2];
    }
    const size_t u = 3 * (size_t)a.st.id[p];
    if (a.F_user) { a.F_user[u] = Ft[0]; a.F_user[u + 1] = Ft[1]; a.F_user[u + 2] = Ft[2]; }
    if (a.Fn_user) { a.Fn_user[u] = Fn[0]; a.Fn_user[u + 1] = Fn[1]; a.Fn_user[u + 2] = Fn[2]; }
    if (a.Ff_user) { a.Ff_user[u] = Ff[0]; a.Ff_user[u + 1] = Ff[1]; a.Ff_user[u + 2] = Ff[2]; }
    return 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / invm;
}

// FP32 build: the total force is formed in FP32 (the Kahan far sum rounded once, plus the
// FP32 near force); FP64 is kept for the velocity kick and the kinetic energy.
__device__ __forceinline__ double finish_particle32(const FarArgs &a, uint32_t p, const float *Ff) {
    const uint32_t N = a.stride;
    const float *fn = (const float *)a.Fn;
    const float Fn[3] = {fn[p], fn[N + p], fn[2 * (size_t)N + p]};
    float Ft[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) Ft[d] = Fn[d] + Ff[d];
    float *F = (float *)a.F;
    F[p] = Ft[0]; F[N + p] = Ft[1]; F[2 * (size_t)N + p] = Ft[2];
    double v[3] = {a.st.vx[p], a.st.vy[p], a.st.vz[p]};
    const double invm = a.st.invm[p];
    if (a.integrate && a.ctr->fvalid) {
        const double hk = 0.5 * a.dt * invm;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] += hk * (double)Ft[d];
        a.st.vx[p] = v[0]; a.st.vy[p] = v[1]; a.st.vz[p] = v[2];
    }
    const size_t u = 3 * (size_t)a.st.id[p];
    if (a.F_user) { a.F_user[u] = Ft[0]; a.F_user[u + 1] = Ft[1]; a.F_user[u + 2] = Ft[2]; }
    if (a.Fn_user) { a.Fn_user[u] = Fn[0]; a.Fn_user[u + 1] = Fn[1]; a.Fn_user[u + 2] = Fn[2]; }
    if (a.Ff_user) { a.Ff_user[u] = Ff[0]; a.Ff_user[u + 1] = Ff[1]; a.Ff_user[u + 2] = Ff[2]; }
    return 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / invm;
}

// FP32: two particles per thread (p and p + 256) share each mode's table entry.  The
// gather sums over modes whose phases are unrelated, so rounding of the phase scaling is
// incoherent here and the argument needs no half-turn reduction (unlike rho).
__device__ __forceinline__ void far32_body(const FarArgs &a, unsigned bx, GTab32 *tab, double *shK) {
    const uint32_t p0 = bx * (2 * kFarThreads) + threadIdx.x;
    const uint32_t p1 = p0 + kFarThreads;
    const bool v0 = p0 < a.N, v1 = p1 < a.N;
    const uint4 r0 = v0 ? ((const uint4 *)a.rec)[p0] : make_uint4(0, 0, 0, 0);
    const uint4 r1 = v1 ? ((const uint4 *)a.rec)[p1] : make_uint4(0, 0, 0, 0);
    float S0[3] = {0.f, 0.f, 0.f}, C0[3] = {0.f, 0.f, 0.f}, S1[3] = {0.f, 0.f, 0.f}, C1[3] = {0.f, 0.f, 0.f};
    for (int base = 0; base < a.P; base += kFarTile) {
        const int tn = min(kFarTile, a.P - base);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) tab[t] = ((const GTab32 *)a.gtab)[base + t];
        __syncthreads();
        const unsigned long long K2 = pk2(kTwoPiOver2p32, kTwoPiOver2p32);
        for (int l0 = 0; l0 < tn; l0 += 32) {
            const int l1 = min(tn, l0 + 32);
            // the two particles of the thread share each packed FP32x2 operation
            unsigned long long A[3] = {0ull, 0ull, 0ull};
            for (int l = l0; l < l1; ++l) {
                const GTab32 t = tab[l];
                const float im = __int_as_float(t.m.w), re = t.f.w;
                const uint32_t th0 = (uint32_t)t.m.x * r0.x + (uint32_t)t.m.y * r0.y + (uint32_t)t.m.z * r0.z;
                const uint32_t th1 = (uint32_t)t.m.x * r1.x + (uint32_t)t.m.y * r1.y + (uint32_t)t.m.z * r1.z;
                float x0, x1;
                upk2(mul2(pk2((float)(int)th0, (float)(int)th1), K2), x0, x1);
                float s0, c0, s1, c1;
                __sincosf(x0, &s0, &c0);
                __sincosf(x1, &s1, &c1);
                const unsigned long long g = fma2(pk2(c0, c1), pk2(im, im), mul2(pk2(s0, s1), pk2(-re, -re)));
                A[0] = fma2(pk2(t.f.x, t.f.x), g, A[0]);
                A[1] = fma2(pk2(t.f.y, t.f.y), g, A[1]);
                A[2] = fma2(pk2(t.f.z, t.f.z), g, A[2]);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float a0, a1;
                upk2(A[d], a0, a1);
                kahan_add(S0[d], C0[d], a0);
                kahan_add(S1[d], C1[d], a1);
            }
        }
    }
    double K = 0.0;
    if (v0) {
        float Ff[3];
        const float q = __uint_as_float(r0.w);
#pragma unroll
        for (int d = 0; d < 3; ++d) Ff[d] = -q * (S0[d] - C0[d]);
        K += finish_particle32(a, p0, Ff);
    }
    if (v1) {
        float Ff[3];
        const float q = __uint_as_float(r1.w);
#pragma unroll
        for (int d = 0; d < 3; ++d) Ff[d] = -q * (S1[d] - C1[d]);
        K += finish_particle32(a, p1, Ff);
    }
    const double tot = block_reduce_sum<double>(K, shK);
    if (threadIdx.x == 0) a.K_part[bx] = tot;
}

// 5 blocks per SM (51 registers) measured faster than 4 with more registers
__global__ void __launch_bounds__(kFarThreads, 5) k_far32(FarArgs a) {
    __shared__ double shK[kFarThreads];
    __shared__ __align__(16) GTab32 tab[kFarTile];
    far32_body(a, blockIdx.x, tab, shK);
}

__global__ void __launch_bounds__(kFarThreads) k_far_batch(const FarArgs *args, const uint32_t *items, int R) {
    __shared__ double shK[kFarThreads];
    __shared__ __align__(16) GTab32 tab[kFarTile];
    const int r = item_system(items, R, blockIdx.x);
    far32_body(args[r], blockIdx.x - items[r], tab, shK);
}

__global__ void __launch_bounds__(kFarThreads) k_far64(FarArgs a) {
    __shared__ double shK[kFarThreads];
    __shared__ __align__(16) GTab64 tab[kFarTile / 2];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < a.N;
    Rec64 ri;
    if (valid) ri = ((const Rec64 *)a.rec)[p];
    else { ri.s[0] = ri.s[1] = ri.s[2] = 0ull; ri.q = 0.0; }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int base = 0; base < a.P; base += kFarTile / 2) {
        const int tn = min(kFarTile / 2, a.P - base);
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) tab[t] = ((const GTab64 *)a.gtab)[base + t];
        __syncthreads();
        for (int l = 0; l < tn; ++l) {
            const GTab64 t = tab[l];
            const unsigned long long th = (unsigned long long)(long long)t.m.x * ri.s[0] +
                                          (unsigned long long)(long long)t.m.y * ri.s[1] +
                                          (unsigned long long)(long long)t.m.z * ri.s[2];
            const double f = (double)(long long)th * 5.421010862427522e-20;
            double sn, cs;
            sincospi(2.0 * f, &sn, &cs);
            const double gv = cs * t.im - sn * t.re;
            acc[0] += t.ck[0] * gv;
            acc[1] += t.ck[1] * gv;
            acc[2] += t.ck[2] * gv;
        }
    }
    double K = 0.0;
    if (valid) {
        double Ff[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) Ff[d] = -ri.q * acc[d];
        K = finish_particle<0>(a, p, Ff);
    }
    const double tot = block_reduce_sum<double>(K, shK);
    if (threadIdx.x == 0) a.K_part[blockIdx.x] = tot;
}

// Fixed-order strided sum of x[0 .. n-1] by this thread with eight independent partial
// sums (eight loads in flight).
__device__ __forceinline__ double strided_sum8(const double *x, int n) {
    double s8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] = 0.0;
    const int st = blockDim.x;
    for (int i0 = threadIdx.x; i0 < n; i0 += 8 * st) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * st;
            if (i < n) s8[u] += x[i];
        }
    }
    return ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
}

__device__ __forceinline__ void energy_body(const EnergyArgs &a, double *sh) {
    // fixed-order per-thread strides, then a fixed tree
    double U = block_reduce_sum<double>(strided_sum8(a.U_part, a.nU), sh);
    double K = block_reduce_sum<double>(strided_sum8(a.K_part, a.nK), sh);
    double uf = 0.0;
    for (int i = threadIdx.x; i < a.nUfar; i += blockDim.x) uf += a.Ufar[i];
    const double Ufs = block_reduce_sum<double>(uf, sh);
    if (threadIdx.x == 0) {
        const double Uf = Ufs + a.Ufar0;
        a.out[0] = U;
        a.out[1] = Uf;
        a.out[2] = a.Uself;
        a.out[3] = K;
        a.out[4] = U + Uf + a.Uself + K;
    }
}

// Sum over the warps of a 256-thread block of three values at once, in a fixed order
// (shuffle tree in each warp, then warp 0 over the 8 warp sums); one barrier.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double (*sh)[3]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) { sh[w][0] = a; sh[w][1] = b; sh[w][2] = c; }
    __syncthreads();
    if (w == 0) {
        a = lane < 8 ? sh[lane][0] : 0.0;
        b = lane < 8 ? sh[lane][1] : 0.0;
        c = lane < 8 ? sh[lane][2] : 0.0;
#pragma unroll
        for (int o = 4; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
    }
}

// FP64 runs at 2 operations per clock per SM here, so one block summing ~5e4 partials
// is FP64-bound; kEnergyBlocks (<= 32) blocks share the sums and the last one to arrive
// combines the per-block results with a fixed shuffle tree over the block index
// (deterministic whichever block is last).
__global__ void __launch_bounds__(256) k_energy(EnergyArgs a) {
    __shared__ double sh[8][3];
    __shared__ int last;
    const int E = gridDim.x, b = blockIdx.x;
    auto part = [&](const double *x, int n) {
        const int lo = (int)((long long)n * b / E), hi = (int)((long long)n * (b + 1) / E);
        return strided_sum8(x + lo, hi - lo);
    };
    double U = part(a.U_part, a.nU), K = part(a.K_part, a.nK), Uf = part(a.Ufar, a.nUfar);
    block_sum3(U, K, Uf, sh);
    if (threadIdx.x == 0) {
        a.scratch[b] = U;
        a.scratch[E + b] = K;
        a.scratch[2 * E + b] = Uf;
        __threadfence();
        last = atomicAdd(a.done, 1u) == (unsigned)(E - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        __threadfence();
        const volatile double *s = a.scratch;
        const int i = threadIdx.x;
        double Us = i < E ? s[i] : 0.0, Ks = i < E ? s[E + i] : 0.0, Ufs = i < E ? s[2 * E + i] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            Us += __shfl_xor_sync(0xffffffffu, Us, o);
            Ks += __shfl_xor_sync(0xffffffffu, Ks, o);
            Ufs += __shfl_xor_sync(0xffffffffu, Ufs, o);
        }
        if (i == 0) {
            const double Ut = Ufs + a.Ufar0;
            a.out[0] = Us;
            a.out[1] = Ut;
            a.out[2] = a.Uself;
            a.out[3] = Ks;
            a.out[4] = Us + Ut + a.Uself + Ks;
            *a.done = 0u;
        }
    }
}

// Close of one force evaluation of a single system: the forces are now valid, and a
// step that integrated counts (a pass that found the forces invalid only evaluated
// them).  The energy reduction (k_energy) runs only when the energies are read.
__global__ void k_close_eval(DevCounters *ctr, int advance_step) {
    if (advance_step && ctr->fvalid) ctr->step += 1ull;
    ctr->fvalid = 1;
}

// The same for the R systems of a batch (their counters are contiguous).
__global__ void __launch_bounds__(256) k_close_eval_batch(DevCounters *ctr, int R, int advance_step) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (advance_step && ctr[r].fvalid) ctr[r].step += 1ull;
    ctr[r].fvalid = 1;
}

__global__ void __launch_bounds__(1024) k_energy_batch(const EnergyArgs *args) {
    __shared__ double sh[1024];
    energy_body(args[blockIdx.x], sh);
}


// modes per lane: four above 256 modes, so that a particle's load and the loop overhead
// serve four phases.  With fewer mode groups per block the warps split the particles into
// more subsets, whose partial sums rho_final adds; that runs off the step's critical path,
// beside the near field.
int rho_ml(int P) { return P <= 256 ? 1 : 4; }

}  // namespace

int rho_blocks(int prec, uint32_t N, int P) {
    (void)prec; (void)P;
    // three blocks per SM: the structure factor shares the SMs with the cell list and the
    // near field (4 per SM measured 3% slower per step, 2 per SM 1%)
    int G = 152 * 3;
    int byN = (int)((N + 63) / 64);
    return G < byN ? G : (byN > 0 ? byN : 1);
}

void launch_rho(int prec, const RhoArgs &a, cudaStream_t st) {
    const int chunk = (int)((a.N + (uint32_t)a.G - 1) / (uint32_t)a.G);
    if (prec == 1) {
        const int ML = rho_ml(a.P);
        dim3 grid(a.G, (a.P + 256 * ML - 1) / (256 * ML));
        if (ML == 1) k_rho32<1><<<grid, kRhoThreads, 0, st>>>(a, chunk);
        else if (ML == 2) k_rho32<2><<<grid, kRhoThreads, 0, st>>>(a, chunk);
        else k_rho32<4><<<grid, kRhoThreads, 0, st>>>(a, chunk);
    } else {
        dim3 grid(a.G, (a.P + 255) / 256);
        k_rho64<<<grid, kRhoThreads, 0, st>>>(a, chunk);
    }
}

void launch_rho_final(int prec, const RhoFinalArgs &a, cudaStream_t st) {
    const dim3 grid((unsigned)((a.P + 31) / 32), 8);
    if (prec == 1) k_rho_final<1><<<grid, 256, 0, st>>>(a, rho_ml(a.P));
    else k_rho_final<0><<<grid, 256, 0, st>>>(a, 1);
}

int launch_far(int prec, const FarArgs &a, cudaStream_t st) {
    if (prec == 1) {
        const unsigned nb = blocks_for(a.N, 2 * kFarThreads);
        k_far32<<<nb, kFarThreads, 0, st>>>(a);
        return (int)nb;
    }
    const unsigned nb = blocks_for(a.N, kFarThreads);
    k_far64<<<nb, kFarThreads, 0, st>>>(a);
    return (int)nb;
}

void launch_close_eval(DevCounters *ctr, int advance_step, cudaStream_t st) { k_close_eval<<<1, 1, 0, st>>>(ctr, advance_step); }
void launch_close_eval_batch(DevCounters *ctr, int R, int advance_step, cudaStream_t st) {
    k_close_eval_batch<<<(R + 255) / 256, 256, 0, st>>>(ctr, R, advance_step);
}

static_assert(kEnergyBlocks <= 32, "k_energy combines the block sums in one warp");
void launch_energy(const EnergyArgs &a, cudaStream_t st) { k_energy<<<kEnergyBlocks, 256, 0, st>>>(a); }

uint32_t rho_batch_blocks(int G, int P) { return (uint32_t)G * (uint32_t)((P + 255) / 256); }
uint32_t rho_final_batch_blocks(int P) { return (uint32_t)((P + 31) / 32); }
uint32_t far_batch_blocks(uint32_t N) { return blocks_for(N, 2 * kFarThreads); }

void launch_rho_batch(const RhoArgs *args, const int *chunk, const uint32_t *items, int R, uint32_t nblocks,
                      cudaStream_t st) {
    k_rho_batch<<<nblocks, kRhoThreads, 0, st>>>(args, chunk, items, R);
}

void launch_rho_final_batch(const RhoFinalArgs *args, const uint32_t *items, int R, uint32_t nblocks,
                            cudaStream_t st) {
    k_rho_final_batch<<<nblocks, 256, 0, st>>>(args, items, R);
}

void launch_far_batch(const FarArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st) {
    k_far_batch<<<nblocks, kFarThreads, 0, st>>>(args, items, R);
}

void launch_energy_batch(const EnergyArgs *args, int R, cudaStream_t st) { k_energy_batch<<<R, 1024, 0, st>>>(args); }

}  // namespace rbsog
