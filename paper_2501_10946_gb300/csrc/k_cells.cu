// Cell list by stable counting sort, fused with the first half of the integrator.
//
// Per step (Algorithm 2: integrate, then rebuild the neighbour structure of Eq. 55):
//   k_bin          v += F dt/2m, drift (BAOAB: half drift, Ornstein-Uhlenbeck, half drift),
//                  wrap into [0, L), fixed point s = floor(frac(r (1/L)) 2^32) (2^64 in FP64),
//                  cell c_a = floor(s_a n_a / 2^32), atomic count -> slot within the cell
//   k_tile_sums    per 4096-cell tile population
//   k_scan_tiles   exclusive scan -> cell_start; clears the counts for the next build
//   k_scatter      key = (particle id, previous position) at cell_start + slot
//   k_gather       each key's rank among its cell's keys (by particle id) gives its place:
//                  the order the atomics produced is discarded, so the result is
//                  deterministic; state and 16/32-byte particle records move there
#include "common.cuh"
#include "devutil.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace rbsog {

namespace {

// FP64 division is slow on this part, so both use the double reciprocal 1/L:
__device__ __forceinline__ double wrap_coord(double r, double L, double invL) {
    // r - L floor(r (1/L)), then into [0, L): IEEE operations without contraction
    double w = __dsub_rn(r, __dmul_rn(L, floor(__dmul_rn(r, invL))));
    if (w < 0.0) w = __dadd_rn(w, L);
    if (w >= L) w = __dsub_rn(w, L);
    return w;
}

// wrap_coord for a position that left [0, L) by less than one box length, with the FP64
// pipe (1/72 of the FP32 rate on this part) used only for the rare correction: the range
// tests compare the IEEE bit patterns as integers (ordered like the values for w >= 0).
// For r in [-L, 2L) the result equals wrap_coord(r) bit for bit; outside, wrap_coord.
__device__ __forceinline__ double wrap_near(double r, double L, double invL) {
    const long long bL = __double_as_longlong(L);
    long long b = __double_as_longlong(r);
    if (b >= 0 && b < bL) return r;                       // already in [0, L) (+0 included)
    double w = r;
    if (b < 0) {                                          // negative (or -0)
        w = __dadd_rn(r, L);
        if (__double_as_longlong(w) < 0) return wrap_coord(r, L, invL);   // below -L
    }
    b = __double_as_longlong(w);
    if (b >= bL) {
        w = __dsub_rn(w, L);
        if (__double_as_longlong(w) >= bL) return wrap_coord(r, L, invL);  // 2L or beyond
    }
    return w;
}

// IEEE 754 conversions on the integer pipe.  On this part the FP64 unit (1/64 of the FP32
// rate) also executes the float <-> double and double -> integer conversion
// instructions, so the FP32 build's integrator, which would otherwise spend most of its
// time there, assembles the results from the fields of the formats instead.  Each
// function returns exactly what the conversion instruction returns; the rare operands
// outside the handled range (subnormal, infinite, NaN) take the instruction itself.

// float -> double (exact): sign, exponent rebiased from 127 to 1023, fraction widened.
__device__ __forceinline__ double f2d_int(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e - 1u < 254u) {                                     // normal
        const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu);
        return __hiloint2double((int)hi, (int)(b << 29));
    }
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)b, 0);   // +-0
    return (double)x;
}

// double -> float, round to nearest even: keep 23 of the 52 fraction bits and round on
// the 29 dropped ones; a carry out of the fraction moves into the exponent, which is the
// correctly rounded result (up to the largest finite float and beyond it to infinity).
__device__ __forceinline__ float d2f_int(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t E = (hi >> 20) & 0x7ffu;
    if (E - 897u < 254u) {                                   // a normal float before rounding
        const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;
        uint32_t v = ((E - 896u) << 23) | mant;
        v += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
        return __uint_as_float((hi & 0x80000000u) | v);
    }
    if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi);   // +-0
    return __double2float_rn(x);
}

// The low 32 bits of the truncation of x in [0, 2^33) (what the 64-bit unsigned
// round-toward-zero conversion gives there): 1.f x 2^e shifted down by 52 - e.
__device__ __forceinline__ uint32_t trunc_lo32(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t E = hi >> 20;                            // sign bit included: x >= 0 here
    if (E < 1023u) return 0u;                                // [0, 1), +0
    if (E > 1055u) return (uint32_t)__double2ull_rz(x);      // 2^33 and above, inf, NaN, x < 0
    const unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
    return (uint32_t)(m >> (52u - (E - 1023u)));
}

// Langevin noise words of particle `id`: Philox key = seed, counter = (id, 0x40000000 + j, n),
// n = force evaluations (k-draws) so far.  Setting a state does not reset n, so a loop
// that uploads the state before every step still draws fresh noise.
__device__ __forceinline__ void noise_words(const BinArgs &a, uint32_t id, U4 &w0, U4 &w1) {
    const unsigned long long n = a.ctr->draw;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    w0 = philox10(id, 0x40000000u, (uint32_t)n, (uint32_t)(n >> 32), k0, k1);
    w1 = philox10(id, 0x40000001u, (uint32_t)n, (uint32_t)(n >> 32), k0, k1);
}

// The inputs of one particle's update, all loaded before any of it is computed
struct BinIn {
    double r[3], v[3], invm, q;
    uint32_t id;
    int integrate;
    float f32[3];
    double f64[3];
};

template <int PREC>
__device__ __forceinline__ void bin_load(const BinArgs &a, uint32_t k, BinIn &b) {
    const uint32_t N = a.stride;
    b.r[0] = a.in.rx[k]; b.r[1] = a.in.ry[k]; b.r[2] = a.in.rz[k];
    b.v[0] = a.in.vx[k]; b.v[1] = a.in.vy[k]; b.v[2] = a.in.vz[k];
    b.invm = a.in.invm[k];
    b.q = a.in.q[k];
    b.id = a.in.id[k];
    // a system whose forces were never evaluated (fvalid = 0) only rebuilds its cells
    b.integrate = a.ctr->fvalid ? a.integrate : 0;
    if (b.integrate) {
        if (PREC == 1) {
            const float *Ff = (const float *)a.F;
#pragma unroll
            for (int d = 0; d < 3; ++d) b.f32[d] = Ff[(size_t)d * N + k];
        } else {
            const double *Fd = (const double *)a.F;
#pragma unroll
            for (int d = 0; d < 3; ++d) b.f64[d] = Fd[(size_t)d * N + k];
        }
    }
}

// The update of particle k: returns its cell and sets ke to its kinetic energy
// m |v|^2 / 2 after the update when a.K_part is set (else 0).
template <int PREC>
__device__ __forceinline__ uint32_t bin_update(const BinArgs &a, uint32_t k, const BinIn &b, double &ke) {
    double r[3] = {b.r[0], b.r[1], b.r[2]};
    double v[3] = {b.v[0], b.v[1], b.v[2]};
    const double invm = b.invm;
    const uint32_t id = b.id;
    const int integrate = b.integrate;
    if (PREC == 1 && integrate) {
        // FP32 build: kick, drift increments and the O step in FP32 (the forces carry FP32
        // errors already); the positions add those increments in FP64.
        const float im = d2f_int(invm);
        float vf[3] = {d2f_int(v[0]), d2f_int(v[1]), d2f_int(v[2])};
        const float hk = a.hdt_f * im;
#pragma unroll
        for (int d = 0; d < 3; ++d) vf[d] = fmaf(hk, b.f32[d], vf[d]);
        float dr[3];
        if (integrate == 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) dr[d] = a.dt_f * vf[d];
        } else {
            // B A O A of BAOAB; Box-Muller pairs from the 24 leading bits of the noise words
            // (FP64 transcendentals would cost more than the rest of this kernel)
            U4 w0, w1;
            noise_words(a, id, w0, w1);
            const float u1 = (float)(w0.x >> 8) * 5.9604645e-08f, u2 = (float)(w0.z >> 8) * 5.9604645e-08f;
            const float u3 = (float)(w1.x >> 8) * 5.9604645e-08f, u4 = (float)(w1.z >> 8) * 5.9604645e-08f;
            const float rad = sqrtf(-2.0f * logf(1.0f - u1)), rad3 = sqrtf(-2.0f * logf(1.0f - u3));
            float s2, c2;
            sincospif(2.0f * u2, &s2, &c2);
            const float xi[3] = {rad * c2, rad * s2, rad3 * cospif(2.0f * u4)};
            const float sig = sqrtf(a.okT_f * im);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float d1 = a.hdt_f * vf[d];
                vf[d] = fmaf(a.c1_f, vf[d], sig * xi[d]);
                dr[d] = fmaf(a.hdt_f, vf[d], d1);
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r[d] = __dadd_rn(r[d], f2d_int(dr[d]));
            v[d] = f2d_int(vf[d]);
        }
    } else if (integrate) {
        // FP64 build
        const double F[3] = {b.f64[0], b.f64[1], b.f64[2]};
        const double hk = 0.5 * a.dt * invm;
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] += hk * F[d];
        if (integrate == 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) r[d] += a.dt * v[d];
        } else {
            // B A O A of BAOAB
            U4 w0, w1;
            noise_words(a, id, w0, w1);
            double xi[3];
            double u1 = u53_of(w0.x, w0.y), u2 = u53_of(w0.z, w0.w);
            double rad = sqrt(-2.0 * log(1.0 - u1));
            double s2, c2;
            sincospi(2.0 * u2, &s2, &c2);
            double u3 = u53_of(w1.x, w1.y), u4 = u53_of(w1.z, w1.w);
            double rad3 = sqrt(-2.0 * log(1.0 - u3));
            xi[0] = rad * c2; xi[1] = rad * s2; xi[2] = rad3 * cospi(2.0 * u4);
            // noise amplitude sqrt((1 - c1^2) kT / m)
            const double sig = sqrt((1.0 - a.c1 * a.c1) * a.kT * invm);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                r[d] += 0.5 * a.dt * v[d];
                v[d] = a.c1 * v[d] + sig * xi[d];
                r[d] += 0.5 * a.dt * v[d];
            }
        }
    }
    uint32_t cc[3];
    uint32_t s32v[3];
    unsigned long long s64v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r[d] = wrap_near(r[d], a.box.L[d], a.box.invL[d]);
        // r in [0, L): u = r (1/L) is in [0, 1], frac(u) = u except u = 1 (frac 0), and
        // u 2^32 = r (2^32/L) exactly (a power-of-two scaling commutes with rounding), so
        // s = floor(frac(r (1/L)) 2^32) takes one multiply and one conversion
        uint32_t s32;
        if (PREC == 1) {
            // u = 1 gives 2^32, whose low 32 bits are 0
            s32 = trunc_lo32(__dmul_rn(r[d], a.box.invL32[d]));
            s32v[d] = s32;
        } else {
            const double u = __dmul_rn(r[d], a.box.invL[d]);
            const unsigned long long s64 =
                __double_as_longlong(u) >= 0x3ff0000000000000LL ? 0ull : __double2ull_rz(u * 18446744073709551616.0);
            s64v[d] = s64;
            s32 = (uint32_t)(s64 >> 32);
        }
        cc[d] = (uint32_t)(((unsigned long long)s32 * (unsigned long long)a.box.nc[d]) >> 32);
    }
    a.out.rx[k] = r[0]; a.out.ry[k] = r[1]; a.out.rz[k] = r[2];
    a.out.vx[k] = v[0]; a.out.vy[k] = v[1]; a.out.vz[k] = v[2];
    a.out.invm[k] = invm;
    const double q = b.q;
    a.out.q[k] = q;
    // the particle record, at this position for the gather (which moves it into the cell
    // order) and at the particle's id for the structure factor: the order of the rho sums
    // then depends on the state alone, not on how the particles were stored before
    if (PREC == 1) {
        const uint4 rw = make_uint4(s32v[0], s32v[1], s32v[2], __float_as_uint(d2f_int(q)));
        ((uint4 *)a.rec_w)[k] = rw;
        ((uint4 *)a.rec_id)[id] = rw;
    } else {
        Rec64 rw;
        rw.s[0] = s64v[0]; rw.s[1] = s64v[1]; rw.s[2] = s64v[2];
        rw.q = q;
        ((Rec64 *)a.rec_w)[k] = rw;
        ((Rec64 *)a.rec_id)[id] = rw;
    }
    a.out.id[k] = id;
    ke = a.K_part ? 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / invm : 0.0;
    return a.cell_base + cc[0] + (uint32_t)a.box.nc[0] * (cc[1] + (uint32_t)a.box.nc[1] * cc[2]);
}

// One particle: update, then its slot in the cell from the cell's counter.  Returns the
// kinetic energy (0 unless a.K_part is set).
template <int PREC>
__device__ __forceinline__ double bin_body(const BinArgs &a, uint32_t k) {
    BinIn b;
    bin_load<PREC>(a, k, b);
    double ke;
    const uint32_t c = bin_update<PREC>(a, k, b, ke);
    a.cell[k] = c;
    a.slot[k] = atomicAdd(&a.count[c], 1u);
    return ke;
}

// Two FP32-build particles (of one system or two) in one thread, for a grid that runs few
// threads per SM: both loads before either update, both counter increments before either
// slot store.
__device__ __forceinline__ void bin_two(const BinArgs &a0, uint32_t k0, const BinArgs &a1, uint32_t k1) {
    BinIn b0, b1;
    bin_load<1>(a0, k0, b0);
    bin_load<1>(a1, k1, b1);
    double ke;
    const uint32_t c0 = bin_update<1>(a0, k0, b0, ke);
    const uint32_t c1 = bin_update<1>(a1, k1, b1, ke);
    const uint32_t s0 = atomicAdd(&a0.count[c0], 1u);
    const uint32_t s1 = atomicAdd(&a1.count[c1], 1u);
    a0.cell[k0] = c0;
    a0.slot[k0] = s0;
    a1.cell[k1] = c1;
    a1.slot[k1] = s1;
}

template <int PREC>
__global__ void __launch_bounds__(256) k_bin(BinArgs a) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (k < a.N) ke = bin_body<PREC>(a, k);
    if (a.K_part) {
        // per-block kinetic energy in a fixed order (warp shuffles, then the 8 warp sums)
        __shared__ double wsum[8];
#pragma unroll
        for (int o = 16; o; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = ke;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += wsum[w];
            a.K_part[blockIdx.x] = t;
        }
    }
}


__global__ void __launch_bounds__(256) k_bin_batch(const BinArgs *args, const uint32_t *items, int R) {
    const int r = item_system(items, R, blockIdx.x);
    const BinArgs &a = args[r];
    const uint32_t k = (blockIdx.x - items[r]) * blockDim.x + threadIdx.x;
    if (k < a.N) bin_body<1>(a, k);
}

__device__ __forceinline__ uint32_t block_sum_1024(uint32_t v, uint32_t *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    uint32_t t = (threadIdx.x < 32) ? sh[threadIdx.x] : 0u;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    uint32_t out = sh[32];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(1024) k_tile_sums(const uint32_t *count, int ncell, uint32_t *tile_sums) {
    __shared__ uint32_t sh[33];
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (base + j < ncell) s += count[base + j];
    s = block_sum_1024(s, sh);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t *count, int ncell, const uint32_t *tile_sums,
                                                     uint32_t *cell_start, uint32_t N) {
    __shared__ uint32_t sh[33];
    __shared__ uint32_t wsum[32];
    // population of the preceding tiles
    uint32_t pre = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) pre += tile_sums[b];
    pre = block_sum_1024(pre, sh);
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    uint32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) c[j] = (base + j < ncell) ? count[base + j] : 0u;
    uint32_t tot = c[0] + c[1] + c[2] + c[3];
    // inclusive warp scan of the thread totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = wsum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - w;   // exclusive
    }
    __syncthreads();
    uint32_t run = pre + wsum[wid] + inc - tot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < ncell) {
            cell_start[base + j] = run;
            count[base + j] = 0u;
        }
        run += c[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) cell_start[ncell] = N;
}

__device__ __forceinline__ void scatter_one(const uint32_t *cell, const uint32_t *slot, const uint32_t *cell_start,
                                            const uint32_t *id, unsigned long long *keys, uint32_t k) {
    keys[cell_start[cell[k]] + slot[k]] = ((unsigned long long)id[k] << 32) | (unsigned long long)k;
}

// The two scan passes for a block of 256 threads (the persistent batched step): tile t
// of kScanTile cells, 16 cells per thread.  Same results as k_tile_sums / k_scan_tiles.
constexpr int kScanPer256 = kScanTile / 256;

__device__ __forceinline__ uint32_t block_sum_256u(uint32_t v, uint32_t *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ void tile_sum_256(const uint32_t *count, int ncell, uint32_t *tile_sums, int tile,
                                             uint32_t *sh) {
    const int base = tile * kScanTile + threadIdx.x * kScanPer256;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer256; ++j)
        if (base + j < ncell) s += count[base + j];
    s = block_sum_256u(s, sh);
    if (threadIdx.x == 0) tile_sums[tile] = s;
}

__device__ __forceinline__ void scan_tile_256(uint32_t *count, int ncell, const uint32_t *tile_sums,
                                              uint32_t *cell_start, uint32_t N, int tile, int ntiles, uint32_t *sh) {
    uint32_t pre = 0;
    for (int b = threadIdx.x; b < tile; b += 256) pre += tile_sums[b];
    pre = block_sum_256u(pre, sh);
    const int base = tile * kScanTile + threadIdx.x * kScanPer256;
    uint32_t c[kScanPer256];
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < kScanPer256; ++j) {
        c[j] = (base + j < ncell) ? count[base + j] : 0u;
        tot += c[j];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) sh[8 + wid] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += sh[8 + w];
    uint32_t run = pre + wpre + inc - tot;
#pragma unroll
    for (int j = 0; j < kScanPer256; ++j) {
        if (base + j < ncell) {
            cell_start[base + j] = run;
            count[base + j] = 0u;
        }
        run += c[j];
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) cell_start[ncell] = N;
}

__global__ void __launch_bounds__(256) k_scatter(const uint32_t *cell, const uint32_t *slot,
                                                 const uint32_t *cell_start, const uint32_t *id, uint32_t N,
                                                 unsigned long long *keys) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    scatter_one(cell, slot, cell_start, id, keys, k);
}

// Thread i takes the key at scattered position i of its cell [lo, hi) and moves particle
// src = low word of the key to lo + (number of the cell's keys below it).  Ids are unique,
// so the ranks of a cell are a permutation of 0 .. n-1: particles in ascending id order,
// as a stable sort by id would leave them.  A cell above kMaxCellOcc keeps the scatter
// order and sets kErrCellOverflow (in the counter of the system that owns the cell when
// c_off is given).  The particle's state and record are loaded as soon as src is known,
// so their loads overlap the cell lookups and the rank count.
template <int PREC> struct RecOf { using T = uint4; };
template <> struct RecOf<0> { using T = Rec64; };

template <int PREC>
struct GatherVals {
    double rx, ry, rz, vx, vy, vz, invm, q;
    uint32_t id;
    typename RecOf<PREC>::T rec;
};

template <int PREC>
__device__ __forceinline__ void gather_load(const GatherArgs &g, uint32_t src, GatherVals<PREC> &v) {
    v.rx = g.in.rx[src]; v.ry = g.in.ry[src]; v.rz = g.in.rz[src];
    v.vx = g.in.vx[src]; v.vy = g.in.vy[src]; v.vz = g.in.vz[src];
    v.invm = g.in.invm[src];
    v.q = g.in.q[src];
    v.id = g.in.id[src];
    v.rec = ((const typename RecOf<PREC>::T *)g.rec_w)[src];
}

template <int PREC>
__device__ __forceinline__ void gather_store(const GatherArgs &g, uint32_t p, const GatherVals<PREC> &v) {
    g.out.rx[p] = v.rx; g.out.ry[p] = v.ry; g.out.rz[p] = v.rz;
    g.out.vx[p] = v.vx; g.out.vy[p] = v.vy; g.out.vz[p] = v.vz;
    g.out.invm[p] = v.invm;
    g.out.q[p] = v.q;
    g.out.id[p] = v.id;
    ((typename RecOf<PREC>::T *)g.rec)[p] = v.rec;
}

// keys[j] < key for j = t0 .. t0 + 3 inside [lo, hi) (a key past hi counts as none)
__device__ __forceinline__ uint32_t count_below4(const unsigned long long *keys, uint32_t j, uint32_t hi,
                                                 unsigned long long key) {
    const unsigned long long k0 = j < hi ? keys[j] : ~0ull;
    const unsigned long long k1 = j + 1 < hi ? keys[j + 1] : ~0ull;
    const unsigned long long k2 = j + 2 < hi ? keys[j + 2] : ~0ull;
    const unsigned long long k3 = j + 3 < hi ? keys[j + 3] : ~0ull;
    return (uint32_t)(k0 < key) + (uint32_t)(k1 < key) + (uint32_t)(k2 < key) + (uint32_t)(k3 < key);
}

// Place of key i in the new order (i itself for an overflowing cell)
__device__ __forceinline__ uint32_t gather_place(const GatherArgs &g, uint32_t i, unsigned long long key,
                                                 uint32_t c, uint32_t lo, uint32_t hi) {
    if (hi - lo <= (uint32_t)kMaxCellOcc) {
        uint32_t p = lo;
        for (uint32_t j = lo; j < hi; j += 4) p += count_below4(g.keys, j, hi, key);
        return p;
    }
    if (i == lo) {
        const int r = g.c_off ? item_system(g.c_off, g.R, c) : 0;
        atomicOr(&g.ctr[r].err, kErrCellOverflow);
    }
    return i;
}

template <int PREC>
__device__ __forceinline__ void gather_one(const GatherArgs &g, uint32_t i) {
    const unsigned long long key = g.keys[i];
    const uint32_t src = (uint32_t)key;
    const uint32_t c = g.cell[src];
    GatherVals<PREC> v;
    gather_load<PREC>(g, src, v);
    const uint32_t lo = g.cell_start[c], hi = g.cell_start[c + 1];
    gather_store<PREC>(g, gather_place(g, i, key, c, lo, hi), v);
}

// Keys i0 and i1 (FP32 records) in one thread, each lookup of the two in flight together:
// for a grid that runs few threads per SM.
__device__ __forceinline__ void gather_two(const GatherArgs &g, uint32_t i0, uint32_t i1) {
    const unsigned long long key0 = g.keys[i0], key1 = g.keys[i1];
    const uint32_t src0 = (uint32_t)key0, src1 = (uint32_t)key1;
    const uint32_t c0 = g.cell[src0], c1 = g.cell[src1];
    GatherVals<1> v0, v1;
    gather_load<1>(g, src0, v0);
    gather_load<1>(g, src1, v1);
    const uint32_t lo0 = g.cell_start[c0], hi0 = g.cell_start[c0 + 1];
    const uint32_t lo1 = g.cell_start[c1], hi1 = g.cell_start[c1 + 1];
    uint32_t p0 = i0, p1 = i1;
    const bool r0 = hi0 - lo0 <= (uint32_t)kMaxCellOcc, r1 = hi1 - lo1 <= (uint32_t)kMaxCellOcc;
    if (r0 && r1) {
        p0 = lo0;
        p1 = lo1;
        const uint32_t n = max(hi0 - lo0, hi1 - lo1);
        for (uint32_t t = 0; t < n; t += 4) {
            p0 += count_below4(g.keys, lo0 + t, hi0, key0);
            p1 += count_below4(g.keys, lo1 + t, hi1, key1);
        }
    } else {
        p0 = gather_place(g, i0, key0, c0, lo0, hi0);
        p1 = gather_place(g, i1, key1, c1, lo1, hi1);
    }
    gather_store<1>(g, p0, v0);
    gather_store<1>(g, p1, v1);
}

template <int PREC>
__global__ void __launch_bounds__(256) k_gather(GatherArgs g) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.N) gather_one<PREC>(g, i);
}

__device__ __forceinline__ void set_state_body(const double *r, const double *v, const double *q_user,
                                               const double *m_user, const State &rest, const Box &box, uint32_t k) {
    rest.rx[k] = wrap_coord(r[3 * (size_t)k], box.L[0], box.invL[0]);
    rest.ry[k] = wrap_coord(r[3 * (size_t)k + 1], box.L[1], box.invL[1]);
    rest.rz[k] = wrap_coord(r[3 * (size_t)k + 2], box.L[2], box.invL[2]);
    rest.vx[k] = v ? v[3 * (size_t)k] : 0.0;
    rest.vy[k] = v ? v[3 * (size_t)k + 1] : 0.0;
    rest.vz[k] = v ? v[3 * (size_t)k + 2] : 0.0;
    rest.invm[k] = 1.0 / m_user[k];
    rest.q[k] = q_user[k];
    rest.id[k] = k;
}

// Caller rows [N][3] in and out of one context, 256 caller indices per block: the block's
// 768 values of an array move between the caller's buffer and shared memory in order (one
// lane per consecutive value), so a caller buffer in pinned host memory, read or written
// by the kernel through its mapped address, is moved in whole lines over the host link.
constexpr int kRowBlock = 256;

template <typename T>
__device__ __forceinline__ void rows_in(const T *src, uint32_t base, uint32_t n, T *sh) {
    const size_t o = 3 * (size_t)base;
    for (uint32_t i = threadIdx.x; i < 3 * n; i += kRowBlock) sh[i] = src[o + i];
}

template <typename T>
__device__ __forceinline__ void rows_out(const T *sh, uint32_t base, uint32_t n, T *dst) {
    const size_t o = 3 * (size_t)base;
    for (uint32_t i = threadIdx.x; i < 3 * n; i += kRowBlock) dst[o + i] = sh[i];
}

__device__ __forceinline__ float conv_to_f(double x) { return d2f_int(x); }
__device__ __forceinline__ float conv_to_f(float x) { return x; }
__device__ __forceinline__ double conv_to_d(float x) { return f2d_int(x); }
__device__ __forceinline__ double conv_to_d(double x) { return x; }
template <typename To, typename Ti> __device__ __forceinline__ To conv(Ti x);
template <> __device__ __forceinline__ float conv<float, double>(double x) { return conv_to_f(x); }
template <> __device__ __forceinline__ float conv<float, float>(float x) { return x; }
template <> __device__ __forceinline__ double conv<double, float>(float x) { return conv_to_d(x); }
template <> __device__ __forceinline__ double conv<double, double>(double x) { return x; }

// A state upload: the particles take the caller's order (id = caller index), positions
// wrapped into [0, L) (wrap_near: the same values as wrap_coord), 1/m from the stored
// inverse masses.
__global__ void __launch_bounds__(kRowBlock) k_set_state(const double *r, const double *v, const double *q_user,
                                                         const double *invm_user, State rest, uint32_t N, Box box) {
    __shared__ double sr[3 * kRowBlock], sv[3 * kRowBlock];
    const uint32_t base = blockIdx.x * kRowBlock;
    const uint32_t n = min((uint32_t)kRowBlock, N - base);
    rows_in(r, base, n, sr);
    if (v) rows_in(v, base, n, sv);
    __syncthreads();
    const uint32_t t = threadIdx.x;
    if (t >= n) return;
    const uint32_t k = base + t;
    rest.rx[k] = wrap_near(sr[3 * t], box.L[0], box.invL[0]);
    rest.ry[k] = wrap_near(sr[3 * t + 1], box.L[1], box.invL[1]);
    rest.rz[k] = wrap_near(sr[3 * t + 2], box.L[2], box.invL[2]);
    rest.vx[k] = v ? sv[3 * t] : 0.0;
    rest.vy[k] = v ? sv[3 * t + 1] : 0.0;
    rest.vz[k] = v ? sv[3 * t + 2] : 0.0;
    rest.invm[k] = invm_user[k];
    rest.q[k] = q_user[k];
    rest.id[k] = k;
}

// New positions and velocities for a particle already resident at position k of the rest
// buffer: it keeps its place, charge and mass; caller index = its id.
__device__ __forceinline__ void set_state_inplace(const double *r, const double *v, const State &rest, const Box &box,
                                                  uint32_t k) {
    const size_t i = 3 * (size_t)rest.id[k];
    rest.rx[k] = wrap_coord(r[i], box.L[0], box.invL[0]);
    rest.ry[k] = wrap_coord(r[i + 1], box.L[1], box.invL[1]);
    rest.rz[k] = wrap_coord(r[i + 2], box.L[2], box.invL[2]);
    rest.vx[k] = v ? v[i] : 0.0;
    rest.vy[k] = v ? v[i + 1] : 0.0;
    rest.vz[k] = v ? v[i + 2] : 0.0;
}

// Batched systems: the caller's arrays hold system r's particles at p_off .. p_off + N - 1.
// With q_user/m_user the system is (re)initialised in caller order; without, its particles
// keep their current places, charges and masses.
__global__ void __launch_bounds__(256) k_set_state_batch(const SysStateArgs *args, const uint32_t *items, int R,
                                                         const double *r, const double *v) {
    const int sys = item_system(items, R, blockIdx.x);
    const SysStateArgs &a = args[sys];
    const uint32_t k = (blockIdx.x - items[sys]) * blockDim.x + threadIdx.x;
    if (k >= a.N) return;
    const double *rr = r + 3 * (size_t)a.p_off, *vv = v ? v + 3 * (size_t)a.p_off : nullptr;
    if (a.q_user) set_state_body(rr, vv, a.q_user, a.m_user, a.rest, a.box, k);
    else set_state_inplace(rr, vv, a.rest, a.box, k);
}

__global__ void k_reset_counters(DevCounters *ctr) {
    ctr->step = 0;
    ctr->err = 0;
    ctr->fvalid = 0;
}

__global__ void k_reset_counters_n(DevCounters *ctr, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        ctr[i].step = 0;
        ctr[i].err = 0;
        ctr[i].fvalid = 0;
    }
}

__global__ void __launch_bounds__(256) k_relayout(State from, State to, const float *F_from, float *F_to,
                                                  uint32_t stride, const uint32_t *old_off, const uint32_t *new_off,
                                                  int R, uint32_t Nnew) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Nnew) return;
    const int r = item_system(new_off, R, p);
    const uint32_t q = old_off[r] + (p - new_off[r]);
    to.rx[p] = from.rx[q]; to.ry[p] = from.ry[q]; to.rz[p] = from.rz[q];
    to.vx[p] = from.vx[q]; to.vy[p] = from.vy[q]; to.vz[p] = from.vz[q];
    to.invm[p] = from.invm[q];
    to.q[p] = from.q[q];
    to.id[p] = from.id[q];
    F_to[p] = F_from[q];
    F_to[stride + p] = F_from[stride + q];
    F_to[2 * (size_t)stride + p] = F_from[2 * (size_t)stride + q];
}

__device__ __forceinline__ void get_state_body(const State &rest, size_t base, uint32_t k, double *r_out,
                                               double *v_out) {
    const size_t u = 3 * (base + (size_t)rest.id[k]);
    if (r_out) { r_out[u] = rest.rx[k]; r_out[u + 1] = rest.ry[k]; r_out[u + 2] = rest.rz[k]; }
    if (v_out) { v_out[u] = rest.vx[k]; v_out[u + 1] = rest.vy[k]; v_out[u + 2] = rest.vz[k]; }
}

// Forces at an uploaded state: caller rows [N][3] into the SoA force buffer of the rest
// order, which is the caller order right after a state upload; marks the forces valid
// (after the counter reset of the upload, on the same stream).  FP64 values into the FP32
// build's buffer are rounded to nearest; FP32 into FP32 are copied.
template <typename Ti, typename To>
__global__ void __launch_bounds__(kRowBlock) k_set_forces(const Ti *F_in, To *F, uint32_t N, DevCounters *ctr) {
    __shared__ Ti sf[3 * kRowBlock];
    const uint32_t base = blockIdx.x * kRowBlock;
    if (base == 0 && threadIdx.x == 0) ctr->fvalid = 1;
    if (base >= N) return;
    const uint32_t n = min((uint32_t)kRowBlock, N - base);
    rows_in(F_in, base, n, sf);
    __syncthreads();
    const uint32_t t = threadIdx.x;
    if (t >= n) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) F[(size_t)d * N + base + t] = conv<To>(sf[3 * t + d]);
}

// Place in the rest order of each caller index: the inverse of rest.id.
__global__ void __launch_bounds__(256) k_rest_pos(const uint32_t *id, uint32_t N, uint32_t *pos) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) pos[id[k]] = k;
}

// The state in caller rows: thread t of the block takes caller index base + t from its
// place in the rest order.
__global__ void __launch_bounds__(kRowBlock) k_get_state(State rest, const uint32_t *pos, uint32_t N, double *r_out,
                                                         double *v_out) {
    __shared__ double sr[3 * kRowBlock], sv[3 * kRowBlock];
    const uint32_t base = blockIdx.x * kRowBlock;
    const uint32_t n = min((uint32_t)kRowBlock, N - base);
    const uint32_t t = threadIdx.x;
    if (t < n) {
        const uint32_t k = pos[base + t];
        if (r_out) { sr[3 * t] = rest.rx[k]; sr[3 * t + 1] = rest.ry[k]; sr[3 * t + 2] = rest.rz[k]; }
        if (v_out) { sv[3 * t] = rest.vx[k]; sv[3 * t + 1] = rest.vy[k]; sv[3 * t + 2] = rest.vz[k]; }
    }
    __syncthreads();
    if (r_out) rows_out(sr, base, n, r_out);
    if (v_out) rows_out(sv, base, n, v_out);
}

// The forces of the rest order in caller rows (FP32 values widened exactly to FP64 for the
// FP64 form; copied for the FP32 form).
template <typename Ti, typename To>
__global__ void __launch_bounds__(kRowBlock) k_get_forces(const uint32_t *pos, const Ti *F, uint32_t N, To *F_out) {
    __shared__ To sf[3 * kRowBlock];
    const uint32_t base = blockIdx.x * kRowBlock;
    const uint32_t n = min((uint32_t)kRowBlock, N - base);
    const uint32_t t = threadIdx.x;
    if (t < n) {
        const uint32_t k = pos[base + t];
#pragma unroll
        for (int d = 0; d < 3; ++d) sf[3 * t + d] = conv<To>(F[(size_t)d * N + k]);
    }
    __syncthreads();
    rows_out(sf, base, n, F_out);
}

__global__ void __launch_bounds__(256) k_get_state_batch(const SysStateArgs *args, const uint32_t *items, int R,
                                                         double *r_out, double *v_out) {
    const int sys = item_system(items, R, blockIdx.x);
    const SysStateArgs &a = args[sys];
    const uint32_t k = (blockIdx.x - items[sys]) * blockDim.x + threadIdx.x;
    if (k < a.N) get_state_body(a.rest, a.p_off, k, r_out, v_out);
}


}  // namespace

void launch_bin(int prec, const BinArgs &a, cudaStream_t st) {
    if (prec == 1) k_bin<1><<<blocks_for(a.N, 256), 256, 0, st>>>(a);
    else k_bin<0><<<blocks_for(a.N, 256), 256, 0, st>>>(a);
}

void launch_bin_batch(const BinArgs *args, const uint32_t *items, int R, uint32_t nblocks, cudaStream_t st) {
    k_bin_batch<<<nblocks, 256, 0, st>>>(args, items, R);
}

void launch_scan(uint32_t *count, uint32_t *tile_sums, uint32_t *cell_start, int ncell, uint32_t N,
                 cudaStream_t st) {
    const int tiles = (ncell + kScanTile - 1) / kScanTile;
    k_tile_sums<<<tiles, 1024, 0, st>>>(count, ncell, tile_sums);
    k_scan_tiles<<<tiles, 1024, 0, st>>>(count, ncell, tile_sums, cell_start, N);
}

void launch_scatter(const uint32_t *cell, const uint32_t *slot, const uint32_t *cell_start, const uint32_t *id,
                    uint32_t N, unsigned long long *keys, cudaStream_t st) {
    k_scatter<<<blocks_for(N, 256), 256, 0, st>>>(cell, slot, cell_start, id, N, keys);
}

void launch_relayout(State from, State to, const float *F_from, float *F_to, uint32_t stride,
                     const uint32_t *old_off, const uint32_t *new_off, int R, uint32_t Nnew, cudaStream_t st) {
    if (Nnew) k_relayout<<<blocks_for(Nnew, 256), 256, 0, st>>>(from, to, F_from, F_to, stride, old_off, new_off, R, Nnew);
}

void launch_gather(int prec, const GatherArgs &g, cudaStream_t st) {
    if (prec == 1) k_gather<1><<<blocks_for(g.N, 256), 256, 0, st>>>(g);
    else k_gather<0><<<blocks_for(g.N, 256), 256, 0, st>>>(g);
}

void launch_set_state(const double *r, const double *v, const double *q_user, const double *invm_user, State rest,
                      uint32_t N, Box box, DevCounters *ctr, cudaStream_t st) {
    k_set_state<<<blocks_for(N, kRowBlock), kRowBlock, 0, st>>>(r, v, q_user, invm_user, rest, N, box);
    k_reset_counters<<<1, 1, 0, st>>>(ctr);
}

uint32_t bin_batch_blocks(uint32_t N) { return blocks_for(N, 256); }

void launch_set_state_batch(const SysStateArgs *args, const uint32_t *items, int R, uint32_t nblocks,
                            const double *r, const double *v, DevCounters *ctr, int nctr, cudaStream_t st) {
    k_set_state_batch<<<nblocks, 256, 0, st>>>(args, items, R, r, v);
    k_reset_counters_n<<<(nctr + 255) / 256, 256, 0, st>>>(ctr, nctr);
}

void launch_get_state_batch(const SysStateArgs *args, const uint32_t *items, int R, uint32_t nblocks, double *r_out,
                            double *v_out, cudaStream_t st) {
    k_get_state_batch<<<nblocks, 256, 0, st>>>(args, items, R, r_out, v_out);
}

void launch_rest_pos(const uint32_t *id, uint32_t N, uint32_t *pos, cudaStream_t st) {
    k_rest_pos<<<blocks_for(N, 256), 256, 0, st>>>(id, N, pos);
}

void launch_get_state(State rest, const uint32_t *pos, uint32_t N, double *r_out, double *v_out, cudaStream_t st) {
    k_get_state<<<blocks_for(N, kRowBlock), kRowBlock, 0, st>>>(rest, pos, N, r_out, v_out);
}

void launch_set_forces(int prec, const double *F_in, void *F, uint32_t N, DevCounters *ctr, cudaStream_t st) {
    const unsigned nb = blocks_for(N > 0 ? N : 1, kRowBlock);
    if (prec == 1) k_set_forces<double, float><<<nb, kRowBlock, 0, st>>>(F_in, (float *)F, N, ctr);
    else k_set_forces<double, double><<<nb, kRowBlock, 0, st>>>(F_in, (double *)F, N, ctr);
}

void launch_set_forces_f32(const float *F_in, float *F, uint32_t N, DevCounters *ctr, cudaStream_t st) {
    k_set_forces<float, float><<<blocks_for(N > 0 ? N : 1, kRowBlock), kRowBlock, 0, st>>>(F_in, F, N, ctr);
}

void launch_get_forces_f32(const uint32_t *pos, const float *F, uint32_t N, float *F_out, cudaStream_t st) {
    k_get_forces<float, float><<<blocks_for(N, kRowBlock), kRowBlock, 0, st>>>(pos, F, N, F_out);
}

void launch_get_forces(int prec, const uint32_t *pos, const void *F, uint32_t N, double *F_out, cudaStream_t st) {
    const unsigned nb = blocks_for(N, kRowBlock);
    if (prec == 1) k_get_forces<float, double><<<nb, kRowBlock, 0, st>>>(pos, (const float *)F, N, F_out);
    else k_get_forces<double, double><<<nb, kRowBlock, 0, st>>>(pos, (const double *)F, N, F_out);
}

}  // namespace rbsog
