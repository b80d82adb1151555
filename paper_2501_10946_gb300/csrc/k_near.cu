// Near field of the RBSOG force step: Eq. (55) first term with F_N1 and F_N2 of
// Eqs. (56)-(57), and U_N of Eq. (50), over the particles within r_c (minimum image).
//
// Two shared-memory tilings of the cell list (cells >= 3 per axis), both staging the
// 27-cell neighbourhood of their target cells with TMA bulk copies completing on one
// mbarrier, pre-filtering candidates in FP32 with ballot masks, and evaluating the exact
// pairs two per pass in packed FP32x2 (FP64 in the FP64 build):
//   * bricks (near_brick_body): a run of W cells in each of by x bz rows, (by + 2)(bz + 2)
//     neighbour rows staged, about 4.5 staged particles per target, which leaves room for
//     precomputed FP32 offsets; the FP32 build uses them for one system (k_near_bricks), a
//     batch of systems (k_near_batch) and the persistent batched step;
//   * row tiles (near_tile_body): a run of W cells in one (y, z) row, its 9 neighbour rows
//     staged; the FP64 build uses them (k_near_tiled64).
// The layout of each is described above its body.
// In both, the pairs of a target are those of a plain loop over the 27 cells in its order;
// which two share a pass follows the pre-filter's hits, so the pre-filter changes the
// rounding of the sums, never the set of pairs.
// Otherwise (fewer than 3 cells on an axis, or a neighbourhood that does not fit the
// buffers): one thread per particle reading candidates from global memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "devmath.cuh"
#include "devutil.cuh"
#include "kernels.h"

namespace rbsog {
namespace {

constexpr int kGlobalThreads = 128;
constexpr int kTileThreads = 128;
constexpr int kSlots = 8;              // candidate slots (32 candidates each) per filter round

__device__ __forceinline__ unsigned long long dup2(float a) { return pk2(a, a); }

// Compensated sum of two lanes at once (the steps of kahan_add on each lane).
__device__ __forceinline__ void kahan2(unsigned long long &s, unsigned long long &c, unsigned long long x) {
    const unsigned long long y = sub2(x, c);
    const unsigned long long t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}

// The two terms of two FP32 pairs (one per lane) before accumulation:
// gsc = q_i q_j [F_N1 + F_N2](r) and uh = q_i q_j [Y - F](r) (the caller halves the sum).
__device__ __forceinline__ void pair_terms2(const NearF &nc, unsigned long long qq, unsigned long long r2,
                                            unsigned long long &gsc, unsigned long long &uh) {
    float r2a, r2b;
    upk2(r2, r2a, r2b);
    const unsigned long long rinv = pk2(rsqrt_ftz(r2a), rsqrt_ftz(r2b));
    const unsigned long long r = mul2(r2, rinv);
    float xa, xb;
    upk2(mul2(r, nc.nl2), xa, xb);
    const unsigned long long e1 = pk2(ex2_approx(xa), ex2_approx(xb));
    unsigned long long nsog = 0ull, fn2 = 0ull;   // nsog = -F(r) of the SOG
    // two Gaussians per iteration (16-byte loads of adjacent constants), same order of sums
    int g = 0;
    for (; g + 1 < nc.mtot; g += 2) {
        const ulonglong2 nb = *reinterpret_cast<const ulonglong2 *>(&nc.nb[g]);
        const ulonglong2 af = *reinterpret_cast<const ulonglong2 *>(&nc.naf[g]);
        const ulonglong2 cf = *reinterpret_cast<const ulonglong2 *>(&nc.cf[g]);
        float ya, yb, za, zb;
        upk2(mul2(r2, nb.x), ya, yb);
        upk2(mul2(r2, nb.y), za, zb);
        const unsigned long long E0 = pk2(ex2_approx(ya), ex2_approx(yb));
        const unsigned long long E1 = pk2(ex2_approx(za), ex2_approx(zb));
        nsog = fma2(af.x, E0, nsog);
        fn2 = fma2(cf.x, E0, fn2);
        nsog = fma2(af.y, E1, nsog);
        fn2 = fma2(cf.y, E1, fn2);
    }
    if (g < nc.mtot) {
        float ya, yb;
        upk2(mul2(r2, nc.nb[g]), ya, yb);
        const unsigned long long E = pk2(ex2_approx(ya), ex2_approx(yb));
        nsog = fma2(nc.naf[g], E, nsog);
        fn2 = fma2(nc.cf[g], E, fn2);
    }
    const unsigned long long rinv3 = mul2(mul2(rinv, rinv), rinv);
    if (!nc.two) {
        const unsigned long long fn1 = mul2(mul2(e1, fma2(r, nc.il2, dup2(1.f))), rinv3);
        gsc = mul2(qq, add2(fn1, fn2));
        uh = mul2(qq, fma2(e1, rinv, nsog));
    } else {
        // two Yukawa terms (EGS): weights folded into the exponents, the second's sign apart
        upk2(fma2(r, nc.nl2, nc.ly1), xa, xb);
        const unsigned long long ew = pk2(ex2_approx(xa), ex2_approx(xb));
        upk2(fma2(r, nc.nl2b, nc.ly2), xa, xb);
        const unsigned long long e2 = mul2(pk2(ex2_approx(xa), ex2_approx(xb)), nc.sg2);
        const unsigned long long fn1 = fma2(mul2(e2, fma2(r, nc.il2b, dup2(1.f))), rinv3,
                                            mul2(mul2(ew, fma2(r, nc.il2, dup2(1.f))), rinv3));
        gsc = mul2(qq, add2(fn1, fn2));
        uh = mul2(qq, fma2(ew, rinv, fma2(e2, rinv, nsog)));
    }
}

// One FP32 pair: accumulate q_i q_j [F_N1 + F_N2](r) (r_i - r_j) and U_N/2 (compensated).
// C is NearConsts (the per-particle path).
template <class C>
__device__ __forceinline__ void pair_f32(const C &nc, float qq, float d0, float d1, float d2, float r2,
                                         float *Fs, float *Fc, float &Us, float &Uc) {
    const float rinv = rsqrt_ftz(r2);
    const float r = r2 * rinv;
    const float e1 = ex2_approx(-r * nc.inv_lam_log2e_f);
    float fsog = 0.f, fn2 = 0.f;
    for (int g = 0; g < nc.mtot; ++g) {
        const float E = ex2_approx(-r2 * nc.bl2f[g]);
        fsog = fmaf(nc.af[g], E, fsog);
        fn2 = fmaf(nc.cf[g], E, fn2);
    }
    if (!nc.two) {
        const float fn1 = e1 * (1.f + r * nc.inv_lam_f) * (rinv * rinv * rinv);
        const float gsc = qq * (fn1 + fn2);
        kahan_add(Fs[0], Fc[0], gsc * d0);
        kahan_add(Fs[1], Fc[1], gsc * d1);
        kahan_add(Fs[2], Fc[2], gsc * d2);
        kahan_add(Us, Uc, 0.5f * qq * (e1 * rinv - fsog));
    } else {
        // two Yukawa terms (EGS): weights folded into the exponents, the second's sign apart
        const float ew = ex2_approx(fmaf(-r, nc.inv_lam_log2e_f, nc.ly1_f));
        const float e2 = nc.sgn2_f * ex2_approx(fmaf(-r, nc.inv_lam2_log2e_f, nc.ly2_f));
        const float rinv3 = rinv * rinv * rinv;
        const float fn1 = fmaf(e2 * (1.f + r * nc.inv_lam2_f), rinv3, ew * (1.f + r * nc.inv_lam_f) * rinv3);
        const float gsc = qq * (fn1 + fn2);
        kahan_add(Fs[0], Fc[0], gsc * d0);
        kahan_add(Fs[1], Fc[1], gsc * d1);
        kahan_add(Fs[2], Fc[2], gsc * d2);
        kahan_add(Us, Uc, 0.5f * qq * fmaf(ew, rinv, fmaf(e2, rinv, -fsog)));
    }
}

// Per-particle near field from global memory (FP32 records).
__device__ void near_one_f32(const NearArgs &a, uint32_t p, float *Fout, double &Uout) {
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const uint4 *rec = (const uint4 *)a.rec;
    const uint4 ri = rec[p];
    const float qi = __uint_as_float(ri.w);
    const uint32_t si[3] = {ri.x, ri.y, ri.z};
    int ci[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ci[d] = (int)(((unsigned long long)si[d] * (unsigned long long)a.box.nc[d]) >> 32);
    float Fs[3] = {0.f, 0.f, 0.f}, Fc[3] = {0.f, 0.f, 0.f}, Us = 0.f, Uc = 0.f;
    const int zlo = nz >= 3 ? -1 : 0, zhi = nz >= 3 ? 1 : 0;
    const int ylo = ny >= 3 ? -1 : 0, yhi = ny >= 3 ? 1 : 0;
    const int xlo = nx >= 3 ? -1 : 0, xhi = nx >= 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int cz = (ci[2] + dz + nz) % nz;
        for (int dy = ylo; dy <= yhi; ++dy) {
            const int cy = (ci[1] + dy + ny) % ny;
            for (int dx = xlo; dx <= xhi; ++dx) {
                const int cx = (ci[0] + dx + nx) % nx;
                const int c = cx + nx * (cy + ny * cz);
                const uint32_t j0 = a.cell_start[c], j1 = a.cell_start[c + 1];
                for (uint32_t j = j0; j < j1; ++j) {
                    if (j == p) continue;
                    const uint4 rj = rec[j];
                    const float d0 = (float)(int)(si[0] - rj.x) * a.box.L_2m32f[0];
                    const float d1 = (float)(int)(si[1] - rj.y) * a.box.L_2m32f[1];
                    const float d2 = (float)(int)(si[2] - rj.z) * a.box.L_2m32f[2];
                    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
                    if (r2 < a.nc.rc2_f) pair_f32(a.nc, qi * __uint_as_float(rj.w), d0, d1, d2, r2, Fs, Fc, Us, Uc);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Fout[d] = Fs[d] - Fc[d];
    Uout = (double)Us - (double)Uc;
}

// One FP64 pair inside r_c: adds q_i q_j [F_N1 + F_N2](r) (r_i - r_j) to F and
// q_i q_j [Y - F](r) / 2 to U (the per-particle and the tiled FP64 paths share it).
__device__ __forceinline__ void pair_f64(const NearConsts &nc, double qq, const double d[3], double r2, double F[3],
                                         double &U) {
    const double r = sqrt(r2);
    const double rinv = 1.0 / r;
    const double e1 = exp(-r * nc.inv_lam);
    double fsog = 0.0, fn2 = 0.0;
    for (int g = 0; g < nc.mtot; ++g) {
        const double E = exp(-r2 * nc.b[g]);
        fsog += nc.a[g] * E;
        fn2 += nc.c[g] * E;
    }
    double fn1 = e1 * (1.0 + r * nc.inv_lam) * (rinv * rinv * rinv);
    double yk = e1 * rinv;
    if (nc.two) {
        // two Yukawa terms (EGS) with weights y1, y2
        const double e2 = nc.y2 * exp(-r * nc.inv_lam2);
        fn1 = nc.y1 * fn1 + e2 * (1.0 + r * nc.inv_lam2) * (rinv * rinv * rinv);
        yk = nc.y1 * yk + e2 * rinv;
    }
    const double gsc = qq * (fn1 + fn2);
    F[0] += gsc * d[0];
    F[1] += gsc * d[1];
    F[2] += gsc * d[2];
    U += 0.5 * qq * (yk - fsog);
}

// Per-particle near field from global memory (FP64 records, 2^64 fixed point).
__device__ void near_one_f64(const NearArgs &a, uint32_t p, double *Fout, double &Uout) {
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const Rec64 *rec = (const Rec64 *)a.rec;
    const Rec64 ri = rec[p];
    int ci[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) ci[d] = (int)(((ri.s[d] >> 32) * (unsigned long long)a.box.nc[d]) >> 32);
    double F[3] = {0.0, 0.0, 0.0}, U = 0.0;
    const int zlo = nz >= 3 ? -1 : 0, zhi = nz >= 3 ? 1 : 0;
    const int ylo = ny >= 3 ? -1 : 0, yhi = ny >= 3 ? 1 : 0;
    const int xlo = nx >= 3 ? -1 : 0, xhi = nx >= 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int cz = (ci[2] + dz + nz) % nz;
        for (int dy = ylo; dy <= yhi; ++dy) {
            const int cy = (ci[1] + dy + ny) % ny;
            for (int dx = xlo; dx <= xhi; ++dx) {
                const int cx = (ci[0] + dx + nx) % nx;
                const int c = cx + nx * (cy + ny * cz);
                const uint32_t j0 = a.cell_start[c], j1 = a.cell_start[c + 1];
                for (uint32_t j = j0; j < j1; ++j) {
                    if (j == p) continue;
                    const Rec64 rj = rec[j];
                    double d[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) d[e] = (double)(long long)(ri.s[e] - rj.s[e]) * a.box.L_2m64[e];
                    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 < a.nc.rc2) pair_f64(a.nc, ri.q * rj.q, d, r2, F, U);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Fout[d] = F[d];
    Uout = U;
}

// Energy partials are per warp (blockDim.x / 32 per block, fixed order), so no block-wide
// barrier waits for the slowest thread at the end of a kernel.  The single-system kernels
// run 128 threads per block.
constexpr int kWarpsPerBlock = 4;
static_assert(kGlobalThreads == 32 * kWarpsPerBlock && kTileThreads == kGlobalThreads, "single-system block size");

// tid: thread index within the group of nt threads that handles block blk
__device__ __forceinline__ void warp_partial(double v, double *U_part, unsigned blk, int tid, int nt) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) U_part[(size_t)blk * (unsigned)(nt >> 5) + (unsigned)(tid >> 5)] = v;
}

// Barrier BAR of a group of NT threads (the near-field kernels use barrier 0 over the whole
// CTA, NT = blockDim.x).
template <int NT, int BAR>
__device__ __forceinline__ void group_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}
template <int NT, int BAR>
__device__ __forceinline__ int group_sync_and(int pred) {
    int r;
    asm volatile(
        "{ .reg .pred a, b; setp.ne.s32 a, %1, 0; bar.red.and.pred b, %2, %3, a; selp.s32 %0, 1, 0, b; }"
        : "=r"(r)
        : "r"(pred), "n"(BAR), "n"(NT)
        : "memory");
    return r;
}

// One block of the per-particle path: particles p0 + [0, blockDim.x) of this system (global
// record indices p0 .. p0 + N - 1).
template <int PREC>
__device__ __forceinline__ void near_global_block(const NearArgs &a, uint32_t p0, unsigned blk,
                                                  int tid = (int)threadIdx.x, int nt = (int)blockDim.x) {
    const uint32_t local = blk * (unsigned)nt + (unsigned)tid;
    double U = 0.0;
    if (local < a.N) {
        const uint32_t p = p0 + local;
        const bool overflow = (a.ctr->err & kErrCellOverflow) != 0;
        if (PREC == 1) {
            float F[3] = {0.f, 0.f, 0.f};
            if (!overflow) near_one_f32(a, p, F, U);
            float *Fn = (float *)a.Fn;
            Fn[p] = F[0]; Fn[a.stride + p] = F[1]; Fn[2 * (size_t)a.stride + p] = F[2];
        } else {
            double F[3] = {0.0, 0.0, 0.0};
            if (!overflow) near_one_f64(a, p, F, U);
            double *Fn = (double *)a.Fn;
            Fn[p] = F[0]; Fn[a.stride + p] = F[1]; Fn[2 * (size_t)a.stride + p] = F[2];
        }
    }
    warp_partial(U, a.U_part, blk, tid, nt);
}

template <int PREC>
__global__ void __launch_bounds__(kGlobalThreads) k_near_global(NearArgs a) {
    near_global_block<PREC>(a, 0u, blockIdx.x);
}

// ---------------------------------------------------------------- row tiles
// One CTA owns a run of W cells along x in one (y, z) row.  Their 27-cell neighbourhood is
// 9 rows of W + 2 cells, each row one (or, across the periodic seam, two) contiguous slices
// of the cell-sorted particle records, staged with TMA bulk copies; while they fly the CTA
// writes, for each of its target cells, the list of staging indices of that cell's 27-cell
// candidates.  A warp owns 32 consecutive targets (about five cells), in two phases:
//   (1) filter, cell by cell: the lanes hold the cell's candidates (32 per slot) as FP32
//       offsets from the cell centre, and the warp tests each target of the cell against
//       all of them at once (packed FP32x2 arithmetic), keeping one ballot mask per slot;
//   (2) pairs: each lane walks its own target's masks in candidate order, recomputes the
//       separation exactly from the fixed-point coordinates, applies the exact r < r_c
//       test and accumulates the pair forces: the two of a pass added in FP32, then one
//       compensated FP32 add (FP64 build: plain FP64 sums, one pair at a time).
// Neighbourhoods larger than 8 slots (256 candidates) run in several such rounds.
// CAP: staged particles per CTA; NT: threads per CTA.  F64: the FP64 build's 32-byte
// records (u64 coordinates), else the FP32 build's 16-byte ones.
template <bool F64>
struct TileRec;
template <>
struct TileRec<false> {
    using T = uint4;
    // the high 32 bits of the fixed-point coordinates (the pre-filter's input)
    __device__ static __forceinline__ uint32_t x(const uint4 &r) { return r.x; }
    __device__ static __forceinline__ uint32_t y(const uint4 &r) { return r.y; }
    __device__ static __forceinline__ uint32_t z(const uint4 &r) { return r.z; }
};
template <>
struct TileRec<true> {
    using T = Rec64;
    __device__ static __forceinline__ uint32_t x(const Rec64 &r) { return (uint32_t)(r.s[0] >> 32); }
    __device__ static __forceinline__ uint32_t y(const Rec64 &r) { return (uint32_t)(r.s[1] >> 32); }
    __device__ static __forceinline__ uint32_t z(const Rec64 &r) { return (uint32_t)(r.s[2] >> 32); }
};

template <int CAP, int NT, int MW, bool F64 = false>
struct TileSmem {
    using Rec = typename TileRec<F64>::T;
    Rec stage[CAP];                         // staged records
    uint32_t mask[kSlots][NT];    // per target (column = owning thread): hit bits of a round
    uint16_t flat[3 * CAP];                 // per target cell: staging indices of its 27-cell candidates
    int fb[MW + 2];                         // target cell i: candidates flat[fb[i] .. fb[i+1])
    NearF nf;                               // the system's FP32 pair constants
    int seg_off[9][MW + 3];                 // per row: offset of each region cell within the row
    int row_base[10];                       // per row: offset of the row in the staging buffer
    uint32_t chunk_g[9][2];                 // per row: global start of up to two slices
    uint32_t chunk_n[9][2];                 // per row: particle count of each slice
    unsigned long long mbar;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Region cell (1 .. wn-2) of the centre row holding staged target jl (offset within row 4):
// the last i with seg_off[4][i] <= jl.
template <class TS>
__device__ __forceinline__ int region_cell(const TS &S, int wn, int jl) {
    int lo = 1, hi = wn - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.seg_off[4][mid] <= jl) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One tile's geometry and the outcome of its staging.
struct TileCtx {
    int x0, x1, wn, ntc, cy, cz;
    uint32_t g_first, g_end;                // the tile's targets in global record order
    int region_n;                           // staged particles
    bool overflow;                          // the cell build overflowed: no pairs at all
    bool staged;                            // the neighbourhood fits the staging buffer
    bool ok;                                // staged, and the copies landed
};

// Prologue of a tile (NT threads tid 0 .. NT-1): cell populations of the
// 9 x wn region, the row slices, the bulk copies of the region into S.stage, the system's
// pair constants, and per target cell the list of its 27-cell candidates (staging index
// << FSH, rows 0..8 in order, each row's cells i-1 .. i+1 in staging order) in S.flat.
template <int NT, int FSH, class TS>
__device__ __forceinline__ TileCtx tile_stage(const NearArgs &a, int W, int tiles_x, unsigned blk, TS &S,
                                              int tid) {
    using RecT = typename TS::Rec;
    constexpr uint32_t kRecBytes = (uint32_t)sizeof(RecT);
    TileCtx c;
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const int tile = (int)(blk % (unsigned)tiles_x);
    const int rest = (int)(blk / (unsigned)tiles_x);
    const int cy = rest % ny, cz = rest / ny;
    const int x0 = tile * W;
    const int x1 = min(x0 + W, nx);
    const int wn = x1 - x0 + 2;                  // region cells per row: x0-1 .. x1
    const int ntc = wn - 2;                      // target cells: region cells 1 .. wn-2
    c.x0 = x0; c.x1 = x1; c.wn = wn; c.ntc = ntc; c.cy = cy; c.cz = cz;
    const uint32_t *cs = a.cell_start;
    c.overflow = (a.ctr->err & kErrCellOverflow) != 0;

    // cell populations of the 9 x wn region cells, loaded in parallel (row r: dz = r/3 - 1,
    // dy = r%3 - 1)
    for (int e = tid; e < 9 * wn; e += NT) {
        const int r = e / wn, i = e - r * wn;
        const int yr = (cy + r % 3 - 1 + ny) % ny, zr = (cz + r / 3 - 1 + nz) % nz;
        int x = x0 - 1 + i;
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        const int cc = x + nx * (yr + ny * zr);
        S.seg_off[r][i + 1] = (int)(cs[cc + 1] - cs[cc]);
    }
    if (tid == 0) {
        S.nf.mtot = a.nc.mtot;
        S.nf.two = a.nc.two;
        S.nf.nl2 = dup2(-a.nc.inv_lam_log2e_f);
        S.nf.il2 = dup2(a.nc.inv_lam_f);
        S.nf.ly1 = dup2(a.nc.ly1_f);
        S.nf.nl2b = dup2(-a.nc.inv_lam2_log2e_f);
        S.nf.il2b = dup2(a.nc.inv_lam2_f);
        S.nf.ly2 = dup2(a.nc.ly2_f);
        S.nf.sg2 = dup2(a.nc.sgn2_f);
    }
    for (int g = tid; g < a.nc.mtot; g += NT) {
        S.nf.nb[g] = dup2(-a.nc.bl2f[g]);
        S.nf.naf[g] = dup2(-a.nc.af[g]);
        S.nf.cf[g] = dup2(a.nc.cf[g]);
    }
    group_sync<NT, 0>();
    // per-row prefix sums and the global slices of each row (a short serial loop per row
    // measured faster here than warp-wide scans)
    if (tid < 9) {
        const int yr = (cy + tid % 3 - 1 + ny) % ny, zr = (cz + tid / 3 - 1 + nz) % nz;
        const int rowbase = nx * (yr + ny * zr);
        int off = 0;
        S.seg_off[tid][0] = 0;
        for (int i = 1; i <= wn; ++i) {
            off += S.seg_off[tid][i];
            S.seg_off[tid][i] = off;
        }
        if (x0 >= 1 && x1 <= nx - 1) {           // one slice: cells x0-1 .. x1
            S.chunk_g[tid][0] = cs[rowbase + x0 - 1];
            S.chunk_n[tid][0] = cs[rowbase + x1 + 1] - cs[rowbase + x0 - 1];
            S.chunk_g[tid][1] = 0; S.chunk_n[tid][1] = 0;
        } else if (x0 == 0) {                    // cell nx-1, then cells 0 .. x1
            S.chunk_g[tid][0] = cs[rowbase + nx - 1];
            S.chunk_n[tid][0] = cs[rowbase + nx] - cs[rowbase + nx - 1];
            S.chunk_g[tid][1] = cs[rowbase];
            S.chunk_n[tid][1] = cs[rowbase + x1 + 1] - cs[rowbase];
        } else {                                 // x1 == nx: cells x0-1 .. nx-1, then cell 0
            S.chunk_g[tid][0] = cs[rowbase + x0 - 1];
            S.chunk_n[tid][0] = cs[rowbase + nx] - cs[rowbase + x0 - 1];
            S.chunk_g[tid][1] = cs[rowbase];
            S.chunk_n[tid][1] = cs[rowbase + 1] - cs[rowbase];
        }
    }
    group_sync<NT, 0>();
    if (tid == 0) {
        int b = 0;
        for (int r = 0; r < 9; ++r) {
            S.row_base[r] = b;
            b += S.seg_off[r][wn];
        }
        S.row_base[9] = b;
    }
    group_sync<NT, 0>();
    const int region_n = S.row_base[9];
    c.region_n = region_n;
    c.staged = !c.overflow && region_n <= (int)(sizeof(S.stage) / sizeof(RecT));
    // center row (r = 4): targets are region cells 1 .. wn-2, contiguous in global memory
    c.g_first = cs[nx * (cy + ny * cz) + x0];
    c.g_end = cs[nx * (cy + ny * cz) + x1];
    c.ok = c.staged;
    if (!c.staged || region_n == 0) return c;

    const uint32_t bar = smem_u32(&S.mbar);
    if (tid == 0) {                              // start the bulk copies of the region
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)region_n * kRecBytes) : "memory");
        const RecT *rec = (const RecT *)a.rec;
        for (int r = 0; r < 9; ++r) {
            uint32_t dst = (uint32_t)S.row_base[r];
            for (int h = 0; h < 2; ++h) {
                const uint32_t n = S.chunk_n[r][h];
                if (n) {
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                        "[%3];" ::"r"(smem_u32(&S.stage[dst])),
                        "l"(rec + S.chunk_g[r][h]), "r"(n * kRecBytes), "r"(bar) : "memory");
                    dst += n;
                }
            }
        }
    }
    // offsets of the target cells' candidate lists: fb[i] = sum of the 27-cell counts
    // of target cells 1 .. i-1.  A staged particle is a candidate of at most 3 target
    // cells, so all lists together fit 3 CAP entries.  (The barriers below also make
    // thread 0's mbarrier initialisation visible before any thread polls it.)
    if (tid < ntc) {
        const int i = tid + 1;
        int tot = 0;
        for (int r = 0; r < 9; ++r) tot += S.seg_off[r][i + 2] - S.seg_off[r][i - 1];
        S.fb[i + 1] = tot;
    }
    group_sync<NT, 0>();
    if (tid == 0) {
        int b = 0;
        S.fb[1] = 0;
        for (int i = 1; i <= ntc; ++i) {
            b += S.fb[i + 1];
            S.fb[i + 1] = b;
        }
    }
    group_sync<NT, 0>();
    // while the copies fly: the candidate list of each target cell i, rows 0..8 in
    // order, each row's cells i-1 .. i+1 in staging order
    for (int e = tid; e < 9 * ntc; e += NT) {
        const int i = e / 9 + 1, r = e - (e / 9) * 9;
        int pos = S.fb[i];
        for (int q = 0; q < r; ++q) pos += S.seg_off[q][i + 2] - S.seg_off[q][i - 1];
        const int a0 = S.seg_off[r][i - 1], n = S.seg_off[r][i + 2] - a0;
        const int st = S.row_base[r] + a0;
        for (int l = 0; l < n; ++l) S.flat[pos + l] = (uint16_t)((st + l) << FSH);
    }
    // bounded wait for the staged bytes (phase 0); the outcome is made block-uniform,
    // and the block barrier also publishes the candidate lists
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    }
    c.ok = group_sync_and<NT, 0>((int)done) != 0;
    if (!c.ok) {
        if (tid == 0) atomicOr(&a.ctr->err, kErrNearStage);
        // let the copies in flight land before the CTA exits (again bounded)
        for (int it = 0; it < (1 << 22) && !done; ++it)
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                : "=r"(done)
                : "r"(bar)
                : "memory");
    }
    return c;
}

// Targets of a tile whose neighbourhood did not fit the staging buffer (or whose cell build
// overflowed): one thread per particle from global memory.  Returns the thread's energy.
template <int NT, bool F64>
__device__ __forceinline__ double tile_fallback(const NearArgs &a, const TileCtx &c, int tid) {
    double Ufall = 0.0;
    for (uint32_t g = c.g_first + tid; g < c.g_end; g += NT) {
        double U = 0.0;
        if constexpr (F64) {
            double F[3] = {0.0, 0.0, 0.0};
            if (!c.overflow) near_one_f64(a, g, F, U);
            double *Fn = (double *)a.Fn;
            Fn[g] = F[0]; Fn[a.stride + g] = F[1]; Fn[2 * (size_t)a.stride + g] = F[2];
        } else {
            float F[3] = {0.f, 0.f, 0.f};
            if (!c.overflow) near_one_f32(a, g, F, U);
            float *Fn = (float *)a.Fn;
            Fn[g] = F[0]; Fn[a.stride + g] = F[1]; Fn[2 * (size_t)a.stride + g] = F[2];
        }
        Ufall += U;
    }
    return Ufall;
}

// The tile is handled by the CTA's NT threads (tid 0 .. NT-1).
template <int CAP, int NT, int MW, bool F64 = false>
__device__ __forceinline__ void near_tile_body(const NearArgs &a, int W, int tiles_x, unsigned blk,
                                               TileSmem<CAP, NT, MW, F64> &S, int tid) {
    using RecT = typename TileRec<F64>::T;
    using RO = TileRec<F64>;
    const int lane = tid & 31, wid = tid >> 5;
    const unsigned full = 0xffffffffu;
    const TileCtx c = tile_stage<NT, 0>(a, W, tiles_x, blk, S, tid);
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const int x0 = c.x0, wn = c.wn, cy = c.cy, cz = c.cz;
    const uint32_t g_first = c.g_first;
    float sumU = 0.f;
    double sumUd = 0.0;            // FP64 build
    double Ufall = 0.0;
    if (c.staged) {
        const bool ok = c.ok;
        if (ok) {
            const int rb4 = S.row_base[4];
            const int t0 = rb4 + S.seg_off[4][1];
            const int t1 = rb4 + S.seg_off[4][wn - 1];
            float *Fn = (float *)a.Fn;
            const float rc2 = a.nc.rc2_f;
            // Pre-filter |t - c|^2 < thr with thr = r_c^2 (1 + 4e-5).  An FP32 offset from the
            // cell centre is within 1.8e-7 c of the exact one (|offset| <= 1.5 c per axis, two
            // roundings; c < 4/3 r_c because n_c = floor(L / r_c) >= 3), so the test decides
            // within 3.3e-6 r_c^2 of the exact comparison and every pair that the exact test
            // accepts passes.
            const float rcf2 = rc2 * 1.00004f;
            const float sx = a.box.L_2m32f[0], sy = a.box.L_2m32f[1], sz = a.box.L_2m32f[2];
            const unsigned long long sx2 = dup2(sx), sy2 = dup2(sy), sz2 = dup2(sz);
            // fixed-point centre of the target row (y, z) and cell width along x; any point
            // near the centre serves, only offsets up to 1.5 cells matter
            const float cwx = 4294967296.f / (float)nx;
            const uint32_t oy = __float2uint_rz(((float)cy + 0.5f) * (4294967296.f / (float)ny));
            const uint32_t oz = __float2uint_rz(((float)cz + 0.5f) * (4294967296.f / (float)nz));
            for (int wlo = t0 + 32 * wid; wlo < t1; wlo += NT) {
                const int whi = min(wlo + 32, t1);
                const int j = wlo + lane;
                const bool has = j < whi;
                const int i_lo = region_cell(S, wn, wlo - rb4);
                const int i_hi = region_cell(S, wn, whi - 1 - rb4);
                const int i_own = has ? region_cell(S, wn, j - rb4) : i_hi;
                const RecT ri = S.stage[has ? j : wlo];
                float qi = 0.f;
                if constexpr (!F64) qi = __uint_as_float(ri.w);
                // FP32: compensated sums, packed: (F_x, F_y) and (F_z, U); FP64: plain sums in
                // candidate order (the order of the per-particle path)
                unsigned long long Fxy = 0ull, Cxy = 0ull, Fzu = 0ull, Czu = 0ull;
                double Fd[3] = {0.0, 0.0, 0.0}, Ud = 0.0;
                int own_cb = 0, own_total = 0;
                for (int base = 0;; base += 32 * kSlots) {
                    bool more = false;
                    // (1) filter, cell by cell: the lanes hold the cell's candidates, the warp
                    // tests each target of the cell against all of them
                    for (int i = i_lo; i <= i_hi; ++i) {
                        const int ta = max(wlo, rb4 + S.seg_off[4][i]);
                        const int tb = min(whi, rb4 + S.seg_off[4][i + 1]);
                        if (ta >= tb) continue;
                        const int cb = S.fb[i], total = S.fb[i + 1] - cb;
                        if (i == i_own) {
                            own_cb = cb;
                            own_total = total;
                        }
                        if (total <= base) continue;
                        more = more || total > base + 32 * kSlots;
                        const int nsl = min(kSlots, (total - base + 31) >> 5);
                        const uint32_t ox = __float2uint_rz(((float)(x0 - 1 + i) + 0.5f) * cwx);
                        // no candidate: far away
                        float X[kSlots], Y[kSlots], Z[kSlots];
#pragma unroll
                        for (int s = 0; s < kSlots; ++s) {
                            X[s] = 3e30f;
                            Y[s] = 0.f;
                            Z[s] = 0.f;
                            const int f = base + 32 * s + lane;
                            if (s < nsl && f < total) {
                                const RecT rk = S.stage[S.flat[cb + f]];
                                X[s] = (float)(int)(RO::x(rk) - ox) * sx;
                                Y[s] = (float)(int)(RO::y(rk) - oy) * sy;
                                Z[s] = (float)(int)(RO::z(rk) - oz) * sz;
                            }
                        }
                        unsigned long long X2[kSlots / 2], Y2[kSlots / 2], Z2[kSlots / 2];
#pragma unroll
                        for (int h = 0; h < kSlots / 2; ++h) {
                            X2[h] = pk2(X[2 * h], X[2 * h + 1]);
                            Y2[h] = pk2(Y[2 * h], Y[2 * h + 1]);
                            Z2[h] = pk2(Z[2 * h], Z[2 * h + 1]);
                        }

                        int t = ta;
                        for (; t + 1 < tb; t += 2) {
                            const RecT pa = S.stage[t], pb = S.stage[t + 1];
                            const float xa = (float)(int)(RO::x(pa) - ox) * sx, ya = (float)(int)(RO::y(pa) - oy) * sy,
                                        za = (float)(int)(RO::z(pa) - oz) * sz;
                            const float xb = (float)(int)(RO::x(pb) - ox) * sx, yb = (float)(int)(RO::y(pb) - oy) * sy,
                                        zb = (float)(int)(RO::z(pb) - oz) * sz;
                            const unsigned long long xa2 = pk2(xa, xa), ya2 = pk2(ya, ya), za2 = pk2(za, za);
                            const unsigned long long xb2 = pk2(xb, xb), yb2 = pk2(yb, yb), zb2 = pk2(zb, zb);
                            // accept |t - c|^2 < thr
                            const int col = 32 * wid + (t - wlo);
#pragma unroll
                            for (int h = 0; h < kSlots / 2; ++h) {
                                if (2 * h < nsl) {
                                    float a0, a1, b0, b1;
                                    const unsigned long long dxa = sub2(xa2, X2[h]), dya = sub2(ya2, Y2[h]), dza = sub2(za2, Z2[h]);
                                    const unsigned long long dxb = sub2(xb2, X2[h]), dyb = sub2(yb2, Y2[h]), dzb = sub2(zb2, Z2[h]);
                                    upk2(fma2(dza, dza, fma2(dya, dya, mul2(dxa, dxa))), a0, a1);
                                    upk2(fma2(dzb, dzb, fma2(dyb, dyb, mul2(dxb, dxb))), b0, b1);
                                    const uint32_t ma0 = __ballot_sync(full, a0 < rcf2);
                                    const uint32_t mb0 = __ballot_sync(full, b0 < rcf2);
                                    if (lane == 0) {
                                        S.mask[2 * h][col] = ma0;
                                        S.mask[2 * h][col + 1] = mb0;
                                    }
                                    if (2 * h + 1 < nsl) {
                                        const uint32_t ma1 = __ballot_sync(full, a1 < rcf2);
                                        const uint32_t mb1 = __ballot_sync(full, b1 < rcf2);
                                        if (lane == 0) {
                                            S.mask[2 * h + 1][col] = ma1;
                                            S.mask[2 * h + 1][col + 1] = mb1;
                                        }
                                    }
                                }
                            }
                        }
                        if (t < tb) {
                            const RecT rt = S.stage[t];
                            const float xt = (float)(int)(RO::x(rt) - ox) * sx;
                            const float yt = (float)(int)(RO::y(rt) - oy) * sy;
                            const float zt = (float)(int)(RO::z(rt) - oz) * sz;
                            const unsigned long long xt2 = pk2(xt, xt), yt2 = pk2(yt, yt), zt2 = pk2(zt, zt);
                            const int col = 32 * wid + (t - wlo);
#pragma unroll
                            for (int h = 0; h < kSlots / 2; ++h) {
                                if (2 * h < nsl) {
                                    float ra, rb;
                                    const unsigned long long dx = sub2(xt2, X2[h]), dy = sub2(yt2, Y2[h]), dz = sub2(zt2, Z2[h]);
                                    upk2(fma2(dz, dz, fma2(dy, dy, mul2(dx, dx))), ra, rb);
                                    const uint32_t ma = __ballot_sync(full, ra < rcf2);
                                    if (lane == 0) S.mask[2 * h][col] = ma;
                                    if (2 * h + 1 < nsl) {
                                        const uint32_t mb = __ballot_sync(full, rb < rcf2);
                                        if (lane == 0) S.mask[2 * h + 1][col] = mb;
                                    }
                                }
                            }
                        }
                    }
                    __syncwarp();
                    // (2) pairs of the own target in candidate order (rows 0..8, staging
                    // order), two per pass: exact separation and exact r < r_c test
                    if constexpr (F64) {
                        // FP64: one pair at a time, the separation from the 2^64 fixed point
                        if (has) {
                            const int nsl = min(kSlots, max(0, (own_total - base + 31) >> 5));
                            for (int s2 = 0; s2 < nsl; ++s2) {
                                uint32_t m = S.mask[s2][tid];
                                while (m != 0) {
                                    const int k = S.flat[own_cb + base + 32 * s2 + (__ffs(m) - 1)];
                                    m &= m - 1;
                                    if (k == j) continue;
                                    const Rec64 &rk = S.stage[k];
                                    double d[3];
#pragma unroll
                                    for (int e = 0; e < 3; ++e)
                                        d[e] = (double)(long long)(ri.s[e] - rk.s[e]) * a.box.L_2m64[e];
                                    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                                    if (r2 < a.nc.rc2) pair_f64(a.nc, ri.q * rk.q, d, r2, Fd, Ud);
                                }
                            }
                        }
                    } else if (has) {
                        const int nsl = min(kSlots, max(0, (own_total - base + 31) >> 5));
                        uint32_t m = 0;
                        int s = -1;
                        while (true) {
                            int kA = -1, kB = -1;
                            while (m == 0 && ++s < nsl) m = S.mask[s][tid];
                            if (m != 0) {
                                kA = S.flat[own_cb + base + 32 * s + (__ffs(m) - 1)];
                                m &= m - 1;
                            }
                            while (m == 0 && ++s < nsl) m = S.mask[s][tid];
                            if (m != 0) {
                                kB = S.flat[own_cb + base + 32 * s + (__ffs(m) - 1)];
                                m &= m - 1;
                            }
                            if (kA < 0) break;
                            const uint4 pa = S.stage[kA], pb = S.stage[kB < 0 ? kA : kB];
                            const unsigned long long d0 = mul2(pk2((float)(int)(ri.x - pa.x), (float)(int)(ri.x - pb.x)), sx2);
                            const unsigned long long d1 = mul2(pk2((float)(int)(ri.y - pa.y), (float)(int)(ri.y - pb.y)), sy2);
                            const unsigned long long d2 = mul2(pk2((float)(int)(ri.z - pa.z), (float)(int)(ri.z - pb.z)), sz2);
                            float a0, b0, a1, b1, a2, b2, r2a, r2b;
                            upk2(d0, a0, b0);
                            upk2(d1, a1, b1);
                            upk2(d2, a2, b2);
                            upk2(fma2(d2, d2, fma2(d1, d1, mul2(d0, d0))), r2a, r2b);
                            const bool va = kA != j && r2a < rc2, vb = kB >= 0 && kB != j && r2b < rc2;
                            unsigned long long g2, u2;
                            pair_terms2(S.nf, pk2(qi * __uint_as_float(pa.w), qi * __uint_as_float(pb.w)),
                                        pk2(va ? r2a : rc2, vb ? r2b : rc2), g2, u2);
                            float ga, gb, ua, ub;
                            upk2(g2, ga, gb);
                            upk2(u2, ua, ub);
                            // the pass's two contributions added in FP32, then one compensated add
                            ga = va ? ga : 0.f; ua = va ? ua : 0.f;
                            gb = vb ? gb : 0.f; ub = vb ? ub : 0.f;
                            kahan2(Fxy, Cxy, fma2(dup2(ga), pk2(a0, a1), mul2(dup2(gb), pk2(b0, b1))));
                            kahan2(Fzu, Czu, fma2(pk2(ga, 1.f), pk2(a2, ua), mul2(pk2(gb, 1.f), pk2(b2, ub))));
                        }
                    }
                    __syncwarp();
                    if (!more) break;
                }
                if (has) {
                    const uint32_t g = g_first + (uint32_t)(j - t0);
                    if constexpr (F64) {
                        double *Fn64 = (double *)a.Fn;
                        Fn64[g] = Fd[0];
                        Fn64[a.stride + g] = Fd[1];
                        Fn64[2 * (size_t)a.stride + g] = Fd[2];
                        sumUd += Ud;
                    } else {
                        float fx, fy, fz, us, cx, cy, cz_, uc;
                        upk2(Fxy, fx, fy);
                        upk2(Cxy, cx, cy);
                        upk2(Fzu, fz, us);
                        upk2(Czu, cz_, uc);
                        Fn[g] = fx - cx;
                        Fn[a.stride + g] = fy - cy;
                        Fn[2 * (size_t)a.stride + g] = fz - cz_;
                        sumU += 0.5f * (us - uc);        // each pair counted from both ends
                    }
                }
            }
        }
    } else {
        Ufall = tile_fallback<NT, F64>(a, c, tid);
    }
    if constexpr (F64) warp_partial(sumUd + Ufall, a.U_part, blk, tid, NT);
    else warp_partial((double)sumU + Ufall, a.U_part, blk, tid, NT);
}

// Lower bound of cell k (any integer, unwrapped) of n in the 2^32 fixed point:
// ceil(k 2^32 / n), the least s with floor(s n / 2^32) = k.
__device__ __forceinline__ long long cell_lo(int k, int n) {
    // the FP64 quotient is within one of the exact one; integer products settle it
    const long long num = (long long)k << 32;
    long long q = (long long)floor((double)k * (4294967296.0 / (double)n));
    while (q * n < num) ++q;
    while ((q - 1) * n >= num) --q;
    return q;
}

// ---------------------------------------------------------------- FP32 brick tiles
// One CTA owns a brick of target cells: a run of W cells along x in each of by x bz
// adjacent (y, z) rows.  Its neighbourhood is (by + 2)(bz + 2) rows of W + 2 cells, each
// row one or two contiguous slices of the cell-sorted records, staged by bulk copies
// completing on one mbarrier: about 4 staged particles per target, where a single row of
// targets stages about 10.  Then:
//   (0) every staged particle's offset c from the brick centre in FP32, with -|c|^2/2;
//   (1) pre-filter, one target cell per warp at a time: the lanes hold the cell's
//       candidates (32 per slot, each loaded once), the cell's targets sit in registers
//       (chunks of 4, 6 or 8, two per packed FP32x2 lane), and each test is three packed FMAs
//       against the expanded form of |t - c|^2 < thr; one ballot mask per (slot, target);
//   (2) pairs, one thread per target: its masks in candidate order, two hits per pass,
//       the exact separation from the fixed-point coordinates, the exact r < r_c test,
//       packed FP32x2 pair terms with the SOG constants read from the kernel parameters,
//       the pass's two contributions added in FP32 and then one compensated add.
// The pairs are those of a plain loop over the 27 cells in its order; which two share a
// pass follows the pre-filter's hits, so the pre-filter changes the rounding of the sums,
// never the set of pairs.

// Shared-memory loads by 32-bit shared address (OFF: a constant byte offset folded into the
// instruction).
template <int OFF = 0>
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Bounded wait for phase 0 of the mbarrier at bar: each try suspends the thread for at most
// 100 us and returns as soon as the phase completes; gives up after `tries`.  1: complete.
__device__ __forceinline__ uint32_t mbar_wait0(uint32_t bar, int tries) {
    uint32_t done = 0;
    for (int it = 0; it < tries && !done; ++it)
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "n"(100000)
            : "memory");
    return done;
}

// Store four hit masks to shared address a from lane 0.
__device__ __forceinline__ void sts4_lane0(int lane, uint32_t a, uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
    asm volatile("{ .reg .pred p; setp.eq.u32 p, %0, 0; @p st.shared.v4.u32 [%1], {%2, %3, %4, %5}; }" ::"r"(lane),
                 "r"(a), "r"(m0), "r"(m1), "r"(m2), "r"(m3)
                 : "memory");
}

template <int CAP, int FCAP, int NT, int MW, int BY, int BZ, int TMX, int MP>
struct BrickSmem {
    static constexpr int NR = (BY + 2) * (BZ + 2);     // neighbourhood rows
    static constexpr int NTR = BY * BZ;                // target rows
    static constexpr int NC = NTR * MW;                // target cells
    static_assert(CAP * 32 <= 65535, "shared addresses of the offsets are 16-bit");
    static_assert(CAP <= 4096 && NC <= 256 && NR <= 32 && NTR <= 32, "packed descriptors, one row per lane");
    uint4 stage[CAP];                       // staged records
    float4 off[CAP];                        // FP32 offsets c from the brick centre (x, y, z, -|c|^2/2)
    uint16_t flat[FCAP];                    // per target cell: shared addresses of its candidates' offsets
    uint32_t mpool[MP];                     // hit masks: per target cell a block of slots x stride
                                            // words (stride: its targets rounded up to 4)
    int seg_off[NR][MW + 3];                // per row: offset of each region cell within the row
    uint32_t cstart[NR][MW + 2];            // per row: global start of each region cell
    int row_tot[NR];                        // per row: staged particles
    int row_base[NR + 1];                   // per row: offset of the row in the staging buffer
    uint32_t cinfo[NC];                     // target cell tc: region row | region cell << 8 |
                                            // first neighbour row << 16 | target row << 24
    int cnt[NC];                            // target cell tc: its targets
    int fb[NC + 1];                         // target cell tc: candidates flat[fb[tc] .. fb[tc+1])
    int mbase[NC];                          // target cell tc: first word of its mask block
    int tp[NTR + 1];                        // target row tr: brick targets tp[tr] .. tp[tr+1]
    uint2 tinfo[TMX];                       // brick target t: global index, staged index | cell
                                            // << 12 | index within the cell << 20
    long long ref[3];                       // fixed-point brick centre
    int staged, next, copied;               // staging decision; next target cell to filter;
                                            // bulk copies started
    NearF nf;                               // a batched system's pair constants
    unsigned long long mbar;
};

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Brick (bx, byi, bzi) of a system whose geometry is bg; blk: its block index among the
// system's bricks (energy partials).  PERSIST: the persistent step reuses S for its next
// brick, so the mbarrier is invalidated once every thread is done with it.
template <int CAP, int FCAP, int NT, int MW, int BY, int BZ, int TMX, int MP, bool PERSIST = false>
__device__ __forceinline__ void near_brick_body(const NearArgs &a, const NearF &nf, const NearBatchGeom &bg, int bx,
                                                int byi, int bzi, unsigned blk,
                                                BrickSmem<CAP, FCAP, NT, MW, BY, BZ, TMX, MP> &S, int tid) {
    constexpr int NW = NT / 32;
    const int lane = tid & 31, wid = tid >> 5;
    const unsigned full = 0xffffffffu;
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const uint32_t *cs = a.cell_start;
    const bool overflow = (a.ctr->err & kErrCellOverflow) != 0;
    // brick: x cells x0 .. x1-1, rows y0 .. y0+by-1, z0 .. z0+bz-1
    const int x0 = bx * bg.W, x1 = min(x0 + bg.W, nx);
    const int y0 = byi * bg.by, z0 = bzi * bg.bz;
    // (persistent step) the mbarrier of a brick whose copies were started, invalidated once
    // every thread is past its last use
    auto release = [&]() {
        if constexpr (PERSIST) {
            if (S.copied) {
                group_sync<NT, 0>();
                if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.mbar)) : "memory");
            }
        }
    };
    const int by = min(bg.by, ny - y0), bz = min(bg.bz, nz - z0);
    const int wn = x1 - x0 + 2, ntc = wn - 2;  // region cells x0-1 .. x1; target cells 1 .. wn-2
    const int nry = by + 2, nr = nry * (bz + 2), ntr = by * bz, ncells = ntr * ntc;
    // (a) one region row (y0-1 + r % nry, z0-1 + r / nry) per warp at a time, one cell per
    // lane: global starts, populations and their prefix within the row; the reference point
    // (threads 0..2: the centre of the region's extent on each axis, exact in the fixed point)
    // (quotients of small integers by float reciprocals: exact, as the operands are far
    // from multiples of the divisor)
    const float inry = 1.f / (float)nry, intc = 1.f / (float)ntc, inby = 1.f / (float)by;
    for (int r = wid; r < nr; r += NW) {
        const int rz = __float2int_rz(((float)r + 0.5f) * inry), ry = r - rz * nry;
        int yr = y0 - 1 + ry, zr = z0 - 1 + rz;
        yr = yr < 0 ? yr + ny : (yr >= ny ? yr - ny : yr);
        zr = zr < 0 ? zr + nz : (zr >= nz ? zr - nz : zr);
        const int rowbase = nx * (yr + ny * zr);
        int n = 0;
        if (lane < wn) {
            int x = x0 - 1 + lane;
            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            const uint32_t c0 = cs[rowbase + x];
            S.cstart[r][lane] = c0;
            n = (int)(cs[rowbase + x + 1] - c0);
        }
        n = warp_incl_scan(n, lane);
        if (lane < wn) S.seg_off[r][lane + 1] = n;
        if (lane == 0) S.seg_off[r][0] = 0;
        if (lane == 31) S.row_tot[r] = n;
    }
    if (tid < 3) {
        const int lo = tid == 0 ? x0 - 1 : (tid == 1 ? y0 - 1 : z0 - 1);
        const int hi = tid == 0 ? x1 + 1 : (tid == 1 ? y0 + by + 1 : z0 + bz + 1);
        S.ref[tid] = (cell_lo(lo, a.box.nc[tid]) + cell_lo(hi, a.box.nc[tid]) ) >> 1;
    }
    if (tid == 32) S.next = 0;
    group_sync<NT, 0>();
    // (b) warp 0: row offsets in the staging buffer and, when the region fits the buffer, the
    // bulk copies, one row per lane (a row is one slice, or two across the periodic seam:
    // cells before the one at x = 0, then the rest); warp 1: targets per target row (target
    // row tr = ty + by tz sits in region row (tz+1) nry + ty+1); the other warps: per target
    // cell tc = tr * ntc + i - 1 its descriptor, its targets and the size of its 27-cell list
    // (neighbour row q = 0..8 of target row tr is region row (tz + q/3) nry + ty + q%3)
    if (wid == 0) {
        const int v = lane < nr ? S.row_tot[lane] : 0;
        const int inc = warp_incl_scan(v, lane);
        if (lane < nr) S.row_base[lane] = inc - v;
        const int region = __shfl_sync(full, inc, 31);
        if (lane == 31) S.row_base[nr] = inc;
        const bool copy = !overflow && region > 0 && region <= CAP;
        if (lane == 0) {
            S.copied = copy;
            if (copy) {
                const uint32_t bar = smem_u32(&S.mbar);
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                             "r"((uint32_t)region * 16u) : "memory");
            }
        }
        __syncwarp();
        if (copy && lane < nr) {
            const uint32_t bar = smem_u32(&S.mbar);
            const uint4 *rec = (const uint4 *)a.rec;
            const int is = x0 == 0 ? 1 : (x1 == nx ? wn - 1 : wn);
            const uint32_t n0 = (uint32_t)S.seg_off[lane][is];
            const uint32_t n1 = (uint32_t)(S.seg_off[lane][wn] - S.seg_off[lane][is]);
            const uint32_t dst = (uint32_t)(inc - v);
            if (n0)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(&S.stage[dst])),
                    "l"(rec + S.cstart[lane][0]), "r"(n0 * 16u), "r"(bar)
                    : "memory");
            if (n1)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(&S.stage[dst + n0])),
                    "l"(rec + S.cstart[lane][is]), "r"(n1 * 16u), "r"(bar)
                    : "memory");
        }
    } else if (wid == 1) {
        int v = 0;
        if (lane < ntr) {
            const int tz = __float2int_rz(((float)lane + 0.5f) * inby);
            const int rt = (tz + 1) * nry + lane - tz * by + 1;
            v = S.seg_off[rt][wn - 1] - S.seg_off[rt][1];
        }
        const int inc = warp_incl_scan(v, lane);
        if (lane < ntr) S.tp[lane] = inc - v;
        if (lane == 31) S.tp[ntr] = inc;
    } else {
        for (int tc = tid - 64; tc < ncells; tc += NT - 64) {
            const int tr = __float2int_rz(((float)tc + 0.5f) * intc), i = tc - tr * ntc + 1;
            const int tz = __float2int_rz(((float)tr + 0.5f) * inby);
            const int rb = tz * nry + tr - tz * by;
            const int rt = rb + nry + 1;
            int tot = 0;
            for (int q = 0; q < 9; ++q) {
                const int r = rb + (q / 3) * nry + q % 3;
                tot += S.seg_off[r][i + 2] - S.seg_off[r][i - 1];
            }
            S.cinfo[tc] = (uint32_t)rt | (uint32_t)i << 8 | (uint32_t)rb << 16 | (uint32_t)tr << 24;
            S.cnt[tc] = S.seg_off[rt][i + 1] - S.seg_off[rt][i];
            S.fb[tc + 1] = tot;
        }
    }
    group_sync<NT, 0>();
    // (c) warp 0: offsets of the candidate lists and of the mask blocks (slots of 32
    // candidates x targets rounded up to 4) of the target cells; the staging decision
    if (wid == 0) {
        int fcarry = 0, mcarry = 0;
        for (int base = 0; base < ncells; base += 32) {
            const int tc = base + lane;
            const int len = tc < ncells ? S.fb[tc + 1] : 0;
            const int words = tc < ncells ? ((len + 31) >> 5) * ((S.cnt[tc] + 3) & ~3) : 0;
            const int fi = warp_incl_scan(len, lane), mi = warp_incl_scan(words, lane);
            if (tc < ncells) {
                S.fb[tc + 1] = fcarry + fi;
                S.mbase[tc] = mcarry + mi - words;
            }
            fcarry += __shfl_sync(full, fi, 31);
            mcarry += __shfl_sync(full, mi, 31);
        }
        if (lane == 0) {
            S.fb[0] = 0;
            const int region_n = S.row_base[nr];
            // (the candidate lists hold 16-bit shared addresses of the offsets: the buffer
            // sits at the start of the block's shared memory, far below 64 KB)
            S.staged = !overflow && region_n <= CAP && fcarry <= FCAP && mcarry <= MP && S.tp[ntr] <= TMX &&
                       smem_u32(&S.off[CAP]) <= 65536u;
        }
    }
    group_sync<NT, 0>();
    const int region_n = S.row_base[nr];
    const int T = S.tp[ntr];
    if (!S.staged) {
        // neighbourhood larger than the buffers (or an overflowing cell): per particle
        double Ufall = 0.0;
        for (int t = tid; t < T; t += NT) {
            int tr = 0;
            while (tr + 1 < ntr && t >= S.tp[tr + 1]) ++tr;
            const int rt = (tr / by + 1) * nry + tr % by + 1;
            const uint32_t g = S.cstart[rt][1] + (uint32_t)(t - S.tp[tr]);
            double U = 0.0;
            float F[3] = {0.f, 0.f, 0.f};
            if (!overflow) near_one_f32(a, g, F, U);
            float *Fn = (float *)a.Fn;
            Fn[g] = F[0]; Fn[a.stride + g] = F[1]; Fn[2 * (size_t)a.stride + g] = F[2];
            Ufall += U;
        }
        if (S.copied) mbar_wait0(smem_u32(&S.mbar), 20000);   // copies in flight land first
        release();
        warp_partial(Ufall, a.U_part, blk, tid, NT);
        return;
    }
    if (region_n == 0) {
        warp_partial(0.0, a.U_part, blk, tid, NT);
        return;
    }
    const uint32_t bar = smem_u32(&S.mbar);
    // (d) while the copies fly: the candidate lists of the target cells, rows q = 0..8 in
    // order, each row's cells i-1 .. i+1 in staging order; three cells per warp at a time,
    // nine lanes per cell (one per row, each writing its row's stretch)
    {
        const int grp = lane / 9, q = lane - 9 * grp;
        for (int tc0 = 3 * wid; tc0 < ncells; tc0 += 3 * NW) {
            const int tc = tc0 + grp;
            const bool act = grp < 3 && tc < ncells;
            int n = 0, a0 = 0, r = 0;
            if (act) {
                const uint32_t ci = S.cinfo[tc];
                const int i = (int)((ci >> 8) & 0xffu), rb = (int)((ci >> 16) & 0xffu);
                r = rb + (q / 3) * nry + q % 3;
                a0 = S.seg_off[r][i - 1];
                n = S.seg_off[r][i + 2] - a0;
            }
            int inc = n;                                     // prefix within the nine lanes
#pragma unroll
            for (int o = 1; o < 9; o <<= 1) {
                const int v = __shfl_up_sync(full, inc, o);
                if (q >= o) inc += v;
            }
            if (act) {
                const int pos = S.fb[tc] + inc - n;
                const uint32_t oa = smem_u32(&S.off[S.row_base[r] + a0]);
                for (int l = 0; l < n; ++l) S.flat[pos + l] = (uint16_t)(oa + 16u * (uint32_t)l);
            }
        }
    }
    // bounded wait for the staged bytes (phase 0, at most about 2 s), made block-uniform
    uint32_t done = mbar_wait0(bar, 20000);
    if (!group_sync_and<NT, 0>((int)done)) {
        if (tid == 0) atomicOr(&a.ctr->err, kErrNearStage);
        if (!done) done = mbar_wait0(bar, 20000);     // let the copies in flight land
        release();
        warp_partial(0.0, a.U_part, blk, tid, NT);
        return;
    }
    // (e) FP32 offsets from the brick centre.  The region spans at most the box on each
    // axis (W <= nx - 2, by <= ny - 2, bz <= nz - 2), so offsets from the centre taken
    // modulo 2^32 are the exact fixed-point differences, rounded once to FP32.
    const float sx = a.box.L_2m32f[0], sy = a.box.L_2m32f[1], sz = a.box.L_2m32f[2];
    {
        const uint32_t rx = (uint32_t)S.ref[0], ry = (uint32_t)S.ref[1], rz = (uint32_t)S.ref[2];
        for (int e = tid; e < region_n; e += NT) {
            const uint4 p = S.stage[e];
            const float X = (float)(int)(p.x - rx) * sx, Y = (float)(int)(p.y - ry) * sy,
                        Z = (float)(int)(p.z - rz) * sz;
            S.off[e] = make_float4(X, Y, Z, -0.5f * fmaf(X, X, fmaf(Y, Y, Z * Z)));
        }
    }
    group_sync<NT, 0>();
    const float rc2 = a.nc.rc2_f;
    // Pre-filter: accept candidate c of target t when t.c - |c|^2/2 > (|t|^2 - thr)/2, which
    // is |t - c|^2 < thr, with thr = r_c^2 (1 + 1e-3).  Offsets from the centre are at most
    // (MW/2 + 1) c = 9 c along x and 3 c along y and z (c < 4/3 r_c, the cell width, as
    // n_c = floor(L / r_c) >= 3), each within 2.4e-7 of its size after two roundings; the
    // ten roundings of the test's terms (each at most 150 c^2) and the offsets' own errors
    // move the decision by less than 4e-4 r_c^2 in r^2, so every pair that the exact test
    // accepts passes.
    static_assert(MW <= 16, "pre-filter margin");
    const float hthr = 0.5f * (rc2 * 1.001f);
    const uint32_t flat_s = smem_u32(S.flat);
    // (f) pre-filter, target cells taken by the warps in turn; the cell's targets in chunks
    // of 8 (two groups of 4 mask columns), a chunk of at most 4 with half the work.  Each cell
    // also records its targets' descriptors.
    while (true) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&S.next, 1);
        c = __shfl_sync(full, c, 0);
        if (c >= ncells) break;
        const uint32_t ci = S.cinfo[c];
        const int rt = (int)(ci & 0xffu), i = (int)((ci >> 8) & 0xffu), tr = (int)(ci >> 24);
        const int ts = S.row_base[rt] + S.seg_off[rt][i];                   // first target, staged
        const int nt = S.cnt[c];
        const int f0 = S.fb[c], len = S.fb[c + 1] - f0;
        const int nsl = (len + 31) >> 5;
        const uint32_t kRowBytes = 4u * (uint32_t)((nt + 3) & ~3);        // bytes between mask slots
        const int tbase = S.tp[tr] + S.seg_off[rt][i] - S.seg_off[rt][1];    // its brick index
        for (int k = lane; k < nt; k += 32)
            S.tinfo[tbase + k] = make_uint2(S.cstart[rt][i] + (uint32_t)k,
                                            (uint32_t)(ts + k) | ((uint32_t)c << 12) | ((uint32_t)k << 20));
        const uint32_t mcol = smem_u32(&S.mpool[S.mbase[c]]);
        for (int t0 = 0; t0 < nt; t0 += 8) {
            const int nct = min(8, nt - t0);
            // the chunk's targets, two per packed register: x, y, z and the bound
            // (|t|^2 - thr)/2 = -h - thr/2 (h = -|t|^2/2); past the chunk, its last target
            unsigned long long TX[4], TY[4], TZ[4], TK[4];
#pragma unroll
            for (int pr = 0; pr < 4; ++pr) {
                const float4 ta = S.off[ts + t0 + min(2 * pr, nct - 1)];
                const float4 tb = S.off[ts + t0 + min(2 * pr + 1, nct - 1)];
                TX[pr] = pk2(ta.x, tb.x);
                TY[pr] = pk2(ta.y, tb.y);
                TZ[pr] = pk2(ta.z, tb.z);
                TK[pr] = pk2(-ta.w - hthr, -tb.w - hthr);
            }
            uint32_t ma = mcol + 4u * (uint32_t)t0;
            // a lane past the list tests its last candidate with h = -inf: never above
            const uint32_t fl = flat_s + 2u * (uint32_t)(f0 + len - 1);
            uint32_t fa = flat_s + 2u * (uint32_t)(f0 + lane);
            // NPR packed pairs of target columns per slot: 2 for at most 4 targets, 3 for 5 or
            // 6, 4 for more; the two words past 6 columns stay zero (no target reads them)
            auto slots = [&](auto npr_c) {
                constexpr int NPR = decltype(npr_c)::value;
                for (int s = 0; s < nsl; ++s, ma += kRowBytes, fa += 64u) {
                    const float4 cf = lds_f4(lds_u16(min(fa, fl)));
                    const float h = fa <= fl ? cf.w : -3e38f;
                    const unsigned long long X2 = pk2(cf.x, cf.x), Y2 = pk2(cf.y, cf.y), Z2 = pk2(cf.z, cf.z),
                                             H2 = pk2(h, h);
                    uint32_t m[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
                    for (int pr = 0; pr < NPR; ++pr) {
                        float va, vb, ka, kb;
                        upk2(fma2(Z2, TZ[pr], fma2(Y2, TY[pr], fma2(X2, TX[pr], H2))), va, vb);
                        upk2(TK[pr], ka, kb);
                        m[2 * pr] = __ballot_sync(full, va > ka);
                        m[2 * pr + 1] = __ballot_sync(full, vb > kb);
                    }
                    sts4_lane0(lane, ma, m[0], m[1], m[2], m[3]);
                    if (NPR > 2) sts4_lane0(lane, ma + 16u, m[4], m[5], m[6], m[7]);
                }
            };
            if (nct > 6) slots(std::integral_constant<int, 4>{});
            else if (nct > 4) slots(std::integral_constant<int, 3>{});
            else slots(std::integral_constant<int, 2>{});
        }
    }
    group_sync<NT, 0>();
    // (g) pairs, one thread per target
    float *Fn = (float *)a.Fn;
    const unsigned long long sx2 = dup2(sx), sy2 = dup2(sy), sz2 = dup2(sz);
    constexpr uint32_t kStageBack = 16u * CAP;                   // stage[i] = off[i] - kStageBack
    float sumU = 0.f;
    for (int wlo = 32 * wid; wlo < T; wlo += NT) {
        const int t = wlo + lane;
        const bool has = t < T;
        const uint2 tinf = S.tinfo[has ? t : wlo];
        const int j = (int)(tinf.y & 0xfffu), tc = (int)((tinf.y >> 12) & 0xffu), kk = (int)(tinf.y >> 20);
        const uint32_t fbase = flat_s + 2u * (uint32_t)S.fb[tc];
        const int nsl = has ? (S.fb[tc + 1] - S.fb[tc] + 31) >> 5 : 0;
        const uint32_t *mrow = &S.mpool[S.mbase[tc] + kk];       // its masks, one per slot
        const int mstride = (S.cnt[tc] + 3) & ~3;
        const uint32_t jo = smem_u32(&S.off[j]);                 // the target's own entry
        const uint4 ri = S.stage[j];
        const float qi = __uint_as_float(ri.w);
        unsigned long long Fxy = 0ull, Cxy = 0ull, Fzu = 0ull, Czu = 0ull;
        uint32_t m = 0;
        int s = -1;
        while (true) {
            uint32_t kA = 0, kB = jo;
            while (m == 0 && ++s < nsl) m = mrow[s * mstride];
            if (m == 0) break;
            kA = lds_u16(fbase + 2u * (uint32_t)(32 * s + __ffs(m) - 1));
            m &= m - 1;
            while (m == 0 && ++s < nsl) m = mrow[s * mstride];
            if (m != 0) {
                kB = lds_u16(fbase + 2u * (uint32_t)(32 * s + __ffs(m) - 1));
                m &= m - 1;
            }
            const uint4 pa = lds_u4(kA - kStageBack), pb = lds_u4(kB - kStageBack);
            const unsigned long long d0 = mul2(pk2((float)(int)(ri.x - pa.x), (float)(int)(ri.x - pb.x)), sx2);
            const unsigned long long d1 = mul2(pk2((float)(int)(ri.y - pa.y), (float)(int)(ri.y - pb.y)), sy2);
            const unsigned long long d2 = mul2(pk2((float)(int)(ri.z - pa.z), (float)(int)(ri.z - pb.z)), sz2);
            float a0, b0, a1, b1, a2, b2, r2a, r2b;
            upk2(d0, a0, b0);
            upk2(d1, a1, b1);
            upk2(d2, a2, b2);
            upk2(fma2(d2, d2, fma2(d1, d1, mul2(d0, d0))), r2a, r2b);
            const bool va = kA != jo && r2a < rc2, vb = kB != jo && r2b < rc2;
            // a pass slot without a pair: zero charge product at a finite r^2
            unsigned long long g2, u2;
            pair_terms2(nf, pk2(va ? qi * __uint_as_float(pa.w) : 0.f, vb ? qi * __uint_as_float(pb.w) : 0.f),
                        pk2(va ? r2a : rc2, vb ? r2b : rc2), g2, u2);
            float ga, gb, ua, ub;
            upk2(g2, ga, gb);
            upk2(u2, ua, ub);
            kahan2(Fxy, Cxy, fma2(dup2(ga), pk2(a0, a1), mul2(dup2(gb), pk2(b0, b1))));
            kahan2(Fzu, Czu, fma2(pk2(ga, 1.f), pk2(a2, ua), mul2(pk2(gb, 1.f), pk2(b2, ub))));
        }
        if (has) {
            const uint32_t g = tinf.x;
            float fx, fy, fz, us, cx, cy, cz_, uc;
            upk2(Fxy, fx, fy);
            upk2(Cxy, cx, cy);
            upk2(Fzu, fz, us);
            upk2(Czu, cz_, uc);
            Fn[g] = fx - cx;
            Fn[a.stride + g] = fy - cy;
            Fn[2 * (size_t)a.stride + g] = fz - cz_;
            sumU += 0.5f * (us - uc);        // each pair counted from both ends
        }
    }
    release();
    warp_partial((double)sumU, a.U_part, blk, tid, NT);
}

static_assert(kNearBrickThreads == 256, "brick CTA");
constexpr int kBrickThreads = kNearBrickThreads, kBrickCap = 1216, kBrickFCap = 7680, kBrickMW = 16, kBrickBY = 2, kBrickBZ = 4,
              kBrickTmax = 288, kBrickMaskWords = 2560;
using BrickSmemSingle =
    BrickSmem<kBrickCap, kBrickFCap, kBrickThreads, kBrickMW, kBrickBY, kBrickBZ, kBrickTmax, kBrickMaskWords>;
// three bricks per SM: 3 x (size + 1 KB reserved per block) within the SM's 228 KB
static_assert(sizeof(BrickSmemSingle) + 1024 <= 228 * 1024 / 3, "three bricks per SM");
__global__ void __launch_bounds__(kBrickThreads, 3)
    k_near_bricks(const __grid_constant__ NearArgs a, const __grid_constant__ NearF nf, NearBatchGeom g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    near_brick_body(a, nf, g, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                    blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                    *reinterpret_cast<BrickSmemSingle *>(smem_raw), (int)threadIdx.x);
}

// FP64 build: the same tiles with the 32-byte records (the staging buffer holds 1280 of
// them, 40 KB); the pre-filter takes the high 32 bits of the coordinates, the pairs the full
// 2^64 fixed point and FP64 arithmetic.
using TileSmem64 = TileSmem<kNearCapSingle, kTileThreads, kNearMaxWSingle, true>;
__global__ void __launch_bounds__(kTileThreads, 4) k_near_tiled64(NearArgs a, int W, int tiles_x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    near_tile_body<kNearCapSingle, kTileThreads, kNearMaxWSingle, true>(
        a, W, tiles_x, blockIdx.x, *reinterpret_cast<TileSmem64 *>(smem_raw), (int)threadIdx.x);
}

// Batched systems: block -> (system, its brick); a system of fewer than 3 cells on an axis
// runs the per-particle path (its first global record index in geom.W).  The system's pair
// constants are copied to shared memory.
__device__ __forceinline__ void near_batch_block(const NearArgs &a, const NearF &nfg, const NearBatchGeom &g,
                                                 unsigned blk, BrickSmemSingle &S, int tid) {
    if (g.tiled) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&nfg);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&S.nf);
        for (int i = tid; i < (int)(sizeof(NearF) / 4); i += kBrickThreads) dst[i] = src[i];
        const int bx = (int)(blk % (unsigned)g.tiles_x);
        const int rest = (int)(blk / (unsigned)g.tiles_x);
        near_brick_body(a, S.nf, g, bx, rest % g.tiles_y, rest / g.tiles_y, blk, S, tid);
    } else {
        near_global_block<1>(a, (uint32_t)g.W, blk, tid, kBrickThreads);
    }
}

__global__ void __launch_bounds__(kBrickThreads, 3) k_near_batch(const NearArgs *args, const NearF *nf,
                                                                 const NearBatchGeom *geom, const uint32_t *items,
                                                                 int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    near_batch_block(args[lo], nf[lo], geom[lo], blockIdx.x - items[lo], *reinterpret_cast<BrickSmemSingle *>(smem_raw),
                     (int)threadIdx.x);
}

}  // namespace

void near_geometry(const Box &box, uint32_t N, int *tiled, int *W, int *tiles_x, uint32_t *nblocks, double target,
                   int cap, int threads, int max_w) {
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    if (nx >= 3 && ny >= 3 && nz >= 3) {
        // tile width: about `target` (default 110) targets per CTA and about 1000 staged
        // particles on average (the staging buffer holds 1280, so Poisson fluctuations
        // rarely overflow it)
        const double occ = (double)N / (double)box.ncell;
        int Wt = (int)(target / (occ > 1e-9 ? occ : 1e-9));
        int Wcap = (int)(0.78 * cap / (9.0 * (occ > 1e-9 ? occ : 1e-9))) - 2;
        if (Wt > Wcap) Wt = Wcap;
        if (Wt > max_w) Wt = max_w;
        // at most nx - 2 cells, so that a tile's two halo cells are distinct from its own
        if (Wt > nx - 2) Wt = nx - 2;
        if (Wt < 1) Wt = 1;
        *tiles_x = (nx + Wt - 1) / Wt;
        *W = (nx + *tiles_x - 1) / *tiles_x;
        *tiled = 1;
        *nblocks = (uint32_t)(*tiles_x) * (uint32_t)ny * (uint32_t)nz;
    } else {
        *tiled = 0;
        *W = 0;
        *tiles_x = 0;
        *nblocks = blocks_for(N, (unsigned)threads);
    }
}

static void set_tile_smem_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_near_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BrickSmemSingle));
        cudaFuncSetAttribute(k_near_tiled64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem64));
        cudaFuncSetAttribute(k_near_bricks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BrickSmemSingle));
        done = true;
    }
}

// The FP32 pair constants of the tiled kernels, each duplicated into both halves of a
// 64-bit word for packed FP32x2 arithmetic.
static unsigned long long dup2_host(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return ((unsigned long long)b << 32) | b;
}
NearF near_f32_consts(const NearConsts &c) {
    NearF f;
    std::memset(&f, 0, sizeof(f));
    f.mtot = c.mtot;
    f.two = c.two;
    f.nl2 = dup2_host(-c.inv_lam_log2e_f);
    f.il2 = dup2_host(c.inv_lam_f);
    f.ly1 = dup2_host(c.ly1_f);
    f.nl2b = dup2_host(-c.inv_lam2_log2e_f);
    f.il2b = dup2_host(c.inv_lam2_f);
    f.ly2 = dup2_host(c.ly2_f);
    f.sg2 = dup2_host(c.sgn2_f);
    for (int g = 0; g < c.mtot; ++g) {
        f.nb[g] = dup2_host(-c.bl2f[g]);
        f.naf[g] = dup2_host(-c.af[g]);
        f.cf[g] = dup2_host(c.cf[g]);
    }
    return f;
}

// Bricks of one system (at least 3 cells per axis): about `target` targets per brick, the
// staged region and the candidate lists within 0.88 and 0.87 of their buffers on average,
// which leaves about four standard deviations of room.
uint32_t near_bricks(const Box &box, uint32_t N, double target, NearBatchGeom *g) {
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    *g = NearBatchGeom{};
    if (nx < 3 || ny < 3 || nz < 3) return 0;
    g->tiled = 1;
    g->by = std::min(kBrickBY, ny - 2);
    g->bz = std::min(kBrickBZ, nz - 2);
    double occ = (double)N / (double)box.ncell;
    if (occ < 1e-9) occ = 1e-9;
    const double tr = (double)(g->by * g->bz);
    int W = (int)(std::min(target, 0.9 * kBrickThreads) / (tr * occ) + 0.5);
    W = std::min(W, (int)(0.88 * kBrickCap / ((g->by + 2) * (g->bz + 2) * occ)) - 2);
    W = std::min(W, (int)(0.87 * kBrickFCap / (tr * 27.0 * occ)));
    W = std::min(std::min(W, kBrickMW), nx - 2);
    if (W < 1) W = 1;
    g->tiles_x = (nx + W - 1) / W;
    g->W = (nx + g->tiles_x - 1) / g->tiles_x;
    g->tiles_y = (ny + g->by - 1) / g->by;
    g->tiles_z = (nz + g->bz - 1) / g->bz;
    return (uint32_t)g->tiles_x * (uint32_t)g->tiles_y * (uint32_t)g->tiles_z;
}

int launch_near(int prec, const NearArgs &a, cudaStream_t st) {
    int tiled, W, tiles_x;
    uint32_t nb;
    near_geometry(a.box, a.N, &tiled, &W, &tiles_x, &nb);
    if (prec == 1 && tiled) {
        set_tile_smem_attr();
        NearBatchGeom g;
        nb = near_bricks(a.box, a.N, kNearBrickTarget, &g);
        k_near_bricks<<<dim3(g.tiles_x, g.tiles_y, g.tiles_z), kBrickThreads, sizeof(BrickSmemSingle), st>>>(
            a, near_f32_consts(a.nc), g);
        return (int)nb * (kBrickThreads / 32);
    }
    if (prec == 0 && tiled) {
        set_tile_smem_attr();
        k_near_tiled64<<<nb, kTileThreads, sizeof(TileSmem64), st>>>(a, W, tiles_x);
        return (int)nb * kWarpsPerBlock;
    }
    nb = blocks_for(a.N, kGlobalThreads);
    if (prec == 1) k_near_global<1><<<nb, kGlobalThreads, 0, st>>>(a);
    else k_near_global<0><<<nb, kGlobalThreads, 0, st>>>(a);
    return (int)nb * kWarpsPerBlock;
}

void launch_near_batch(const NearArgs *args, const NearF *nf, const NearBatchGeom *geom, const uint32_t *items,
                       int R, uint32_t nblocks, cudaStream_t st) {
    set_tile_smem_attr();
    k_near_batch<<<nblocks, kBrickThreads, sizeof(BrickSmemSingle), st>>>(args, nf, geom, items, R);
}

}  // namespace rbsog
