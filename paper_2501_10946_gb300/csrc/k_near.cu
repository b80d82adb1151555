// Near field of the RBSOG force step: Eq. (55) first term with F_N1 and F_N2 of
// Eqs. (56)-(57), and U_N of Eq. (50), over the particles within r_c (minimum image).
//
// FP32 build, cells >= 3 per axis: k_near_tiled.  One CTA owns a run of W cells along x
// in one (y, z) row.  Their 27-cell neighbourhood is 9 rows of W + 2 cells, and each such
// row is one (or, across the periodic seam, two) contiguous slices of the cell-sorted
// 16-byte particle records, so the CTA stages the whole neighbourhood in shared memory
// with TMA bulk copies completing on one mbarrier.  Each target particle then
//   (1) tests its 27 cells with exact fixed-point differences (r^2 < r_c^2) and lists
//       the hits by staging index, and
//   (2) evaluates the pair force on the listed candidates,
// with the list flushed at three points per target where the warp is converged (after
// rows 2, 5 and 8), so the expensive pair arithmetic runs on whole warps instead of
// diverging inside the candidate loop.  One 16-byte record per staged particle and a
// 32-entry list keep enough CTAs resident to hide latency.
// Otherwise (FP64 build, fewer than 3 cells on an axis, or a neighbourhood that does
// not fit the staging buffer): one thread per particle reading candidates from global
// memory.
#include <cuda_runtime.h>

#include "common.cuh"
#include "devmath.cuh"
#include "kernels.h"

namespace rbsog {
namespace {

constexpr int kGlobalThreads = 128;
constexpr int kTileThreads = 128;
constexpr int kListCap = 32;           // listed candidates per thread between flushes
constexpr int kMaxTileW = 48;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 pair constants of one system, copied to shared memory by each tiled CTA (a batch
// reads its systems' arguments from global memory, and the pair loop reads them per
// Gaussian).
struct NearF {
    int mtot;
    float inv_lam_log2e_f, inv_lam_f, rc2_f;
    float af[kMaxGauss], bl2f[kMaxGauss], cf[kMaxGauss];
};

// One FP32 pair: accumulate q_i q_j [F_N1 + F_N2](r) (r_i - r_j) and U_N/2 (compensated).
// C is NearConsts or NearF (the same float fields).
template <class C>
__device__ __forceinline__ void pair_f32(const C &nc, float qq, float d0, float d1, float d2, float r2,
                                         float *Fs, float *Fc, float &Us, float &Uc) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float e1 = ex2_approx(-r * nc.inv_lam_log2e_f);
    float fsog = 0.f, fn2 = 0.f;
    for (int g = 0; g < nc.mtot; ++g) {
        const float E = ex2_approx(-r2 * nc.bl2f[g]);
        fsog = fmaf(nc.af[g], E, fsog);
        fn2 = fmaf(nc.cf[g], E, fn2);
    }
    const float fn1 = e1 * (1.f + r * nc.inv_lam_f) * (rinv * rinv * rinv);
    const float gsc = qq * (fn1 + fn2);
    kahan_add(Fs[0], Fc[0], gsc * d0);
    kahan_add(Fs[1], Fc[1], gsc * d1);
    kahan_add(Fs[2], Fc[2], gsc * d2);
    kahan_add(Us, Uc, 0.5f * qq * (e1 * rinv - fsog));
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
                    if (r2 < a.nc.rc2) {
                        const double r = sqrt(r2);
                        const double rinv = 1.0 / r;
                        const double e1 = exp(-r * a.nc.inv_lam);
                        double fsog = 0.0, fn2 = 0.0;
                        for (int g = 0; g < a.nc.mtot; ++g) {
                            const double E = exp(-r2 * a.nc.b[g]);
                            fsog += a.nc.a[g] * E;
                            fn2 += a.nc.c[g] * E;
                        }
                        const double qq = ri.q * rj.q;
                        const double fn1 = e1 * (1.0 + r * a.nc.inv_lam) * (rinv * rinv * rinv);
                        const double gsc = qq * (fn1 + fn2);
                        F[0] += gsc * d[0];
                        F[1] += gsc * d[1];
                        F[2] += gsc * d[2];
                        U += 0.5 * qq * (e1 * rinv - fsog);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Fout[d] = F[d];
    Uout = U;
}

// Energy partials are per warp (4 per block, fixed order), so no block-wide barrier waits
// for the slowest thread at the end of a kernel.
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ void warp_partial(double v, double *U_part, unsigned blk) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) U_part[(size_t)blk * kWarpsPerBlock + (threadIdx.x >> 5)] = v;
}

// One block of the per-particle path: particles p0 + [0, 128) of this system (global
// record indices p0 .. p0 + N - 1).
template <int PREC>
__device__ __forceinline__ void near_global_block(const NearArgs &a, uint32_t p0, unsigned blk) {
    const uint32_t local = blk * blockDim.x + threadIdx.x;
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
    warp_partial(U, a.U_part, blk);
}

template <int PREC>
__global__ void __launch_bounds__(kGlobalThreads) k_near_global(NearArgs a) {
    near_global_block<PREC>(a, 0u, blockIdx.x);
}

// ---------------------------------------------------------------- tiled (TMA) FP32 path
// CAP: staged particles per CTA (16 B each).  One large system stages 1280 (7 CTAs per
// SM); batches of many systems stage 1024 (8 CTAs per SM), which measured faster there.
template <int CAP>
struct TileSmem {
    uint4 stage[CAP];                       // staged records
    uint16_t list[kListCap][kTileThreads];  // per-thread candidate lists (staging indices)
    NearF nf;                               // the system's FP32 pair constants
    int seg_off[9][kMaxTileW + 3];          // per row: offset of each region cell within the row
    int row_base[10];                       // per row: offset of the row in the staging buffer
    uint32_t chunk_g[9][2];                 // per row: global start of up to two slices
    uint32_t chunk_n[9][2];                 // per row: particle count of each slice
    unsigned long long mbar;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int CAP>
__device__ __forceinline__ void flush_list(const TileSmem<CAP> &S, const NearF &nc, const Box &box, int cnt,
                                           uint4 ri, float qi, float *Fs, float *Fc, float &Us, float &Uc) {
    for (int k = 0; k < cnt; ++k) {
        const uint4 rj = S.stage[S.list[k][threadIdx.x]];
        const float d0 = (float)(int)(ri.x - rj.x) * box.L_2m32f[0];
        const float d1 = (float)(int)(ri.y - rj.y) * box.L_2m32f[1];
        const float d2 = (float)(int)(ri.z - rj.z) * box.L_2m32f[2];
        pair_f32(nc, qi * __uint_as_float(rj.w), d0, d1, d2, d0 * d0 + d1 * d1 + d2 * d2, Fs, Fc, Us, Uc);
    }
}

template <int CAP>
__device__ __forceinline__ void near_tile_body(const NearArgs &a, int W, int tiles_x, unsigned blk,
                                               TileSmem<CAP> &S) {
    const int tid = threadIdx.x;
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const int tile = (int)(blk % (unsigned)tiles_x);
    const int rest = (int)(blk / (unsigned)tiles_x);
    const int cy = rest % ny, cz = rest / ny;
    const int x0 = tile * W;
    const int x1 = min(x0 + W, nx);
    const int wn = x1 - x0 + 2;                  // region cells per row: x0-1 .. x1
    const uint32_t *cs = a.cell_start;
    const bool overflow = (a.ctr->err & kErrCellOverflow) != 0;

    // cell populations of the 9 x wn region cells, loaded in parallel (row r: dz = r/3 - 1,
    // dy = r%3 - 1), then per-row prefix sums and global slices
    for (int e = tid; e < 9 * wn; e += kTileThreads) {
        const int r = e / wn, i = e - r * wn;
        const int yr = (cy + r % 3 - 1 + ny) % ny, zr = (cz + r / 3 - 1 + nz) % nz;
        int x = x0 - 1 + i;
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        const int c = x + nx * (yr + ny * zr);
        S.seg_off[r][i + 1] = (int)(cs[c + 1] - cs[c]);
    }
    if (tid == 0) {
        S.nf.mtot = a.nc.mtot;
        S.nf.inv_lam_log2e_f = a.nc.inv_lam_log2e_f;
        S.nf.inv_lam_f = a.nc.inv_lam_f;
        S.nf.rc2_f = a.nc.rc2_f;
    }
    for (int g = tid; g < a.nc.mtot; g += kTileThreads) {
        S.nf.af[g] = a.nc.af[g];
        S.nf.bl2f[g] = a.nc.bl2f[g];
        S.nf.cf[g] = a.nc.cf[g];
    }
    __syncthreads();
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
    __syncthreads();
    if (tid == 0) {
        int b = 0;
        for (int r = 0; r < 9; ++r) {
            S.row_base[r] = b;
            b += S.seg_off[r][wn];
        }
        S.row_base[9] = b;
    }
    __syncthreads();
    const int region_n = S.row_base[9];
    const bool staged = !overflow && region_n <= CAP;
    // center row (r = 4): targets are region cells 1 .. wn-2, contiguous in global memory
    const uint32_t g_first = cs[nx * (cy + ny * cz) + x0];
    const uint32_t g_end = cs[nx * (cy + ny * cz) + x1];

    float sumU = 0.f;
    double Ufall = 0.0;
    if (staged) {
        bool ok = true;
        if (region_n > 0) {
            const uint32_t bar = smem_u32(&S.mbar);
            if (tid == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                             "r"((uint32_t)region_n * 16u)
                             : "memory");
                const uint4 *rec = (const uint4 *)a.rec;
                for (int r = 0; r < 9; ++r) {
                    uint32_t dst = (uint32_t)S.row_base[r];
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t n = S.chunk_n[r][h];
                        if (n) {
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                                "[%3];" ::"r"(smem_u32(&S.stage[dst])),
                                "l"(rec + S.chunk_g[r][h]), "r"(n * 16u), "r"(bar)
                                : "memory");
                            dst += n;
                        }
                    }
                }
            }
            __syncthreads();
            // bounded wait for the staged bytes (phase 0); the outcome is made block-uniform
            uint32_t done = 0;
            for (int it = 0; it < (1 << 22) && !done; ++it) {
                asm volatile(
                    "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                    : "=r"(done)
                    : "r"(bar)
                    : "memory");
            }
            ok = __syncthreads_and((int)done) != 0;
            if (!ok) {
                if (tid == 0) atomicOr(&a.ctr->err, kErrNearStage);
                // let the copies in flight land before the CTA exits (again bounded)
                for (int it = 0; it < (1 << 22) && !done; ++it)
                    asm volatile(
                        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                        : "=r"(done)
                        : "r"(bar)
                        : "memory");
            }
        }
        if (ok) {
            const int t0 = S.row_base[4] + S.seg_off[4][1];
            const int t1 = S.row_base[4] + S.seg_off[4][wn - 1];
            float *Fn = (float *)a.Fn;
            const float rc2 = a.nc.rc2_f;
            for (int j = t0 + tid; j < t1; j += kTileThreads) {
                // region cell i (1 .. wn-2) holding target j: last i with seg_off[4][i] <= j - row_base[4]
                const int jl = j - S.row_base[4];
                int lo = 1, hi = wn - 2;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (S.seg_off[4][mid] <= jl) lo = mid;
                    else hi = mid - 1;
                }
                const int i = lo;
                const uint4 ri = S.stage[j];
                const float qi = __uint_as_float(ri.w);
                float Fs[3] = {0.f, 0.f, 0.f}, Fc[3] = {0.f, 0.f, 0.f}, Us = 0.f, Uc = 0.f;
                const float sx = a.box.L_2m32f[0], sy = a.box.L_2m32f[1], sz = a.box.L_2m32f[2];
                for (int r0 = 0; r0 < 9; r0 += 3) {
                    // filter: list the hits of three rows (the list keeps the first kListCap,
                    // the count keeps going); the loop holds no pair arithmetic
                    int cnt = 0;
                    for (int r = r0; r < r0 + 3; ++r) {
                        const int rb = S.row_base[r];
                        const int k0 = rb + S.seg_off[r][i - 1];
                        const int k1 = rb + S.seg_off[r][i + 2];
#pragma unroll 2
                        for (int k = k0; k < k1; ++k) {
                            const uint4 rk = S.stage[k];
                            const float d0 = (float)(int)(ri.x - rk.x) * sx;
                            const float d1 = (float)(int)(ri.y - rk.y) * sy;
                            const float d2 = (float)(int)(ri.z - rk.z) * sz;
                            if (d0 * d0 + d1 * d1 + d2 * d2 < rc2 && k != j) {
                                if (cnt < kListCap) S.list[cnt][tid] = (uint16_t)k;
                                ++cnt;
                            }
                        }
                    }
                    if (cnt <= kListCap) {
                        flush_list(S, S.nf, a.box, cnt, ri, qi, Fs, Fc, Us, Uc);
                    } else {
                        // rare: more hits than the list holds; evaluate the three rows
                        // directly, in the same candidate order
                        for (int r = r0; r < r0 + 3; ++r) {
                            const int rb = S.row_base[r];
                            const int k1 = rb + S.seg_off[r][i + 2];
                            for (int k = rb + S.seg_off[r][i - 1]; k < k1; ++k) {
                                const uint4 rk = S.stage[k];
                                const float d0 = (float)(int)(ri.x - rk.x) * sx;
                                const float d1 = (float)(int)(ri.y - rk.y) * sy;
                                const float d2 = (float)(int)(ri.z - rk.z) * sz;
                                if (d0 * d0 + d1 * d1 + d2 * d2 < rc2 && k != j)
                                    pair_f32(S.nf, qi * __uint_as_float(rk.w), d0, d1, d2,
                                             d0 * d0 + d1 * d1 + d2 * d2, Fs, Fc, Us, Uc);
                            }
                        }
                    }
                }
                const uint32_t g = g_first + (uint32_t)(j - t0);
                Fn[g] = Fs[0] - Fc[0];
                Fn[a.stride + g] = Fs[1] - Fc[1];
                Fn[2 * (size_t)a.stride + g] = Fs[2] - Fc[2];
                sumU += Us - Uc;
            }
        }
    } else {
        // neighbourhood larger than the staging buffer (or an overflowing cell): global path
        float *Fn = (float *)a.Fn;
        for (uint32_t g = g_first + tid; g < g_end; g += kTileThreads) {
            float F[3] = {0.f, 0.f, 0.f};
            double U = 0.0;
            if (!overflow) near_one_f32(a, g, F, U);
            Fn[g] = F[0]; Fn[a.stride + g] = F[1]; Fn[2 * (size_t)a.stride + g] = F[2];
            Ufall += U;
        }
    }
    warp_partial((double)sumU + Ufall, a.U_part, blk);
}

__global__ void __launch_bounds__(kTileThreads) k_near_tiled(NearArgs a, int W, int tiles_x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    near_tile_body<kNearCapSingle>(a, W, tiles_x, blockIdx.x, *reinterpret_cast<TileSmem<kNearCapSingle> *>(smem_raw));
}

// Batched systems: block -> (system, local block); each system uses tiles or the
// per-particle path as its geometry says.  geom.W doubles as the first global record
// index of the system for the per-particle path.
__global__ void __launch_bounds__(kTileThreads) k_near_batch(const NearArgs *args, const NearBatchGeom *geom,
                                                            const uint32_t *items, int R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const NearArgs &a = args[lo];
    const NearBatchGeom g = geom[lo];
    const unsigned blk = blockIdx.x - items[lo];
    if (g.tiled)
        near_tile_body<kNearCapBatch>(a, g.W, g.tiles_x, blk, *reinterpret_cast<TileSmem<kNearCapBatch> *>(smem_raw));
    else near_global_block<1>(a, (uint32_t)g.W, blk);
}

inline unsigned blocks_for(uint32_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void near_geometry(const Box &box, uint32_t N, int *tiled, int *W, int *tiles_x, uint32_t *nblocks, double target,
                   int cap) {
    const int nx = box.nc[0], ny = box.nc[1], nz = box.nc[2];
    if (nx >= 3 && ny >= 3 && nz >= 3) {
        // tile width: about `target` (default 110) targets per CTA and about 1000 staged
        // particles on average (the staging buffer holds 1280, so Poisson fluctuations
        // rarely overflow it)
        const double occ = (double)N / (double)box.ncell;
        int Wt = (int)(target / (occ > 1e-9 ? occ : 1e-9));
        int Wcap = (int)(0.78 * cap / (9.0 * (occ > 1e-9 ? occ : 1e-9))) - 2;
        if (Wt > Wcap) Wt = Wcap;
        if (Wt > kMaxTileW) Wt = kMaxTileW;
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
        *nblocks = blocks_for(N, kGlobalThreads);
    }
}

static void set_tile_smem_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_near_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileSmem<kNearCapSingle>));
        cudaFuncSetAttribute(k_near_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileSmem<kNearCapBatch>));
        done = true;
    }
}

int launch_near(int prec, const NearArgs &a, cudaStream_t st) {
    int tiled, W, tiles_x;
    uint32_t nb;
    near_geometry(a.box, a.N, &tiled, &W, &tiles_x, &nb);
    if (prec == 1 && tiled) {
        set_tile_smem_attr();
        k_near_tiled<<<nb, kTileThreads, sizeof(TileSmem<kNearCapSingle>), st>>>(a, W, tiles_x);
        return (int)nb * kWarpsPerBlock;
    }
    nb = blocks_for(a.N, kGlobalThreads);
    if (prec == 1) k_near_global<1><<<nb, kGlobalThreads, 0, st>>>(a);
    else k_near_global<0><<<nb, kGlobalThreads, 0, st>>>(a);
    return (int)nb * kWarpsPerBlock;
}

void launch_near_batch(const NearArgs *args, const NearBatchGeom *geom, const uint32_t *items, int R,
                       uint32_t nblocks, cudaStream_t st) {
    set_tile_smem_attr();
    k_near_batch<<<nblocks, kTileThreads, sizeof(TileSmem<kNearCapBatch>), st>>>(args, geom, items, R);
}

}  // namespace rbsog
