// Near field of the RBSOG force step: Eq. (55) first term with F_N1 and F_N2 of
// Eqs. (56)-(57), and U_N of Eq. (50), over the particles within r_c (minimum image).
//
// FP32 build, cells >= 3 per axis: k_near_tiled.  One CTA owns a run of W cells along x
// in one (y, z) row.  Their 27-cell neighbourhood is 9 rows of W + 2 cells, and each such
// row is one (or, across the periodic seam, two) contiguous slices of the cell-sorted
// 16-byte particle records, so the CTA stages the whole neighbourhood in shared memory
// with TMA bulk copies completing on one mbarrier.  Each target particle then
//   (1) filters its 27 cells with float coordinates relative to the tile (3 FADD per
//       candidate, permissive by 1e-4 in r^2) into a short per-thread list, and
//   (2) evaluates the pair force on the listed candidates from exact fixed-point
//       differences, applying the exact test r^2 < r_c^2,
// so the expensive pair arithmetic runs without the divergence of a fused loop.
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
constexpr int kRegionCap = 1536;       // staged particles per CTA (2 x 24 KB)
constexpr int kListCap = 64;           // listed candidates per thread before a flush
constexpr int kMaxTileW = 64;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One FP32 pair: accumulate q_i q_j [F_N1 + F_N2](r) (r_i - r_j) and U_N/2 (compensated).
__device__ __forceinline__ void pair_f32(const NearConsts &nc, float qq, float d0, float d1, float d2, float r2,
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

__device__ __forceinline__ double block_sum_128(double v, double *sh) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

template <int PREC>
__global__ void __launch_bounds__(kGlobalThreads) k_near_global(NearArgs a) {
    __shared__ double sh[kGlobalThreads / 32];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    double U = 0.0;
    if (p < a.N) {
        const bool overflow = (a.ctr->err & kErrCellOverflow) != 0;
        if (PREC == 1) {
            float F[3] = {0.f, 0.f, 0.f};
            if (!overflow) near_one_f32(a, p, F, U);
            float *Fn = (float *)a.Fn;
            Fn[p] = F[0]; Fn[a.N + p] = F[1]; Fn[2 * (size_t)a.N + p] = F[2];
        } else {
            double F[3] = {0.0, 0.0, 0.0};
            if (!overflow) near_one_f64(a, p, F, U);
            double *Fn = (double *)a.Fn;
            Fn[p] = F[0]; Fn[a.N + p] = F[1]; Fn[2 * (size_t)a.N + p] = F[2];
        }
    }
    const double tot = block_sum_128(U, sh);
    if (threadIdx.x == 0) a.U_part[blockIdx.x] = tot;
}

// ---------------------------------------------------------------- tiled (TMA) FP32 path
struct TileSmem {
    uint4 srec[kRegionCap];                 // staged records, 16-byte aligned
    float4 spos[kRegionCap];                // x, y, z relative to the tile origin, q
    uint16_t list[kListCap][kTileThreads];  // per-thread candidate lists (smem indices)
    int seg_off[9][kMaxTileW + 3];          // per row: offset of each region cell within the row
    int row_base[10];                       // per row: offset of the row in srec
    uint32_t chunk_g[9][2];                 // per row: global start of up to two slices
    uint32_t chunk_n[9][2];                 // per row: particle count of each slice
    unsigned long long mbar;
    double red[kTileThreads / 32];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void flush_list(const TileSmem &S, const NearConsts &nc, const Box &box, int cnt,
                                           uint4 ri, float qi, float *Fs, float *Fc, float &Us, float &Uc) {
    for (int k = 0; k < cnt; ++k) {
        const uint4 rj = S.srec[S.list[k][threadIdx.x]];
        const float d0 = (float)(int)(ri.x - rj.x) * box.L_2m32f[0];
        const float d1 = (float)(int)(ri.y - rj.y) * box.L_2m32f[1];
        const float d2 = (float)(int)(ri.z - rj.z) * box.L_2m32f[2];
        const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 < nc.rc2_f) pair_f32(nc, qi * __uint_as_float(rj.w), d0, d1, d2, r2, Fs, Fc, Us, Uc);
    }
}

__global__ void __launch_bounds__(kTileThreads) k_near_tiled(NearArgs a, int W, int tiles_x) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    const int tile = blockIdx.x % tiles_x;
    const int rest = blockIdx.x / tiles_x;
    const int cy = rest % ny, cz = rest / ny;
    const int x0 = tile * W;
    const int x1 = min(x0 + W, nx);
    const int wn = x1 - x0 + 2;                  // region cells per row: x0-1 .. x1
    const uint32_t *cs = a.cell_start;
    const bool overflow = (a.ctr->err & kErrCellOverflow) != 0;

    // per-row cell offsets and global slices (row r: dz = r/3 - 1, dy = r%3 - 1)
    if (tid < 9) {
        const int yr = (cy + tid % 3 - 1 + ny) % ny, zr = (cz + tid / 3 - 1 + nz) % nz;
        const int rowbase = nx * (yr + ny * zr);
        int off = 0;
        for (int i = 0; i < wn; ++i) {
            const int c = rowbase + (x0 - 1 + i + nx) % nx;
            S.seg_off[tid][i] = off;
            off += (int)(cs[c + 1] - cs[c]);
        }
        S.seg_off[tid][wn] = off;
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
    const bool staged = !overflow && region_n <= kRegionCap;
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
                                "[%3];" ::"r"(smem_u32(&S.srec[dst])),
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
            // float coordinates: unsigned fixed-point offsets from the lower corner of the
            // region's first cell (x0-1, cy-1, cz-1).  The region is a run of consecutive cells
            // that spans at most the whole periodic box, so every pair of neighbouring cells
            // lies on the same side of this frame's seam (a frame centred on the tile would put
            // its seam inside the region whenever W + 2 exceeds half the row).
            const uint32_t o0 = (uint32_t)((((unsigned long long)((x0 - 1 + nx) % nx)) << 32) / (unsigned)nx);
            const uint32_t o1 = (uint32_t)((((unsigned long long)((cy - 1 + ny) % ny)) << 32) / (unsigned)ny);
            const uint32_t o2 = (uint32_t)((((unsigned long long)((cz - 1 + nz) % nz)) << 32) / (unsigned)nz);
            for (int j = tid; j < region_n; j += kTileThreads) {
                const uint4 r = S.srec[j];
                S.spos[j] = make_float4((float)(r.x - o0) * a.box.L_2m32f[0], (float)(r.y - o1) * a.box.L_2m32f[1],
                                        (float)(r.z - o2) * a.box.L_2m32f[2], __uint_as_float(r.w));
            }
            __syncthreads();
            const float rc2_filter = a.nc.rc2_f * 1.0001f;
            const int t0 = S.row_base[4] + S.seg_off[4][1];
            const int t1 = S.row_base[4] + S.seg_off[4][wn - 1];
            float *Fn = (float *)a.Fn;
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
                const float4 pt = S.spos[j];
                const uint4 ri = S.srec[j];
                float Fs[3] = {0.f, 0.f, 0.f}, Fc[3] = {0.f, 0.f, 0.f}, Us = 0.f, Uc = 0.f;
                int cnt = 0;
                for (int r = 0; r < 9; ++r) {
                    const int k0 = S.row_base[r] + S.seg_off[r][i - 1];
                    const int k1 = S.row_base[r] + S.seg_off[r][i + 2];
                    for (int k = k0; k < k1; ++k) {
                        const float4 pk = S.spos[k];
                        const float dx = pt.x - pk.x, dy = pt.y - pk.y, dz = pt.z - pk.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < rc2_filter && k != j) {
                            S.list[cnt][tid] = (uint16_t)k;
                            if (++cnt == kListCap) {
                                flush_list(S, a.nc, a.box, cnt, ri, pt.w, Fs, Fc, Us, Uc);
                                cnt = 0;
                            }
                        }
                    }
                }
                flush_list(S, a.nc, a.box, cnt, ri, pt.w, Fs, Fc, Us, Uc);
                const uint32_t g = g_first + (uint32_t)(j - t0);
                Fn[g] = Fs[0] - Fc[0];
                Fn[a.N + g] = Fs[1] - Fc[1];
                Fn[2 * (size_t)a.N + g] = Fs[2] - Fc[2];
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
            Fn[g] = F[0]; Fn[a.N + g] = F[1]; Fn[2 * (size_t)a.N + g] = F[2];
            Ufall += U;
        }
    }
    const double tot = block_sum_128((double)sumU + Ufall, S.red);
    if (tid == 0) a.U_part[blockIdx.x] = tot;
}

inline unsigned blocks_for(uint32_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int launch_near(int prec, const NearArgs &a, cudaStream_t st) {
    const int nx = a.box.nc[0], ny = a.box.nc[1], nz = a.box.nc[2];
    if (prec == 1 && nx >= 3 && ny >= 3 && nz >= 3) {
        // tile width: about 110 targets per CTA and about 1200 staged particles
        const double occ = (double)a.N / (double)a.box.ncell;
        int Wt = (int)(110.0 / (occ > 1e-9 ? occ : 1e-9));
        int Wcap = (int)(1200.0 / (9.0 * (occ > 1e-9 ? occ : 1e-9))) - 2;
        if (Wt > Wcap) Wt = Wcap;
        if (Wt > kMaxTileW) Wt = kMaxTileW;
        if (Wt > nx - 2) Wt = nx - 2;
        if (Wt < 1) Wt = 1;
        const int tiles_x = (nx + Wt - 1) / Wt;
        const int W = (nx + tiles_x - 1) / tiles_x;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_near_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem));
            attr_set = true;
        }
        const int nb = tiles_x * ny * nz;
        k_near_tiled<<<nb, kTileThreads, sizeof(TileSmem), st>>>(a, W, tiles_x);
        return nb;
    }
    const unsigned nb = blocks_for(a.N, kGlobalThreads);
    if (prec == 1) k_near_global<1><<<nb, kGlobalThreads, 0, st>>>(a);
    else k_near_global<0><<<nb, kGlobalThreads, 0, st>>>(a);
    return (int)nb;
}

}  // namespace rbsog
