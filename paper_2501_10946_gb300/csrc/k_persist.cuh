// Persistent batched step: one cooperative launch advances every resident system by one
// step of Algorithm 2 (or evaluates their forces).  Included by k_all.cu after the kernel
// files, whose per-block bodies it calls.
//
// The grid (every CTA resident, 256 threads each) walks the phases of the step; between
// phases that depend on each other it meets at a grid barrier:
//   1  sample (every system's P modes) and bin (integrator first half, cells)
//   2  per-tile cell counts          3  scan -> cell_start
//   4  scatter of the sort keys      5  gather into the cell order
//   6  near field (one brick per CTA at a time) then the structure factor, both from work
//      counters that CTAs take items from as they finish
//   7  rho_final                      8  far gather + closing half kick
//   9  close (step counters, forces-valid flags)
// Each work item of a phase is a (system, local block) of the batched kernels, found
// through the same block-prefix arrays, so every item computes what the batched kernel's
// block computes.  Every barrier wait is bounded: a CTA that waits longer than wait_limit
// polls sets the status flag and returns, and the others give up at their next barrier.
#pragma once

namespace rbsog {

namespace {

constexpr int kPersistThreads = 256;
static_assert(kPersistThreads == kNearBrickThreads, "one near-field brick per CTA");

struct PersistSmem {
    union {
        BrickSmemSingle brick;
        uint4 rho_sp[kRhoTile];
        double2 rf_sh[8][32];
        struct {
            double shK[kFarThreads];
            GTab32 tab[kFarTile];
        } far;
        uint32_t scan_sh[16];
    } u;
    unsigned int item[2];
    int ok;
};

// Grid barrier with a bounded wait.  The last CTA to arrive resets the arrival count (and,
// when asked, the work counters of the next phase) before it opens the next generation.
__device__ __forceinline__ bool grid_barrier(GridBar *b, long long limit, bool reset_queues, PersistSmem &S) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = &b->gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&b->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            b->count = 0u;
            if (reset_queues) {
                b->q_near = 0u;
                b->q_rho = 0u;
            }
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long it = 0;
            while (*vgen == g0) {
                if (++it > limit) {
                    ok = 0;
                    atomicOr(&b->status, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int *)&b->status) ok = 0;
        S.ok = ok;
    }
    __syncthreads();
    return S.ok != 0;
}

__global__ void __launch_bounds__(kPersistThreads, 3) k_step_persist(PersistArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistSmem &S = *reinterpret_cast<PersistSmem *>(smem_raw);
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x;
    const long long lim = a.wait_limit;
    // 1: the k-sample (two 4-warp sample blocks per CTA) and binning
    {
        const int half = tid >> 7, w = (tid >> 5) & 3;
        for (unsigned vb = 2 * blockIdx.x + half; vb < a.nb_sample; vb += 2 * G) {
            const int r = item_system(a.it_sample, a.R, vb);
            const SampleArgs &sa = a.sample[r];
            const int l = (int)(vb - a.it_sample[r]) * 4 + w;
            if (l < sa.P) sample_warp(sa, l);
        }
        // items vb and vb + G together (two particles per thread: this grid runs 768
        // threads per SM, so each thread keeps two sets of loads in flight)
        for (unsigned vb = blockIdx.x; vb < a.nb_bin; vb += 2 * G) {
            const int r0 = item_system(a.it_bin, a.R, vb);
            const BinArgs &b0 = a.bin[r0];
            const uint32_t k0 = (vb - a.it_bin[r0]) * kPersistThreads + tid;
            const bool v0 = k0 < b0.N;
            bool v1 = false;
            uint32_t k1 = 0;
            int r1 = r0;
            if (vb + G < a.nb_bin) {
                r1 = item_system(a.it_bin, a.R, vb + G);
                k1 = (vb + G - a.it_bin[r1]) * kPersistThreads + tid;
                v1 = k1 < a.bin[r1].N;
            }
            if (v0 && v1) bin_two(b0, k0, a.bin[r1], k1);
            else if (v0) bin_body<1>(b0, k0);
            else if (v1) bin_body<1>(a.bin[r1], k1);
        }
    }
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 2, 3: scan of the cell counts
    for (int t = blockIdx.x; t < a.ntiles; t += G) tile_sum_256(a.count, a.ncell, a.tile_sums, t, S.u.scan_sh);
    if (!grid_barrier(a.bar, lim, false, S)) return;
    for (int t = blockIdx.x; t < a.ntiles; t += G)
        scan_tile_256(a.count, a.ncell, a.tile_sums, a.cell_start, a.N, t, a.ntiles, S.u.scan_sh);
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 4, 5: sort keys and the gather into the cell order
    for (uint32_t k = blockIdx.x * kPersistThreads + tid; k < a.N; k += G * kPersistThreads)
        scatter_one(a.cell, a.slot, a.cell_start, a.id, a.keys, k);
    if (!grid_barrier(a.bar, lim, true, S)) return;
    {
        const uint32_t stride = G * kPersistThreads;
        for (uint32_t i = blockIdx.x * kPersistThreads + tid; i < a.N; i += 2 * stride) {
            if (i + stride < a.N) gather_two(a.gather, i, i + stride);
            else gather_one<1>(a.gather, i);
        }
    }
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 6: near field, then the structure factor
    while (true) {
        if (tid == 0) S.item[0] = atomicAdd(&a.bar->q_near, 1u);
        __syncthreads();
        const unsigned vb = S.item[0];
        __syncthreads();
        if (vb >= a.nb_near) break;
        const int r = item_system(a.it_near, a.R, vb);
        const NearBatchGeom g = a.geom[r];
        const unsigned blk = vb - a.it_near[r];
        if (g.tiled) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&a.nearf[r]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&S.u.brick.nf);
            for (int i = tid; i < (int)(sizeof(NearF) / 4); i += kPersistThreads) dst[i] = src[i];
            const int bx = (int)(blk % (unsigned)g.tiles_x);
            const int rest = (int)(blk / (unsigned)g.tiles_x);
            near_brick_body<kBrickCap, kBrickFCap, kBrickThreads, kBrickMW, kBrickBY, kBrickBZ, kBrickTmax,
                            kBrickMaskWords, true>(a.near[r], S.u.brick.nf, g, bx, rest % g.tiles_y,
                                                   rest / g.tiles_y, blk, S.u.brick, tid);
        } else {
            near_global_block<1>(a.near[r], (uint32_t)g.W, blk, tid, kPersistThreads);
        }
    }
    __syncthreads();
    while (true) {
        if (tid == 0) S.item[0] = atomicAdd(&a.bar->q_rho, 1u);
        __syncthreads();
        const unsigned vb = S.item[0];
        __syncthreads();
        if (vb >= a.nb_rho) break;
        const int r = item_system(a.it_rho, a.R, vb);
        const RhoArgs &ra = a.rho[r];
        const unsigned local = vb - a.it_rho[r];
        rho32_body<1>(ra, a.chunk[r], local % (unsigned)ra.G, local / (unsigned)ra.G, S.u.rho_sp);
    }
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 7: rho, U*_F terms, gather tables; each system's first block advances its draw counter
    for (unsigned vb = blockIdx.x; vb < a.nb_rf; vb += G) {
        const int r = item_system(a.it_rf, a.R, vb);
        rho_final_body<1>(a.rf[r], 1, vb - a.it_rf[r], vb == a.it_rf[r], S.u.rf_sh);
        __syncthreads();
    }
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 8: far force, total force, closing half kick
    for (unsigned vb = blockIdx.x; vb < a.nb_far; vb += G) {
        const int r = item_system(a.it_far, a.R, vb);
        far32_body(a.far[r], vb - a.it_far[r], S.u.far.tab, S.u.far.shK);
    }
    if (!grid_barrier(a.bar, lim, false, S)) return;
    // 9: close of the evaluation
    if (blockIdx.x == 0)
        for (int r = tid; r < a.R; r += kPersistThreads) {
            if (a.advance && a.ctr[r].fvalid) a.ctr[r].step += 1ull;
            a.ctr[r].fvalid = 1;
        }
}

}  // namespace

size_t persist_smem_bytes() { return sizeof(PersistSmem); }

int persist_grid(int device, int *grid) {
    static int cached_dev = -1, cached = 0;
    if (cached_dev == device) {
        *grid = cached;
        return 0;
    }
    const int smem = (int)sizeof(PersistSmem);
    cudaError_t e = cudaFuncSetAttribute(k_step_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persist, kPersistThreads, smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    cached_dev = device;
    cached = per_sm * sms;
    *grid = cached;
    return 0;
}

cudaError_t launch_step_persist(const PersistArgs &a, int grid, cudaStream_t st) {
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_step_persist, dim3(grid), dim3(kPersistThreads), args,
                                       sizeof(PersistSmem), st);
}

}  // namespace rbsog
