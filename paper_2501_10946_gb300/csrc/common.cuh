// Shared device-side definitions of the RBSOG force step (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rbsog {

constexpr int kMaxGauss = 40;        // Gaussians of the SOG far part the kernels accept
constexpr int kMaxCellOcc = 4096;    // particles per cell the cell sort accepts
constexpr int kScanTile = 4096;      // cells per scan tile (1024 threads x 4)
constexpr int kMaxAttempts = 1 << 20;

// error bits raised by kernels (device flag)
constexpr int kErrCellOverflow = 1;
constexpr int kErrSampler = 2;
constexpr int kErrNearStage = 4;     // a bounded wait for staged near-field data gave up

// Device counters that advance inside captured graphs.
struct DevCounters {
    unsigned long long step;    // steps taken since set_state
    unsigned long long draw;    // k-set draws so far
    int inject;                 // 1: the next k-set comes from the injected buffer
    int err;                    // error bits
    int fvalid;                 // 1: the forces of the current state have been evaluated
    int pad;
};

// Per-particle record staged by the near and far kernels.
// FP32 build: 16 bytes {s_x, s_y, s_z, q as float bits}, s = floor(frac(r/L) 2^32).
// FP64 build: 32 bytes {s_x, s_y, s_z (2^64 fixed point), q}.
struct __align__(16) Rec64 {
    unsigned long long s[3];
    double q;
};

// Constants of the near-field pair kernel (Eqs. 55-57) in both precisions.
// With E_m = exp(-r^2 b_m), b_m = e^{t_m}:
//   F(r)    = sum_m a_m E_m,                    a_m = h w_m f(t_m, 0)
//   F_N2(r) = sum_m c_m E_m,                    c_m = -2 b_m a_m
//   F_N1(r) = exp(-r/lambda)(1 + r/lambda)/r^3
// The Yukawa part is sum_i y_i exp(-r/lambda_i)/r over one term (y_1 = 1, the Yukawa
// kernel) or two (the EGS screening, y_1 > 0 > y_2); F_N1 and Y carry the same weights,
// and the Gaussians a_m, c_m already include their term's weight.
struct NearConsts {
    int mtot;
    double inv_lam;                    // 1/lambda_1
    double rc2;
    double a[kMaxGauss], b[kMaxGauss], c[kMaxGauss];
    float inv_lam_log2e_f;             // log2(e)/lambda_1
    float inv_lam_f;
    float rc2_f;
    float af[kMaxGauss], bl2f[kMaxGauss], cf[kMaxGauss];   // bl2f = b_m log2(e)
    double y1;                         // weight of the first term (1 for the Yukawa kernel)
    float ly1_f;                       // log2(y1): the FP32 path folds the weight into exp
    int two;                           // 1: a second Yukawa term
    double y2, inv_lam2;               // its weight and 1/lambda_2
    float ly2_f, sgn2_f;               // log2|y2| and the sign of y2
    float inv_lam2_log2e_f, inv_lam2_f;
};

// Yukawa terms of the interaction in Fourier space: 4 pi psi(k), psi(k) = sum_i c_i /
// (k^2 + lambda_i^-2); one term of weight 1 (Yukawa kernel) or two (EGS screening).
struct Yterms {
    int n;
    double c[2];
    double inv_lam2[2];
};

struct Box {
    double L[3];
    double invL[3];       // 1/L rounded to double (fixed point and wrap multiply by it)
    int nc[3];
    int ncell;
    double invL32[3];     // 2^32 / L (exact scaling of invL)
    double L_2m32[3];     // L / 2^32
    double L_2m64[3];     // L / 2^64
    float L_2m32f[3];
    double tpl[3];        // 2 pi / L
};

// State arrays (SoA). The same layout serves the "rest" buffer (cell-sorted order,
// between steps) and the "work" buffer (previous order, inside a step).
struct State {
    double *rx, *ry, *rz;
    double *vx, *vy, *vz;
    double *invm;
    double *q;
    uint32_t *id;        // caller's particle index
};

}  // namespace rbsog
