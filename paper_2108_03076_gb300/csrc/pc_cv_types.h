// pc_cv_types.h -- the control-variate kernels' device arguments (CvArgs)
// and sizes: the part of pc_cv.h that the run-time compiler also sees.
#pragma once

#include "pc_types.h"

namespace pc {

constexpr int kCvMaxDates = 32;   // observation dates of the template
constexpr int kCvMaxD = 3;        // underlyings
constexpr int kCvFeatures = 16;   // network inputs
constexpr int kCvOutputs = 5;     // network outputs: value, up to 4 hedge ratios
// floats of a table node: hedge ratios 0..2, then the slopes d Delta_i / d u_j
// at 3 + 3 i + j (u: the grid coordinate; zero beyond d)
constexpr int kCvRecord = 12;

struct CvArgs {
  const float *tables;            // [(n-1) * 2][nodes][kCvRecord], 16-byte aligned
  int32_t d, n, grid, nodes;      // nodes = grid^d
  float ref[kCvMaxD];
  float call_level, ki_level, coupon;
  float lo[kCvMaxDates][kCvMaxD], h[kCvMaxDates][kCvMaxD];  // row k-1: date k
  // u = log2(S) * ua - ub = (ln S - lo) / h: ua = ln 2 / h, ub = lo / h
  float ua[kCvMaxDates][kCvMaxD], ub[kCvMaxDates][kCvMaxD];
  float inv_h[kCvMaxDates][kCvMaxD];
  // second-order term: cq[k][i*3+j] = exp(rho_ij sigma_i sigma_j (tau_{k+1} - tau_k)) - 1
  float cq[kCvMaxDates][kCvMaxD * kCvMaxD];
  float inv_ref[kCvMaxD];
  float delta0[kCvMaxD];
  const float *delta0_dev;         // non-null: delta0 read from the device instead
  float beta, beta2;              // Y = X - beta M - beta2 M2
  int32_t use_gamma;              // add the second-order term M2
  int32_t pilot;                  // 1: sums of X, M, M2 and their products (8), else X, X^2, Y, Y^2
};

// Template and model inputs of the network that are the same for every
// table node.
struct CvFeatureArgs {
  float ln_spot[kCvMaxD];
  float sigma[kCvMaxD];
  float rho, r;
  float tau[kCvMaxDates + 1];     // year fractions of ordinals 0..n
};

#ifdef __CUDACC__
// The network inputs of table row r of `rows`: node r mod G^d of the grid
// of date k = (r / G^d) / 2 + 1 and knock-in state (r / G^d) mod 2, the
// node's ln S per axis; the last row is the spot at t_0 (k = 0, no
// knock-in).  Inputs: ln S - ln ref, sigmas, rho, r, the period's length,
// remaining and elapsed dates / 5, knock-in, coupon, call and knock-in
// levels, 1.
__device__ __forceinline__ void cv_feature_row(const CvArgs &c, const CvFeatureArgs &fa, size_t r, size_t rows,
                                               float (&f)[kCvFeatures]) {
  float y[3] = {0.f, 0.f, 0.f};
  int k = 0, ki = 0;
  if (r + 1 < rows) {
    size_t node = r % size_t(c.nodes);
    const size_t grp = r / size_t(c.nodes);
    k = int(grp / 2) + 1;
    ki = int(grp % 2);
    for (int ax = c.d - 1; ax >= 0; --ax) {
      const int a = int(node % size_t(c.grid));
      node /= size_t(c.grid);
      y[ax] = c.lo[k - 1][ax] + float(a) * c.h[k - 1][ax];
    }
  } else {
    for (int i = 0; i < c.d; ++i) y[i] = fa.ln_spot[i];
  }
  for (int i = 0; i < 3; ++i) f[i] = i < c.d ? y[i] - logf(c.ref[i]) : 0.f;
  for (int i = 0; i < 3; ++i) f[3 + i] = i < c.d ? fa.sigma[i] : 0.f;
  f[6] = fa.rho;
  f[7] = fa.r;
  f[8] = fa.tau[k + 1] - fa.tau[k];
  f[9] = float(c.n - k) / 5.f;
  f[10] = float(k) / 5.f;
  f[11] = float(ki);
  f[12] = c.coupon;
  f[13] = c.call_level;
  f[14] = c.ki_level;
  f[15] = 1.f;
}
#endif

// MODE bits of the control-variate kernels: kCvWrite (per-path X, M, M2
// out), kCvGamma (second-order term), kCvPilot (moment sums for the betas
// instead of X, X^2, Y, Y^2); and for the run-time specialised kernel
// kCvWinRegs (a window of one date, the frontier's S in registers).
constexpr int kCvWrite = 1, kCvGamma = 2, kCvPilot = 4, kCvWinRegs = 8;

}  // namespace pc
