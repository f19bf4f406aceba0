// pc_cv_types.h -- the control-variate kernels' device arguments (CvArgs)
// and sizes: the part of pc_cv.h that the run-time compiler also sees.
#pragma once

#include "pc_types.h"

namespace pc {

constexpr int kCvMaxDates = 32;   // observation dates of the template
constexpr int kCvMaxD = 3;        // underlyings
constexpr int kCvFeatures = 16;   // network inputs
constexpr int kCvOutputs = 5;     // network outputs: value, up to 4 hedge ratios

struct CvArgs {
  const float *tables;            // [(n-1) * 2][nodes][4] (d used), 16-byte aligned
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
  float beta, beta2;              // Y = X - beta M - beta2 M2
  int32_t use_gamma;              // add the second-order term M2
  int32_t pilot;                  // 1: sums of X, M, M2 and their products (8), else X, X^2, Y, Y^2
};

// MODE bits of the control-variate kernels: kCvWrite (per-path X, M, M2
// out), kCvGamma (second-order term), kCvPilot (moment sums for the betas
// instead of X, X^2, Y, Y^2); and for the run-time specialised kernel
// kCvWinRegs (a window of one date, the frontier's S in registers).
constexpr int kCvWrite = 1, kCvGamma = 2, kCvPilot = 4, kCvWinRegs = 8;

}  // namespace pc
