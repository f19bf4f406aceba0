// pc_cv.h -- device arguments of the control-variate kernels (pc_cv.cu).
// Private to the library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "pc_internal.h"

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

// Device scratch owned by a network (grow-only, freed with it).
float *mlp_scratch(struct ::pc_mlp *net, size_t floats);
// Waits for the context's stream; PC_ETIMEOUT (and the status cleared) if a
// tensor-core product of the network reported an expired wait.
pc_status mlp_status(struct ::pc_mlp *net);

struct CvFeatureArgs {
  float ln_spot[kCvMaxD];
  float sigma[kCvMaxD];
  float rho, r;
  float tau[kCvMaxDates + 1];     // year fractions of ordinals 0..n
};

cudaError_t launch_cv(const PriceArgs &a, const CvArgs &c, int grid, int block, size_t smem, cudaStream_t s);
int cv_blocks_per_sm(int d, int block, size_t smem, const CvArgs &c);
cudaError_t launch_cv_features(const CvArgs &c, const CvFeatureArgs &fa, float *X, size_t rows,
                               cudaStream_t s);
cudaError_t launch_cv_scatter(const float *Y, int out_w, size_t rows, int d, float *tables, float *delta0,
                              cudaStream_t s);

}  // namespace pc
