// pc_cv.h -- device arguments of the control-variate kernels (pc_cv.cu).
// Private to the library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "pc_internal.h"
#include "pc_cv_types.h"
#include "pc_mlp.h"

namespace pc {

// Device scratch owned by a network (grow-only, freed with it).
float *mlp_scratch(struct ::pc_mlp *net, size_t floats);
// The fused table build's network description (false: build with the
// layer products).
bool mlp_cv_tables_tc(struct ::pc_mlp *net, size_t rows, float *tables, float *delta0, CvTablesTc &t);
// Waits for the context's stream; PC_ETIMEOUT (and the status cleared) if a
// tensor-core product of the network reported an expired wait.
pc_status mlp_status(struct ::pc_mlp *net);
// The network's forward on a given stream (capturable), and what a
// captured table build needs: the slot of its graph by key (created empty),
// the network's pinned read-back buffer [8] (null if none), its status word.
pc_status mlp_forward_on(struct ::pc_mlp *net, const float *d_x, size_t n, float *d_y, cudaStream_t s);
cudaGraphExec_t *mlp_graph(struct ::pc_mlp *net, const std::vector<uint8_t> &key);
float *mlp_pinned(struct ::pc_mlp *net);
int32_t *mlp_status_word(struct ::pc_mlp *net);

cudaError_t launch_cv(const PriceArgs &a, const CvArgs &c, int grid, int block, size_t smem, cudaStream_t s);
// The kernel mode (kCv* bits) of a launch: per-path outputs, second-order
// term, pilot sums.
int cv_mode(bool write, const CvArgs &c);
int cv_blocks_per_sm(int d, int block, size_t smem, const CvArgs &c);
cudaError_t launch_cv_features(const CvArgs &c, const CvFeatureArgs &fa, float *X, size_t rows,
                               cudaStream_t s);
cudaError_t launch_cv_scatter(const float *Y, int out_w, size_t rows, int d, float *tables, float *delta0,
                              cudaStream_t s);
// The node records' slopes from their ratios (after the scatter or the fused
// build): records = (n - 1) * 2 * nodes.
cudaError_t launch_cv_slopes(float *tables, size_t records, int nodes, int G, int d, cudaStream_t s);

}  // namespace pc
