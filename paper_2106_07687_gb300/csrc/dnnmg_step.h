// Launchers of the DNN-MG correction kernels (internal to libdnnmg).
#pragma once
#include "kernels.h"

namespace dnnmg {

// constrained DOFs of a level state get their Dirichlet values
void launch_impose_dirichlet64(const Grid& g, double* x, cudaStream_t st);
// Patches are the fluid cells of level L (gL); their K x K nodes (K = 3 for
// one replaced level, 5 for two) lie on the fine level gF.
// network inputs X [P][4 K^2 + 4] (bfloat16) from the prolongated state xt
// and the fine residual r, standardised with mean / stdv
void launch_gather(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                   const double* xt, const double* r, const float* mean, const float* stdv,
                   double nu, double dt, uint16_t* X, cudaStream_t st);
// vcorr = xt + (patch-averaged correction), zero correction on Dirichlet nodes
void launch_scatter(const Grid& gL, const Grid& gF, int K, const int* cell_patch, const float* out,
                    int c_out, const double* xt, double* vcorr, cudaStream_t st);

// raw (unstandardised FP32) features and training targets [P][2 K^2] of
// every patch
void launch_gather_raw(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                       const double* xt, const double* r, double nu, double dt, float* Xraw,
                       cudaStream_t st);
void launch_targets(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                    const double* xnext, const double* xt, float* Y, cudaStream_t st);
// per-feature mean / std (FP64 sums, fixed order) of rows x C features;
// partial needs nb * C * 2 doubles
void launch_feature_stats(const float* X, long long rows, int C, double* partial, int nb,
                          float* mean, float* stdv, cudaStream_t st);
void launch_gather_batch(const float* Xraw, const float* Yc, const int* idx, int B, int T,
                         long long stride, int Ci, int Co, const float* mean, const float* stdv,
                         uint16_t* Xb, float* Yb, cudaStream_t st);

}  // namespace dnnmg
