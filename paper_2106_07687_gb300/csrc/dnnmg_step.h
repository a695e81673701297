// Launchers of the DNN-MG correction kernels (internal to libdnnmg).
#pragma once
#include "kernels.h"

namespace dnnmg {

// constrained DOFs of a level state get their Dirichlet values
void launch_impose_dirichlet64(const Grid& g, double* x, cudaStream_t st);
// network inputs X [P][40] (bfloat16) from the prolongated state xt and the
// fine residual r, standardised with mean / stdv
void launch_gather(const Grid& gL, const Grid& gF, const int* patch_cell, int P, const double* xt,
                   const double* r, const float* mean, const float* stdv, double nu, double dt,
                   uint16_t* X, cudaStream_t st);
// vcorr = xt + (patch-averaged correction), zero correction on Dirichlet nodes
void launch_scatter(const Grid& gL, const Grid& gF, const int* cell_patch, const float* out,
                    int c_out, const double* xt, double* vcorr, cudaStream_t st);

}  // namespace dnnmg
