// Persistent V-cycle (internal to libdnnmg).
#pragma once
#include <vector>

#include "kernels.h"

namespace dnnmg {

// Everything the cycle needs on one level; an array of these lives in
// device memory (index = level - coarsest level).
template <typename T>
struct VLevel {
  Grid g;
  Sten<T> s;
  T *x, *x2, *b, *d, *vb, *inv;
};

enum PhaseType {
  kPhasePass,
  kPhaseDefect,
  kPhaseRestrict,
  kPhaseCoarse,
  kPhaseProlong,
  kPhaseZeroTop,
  kPhasePassZero  // first pass of a sweep from x = 0 (the input is not read)
};

// in / out select the level's iterate (0: x, the caller's buffer on the top
// level; 1: the second buffer x2); a restriction with colour = 1 also zeroes
// the coarse iterate (needed when no pre-smoothing pass starts from zero)
struct Phase {
  int type, level, colour, in, out;
};

// phase list of one V(nu1, nu2) cycle with top level `top`, x zeroed first
std::vector<Phase> vcycle_phases(int top, int nu1, int nu2);
// whether a launch of nphases phases over nlevels levels fits the kernels'
// shared-memory tables
bool vcycle_fits(int nphases, int nlevels);
// colour-pass tiles of the cooperative kernel on a level (its natural grid)
int vcycle_coop_tiles(const Grid& g);
// co-resident grid size for the cooperative launch (0 if not available)
template <typename T>
int vcycle_grid(int coarse_nd);
// blocks of the largest single-cluster launch that can be resident (16 or
// 8; 0 if none)
template <typename T>
int vcycle_cluster_size(int coarse_nd);
// the same cycle as one thread-block cluster of `cluster` blocks; 0 on success
template <typename T>
int launch_vcycle_cluster(const VLevel<T>* lv, const Phase* ph, int nph, int top, const T* topb,
                          T* topx, const double* Ainv, T omega, int cluster, int coarse_nd,
                          cudaStream_t st);
// returns 0 on success; with skip, nothing runs when *skip != 0 at the
// launch's start
template <typename T>
int launch_vcycle_persistent(const VLevel<T>* lv, const Phase* ph, int nph, int top, const T* topb,
                             T* topx, const double* Ainv, T omega, int grid, int coarse_nd,
                             cudaStream_t st, const int* skip = nullptr);

}  // namespace dnnmg
