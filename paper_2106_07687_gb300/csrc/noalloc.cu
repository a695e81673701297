// Allocation-free variant of the coarse-level direct solve.
//
// dnnmg_coarse_solve_noalloc() does what the coarse level of a V-cycle does
// after linearisation (assemble the coarse Jacobian, factor it by banded LU
// with partial pivoting, solve), but without a context and without any
// device allocation: its working memory (band matrix, pivots, boundary
// masks) is a file-scope __device__ array of fixed size.  It serves callers
// that cannot call cudaMalloc, for instance code running under an external
// memory manager that owns the whole device heap, or a real-time loop where
// an allocation (and the implicit synchronisation it can cause) is not
// allowed.
#include <mutex>

#include "runtime.h"

namespace {

// Upper bound of the working memory; level 1 (the coarse level this library
// supports) needs 891 x 187 doubles of band plus pivots and masks, ~1.34 MB.
constexpr size_t kScratchBytes = size_t(2) << 20;  // 2 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Solid cells and boundary flags of one level, computed on the device from
// the obstacle block (same rules as the host-side level construction).
__global__ void level_masks_kernel(int ell, int oi0, int oj0, int nx, int ny, uint8_t* solid,
                                   uint8_t* flags) {
  const int nnx = nx + 1, nny = ny + 1;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nnx * nny; n += gridDim.x * blockDim.x) {
    const int i = n % nnx, j = n / nnx;
    auto is_solid = [&](int ci, int cj) {
      if (oi0 < 0) return false;
      const int I = ci >> ell, J = cj >> ell;
      return I >= oi0 && I < oi0 + 2 && J >= oj0 && J < oj0 + 2;
    };
    if (i < nx && j < ny) solid[j * nx + i] = is_solid(i, j) ? 1 : 0;
    bool ts = false, tf = false;
    for (int cy = -1; cy <= 0; ++cy)
      for (int cx = -1; cx <= 0; ++cx) {
        const int ci = i + cx, cj = j + cy;
        if (ci < 0 || cj < 0 || ci >= nx || cj >= ny) continue;
        if (is_solid(ci, cj))
          ts = true;
        else
          tf = true;
      }
    uint8_t f = 0;
    if (ts || i == 0 || j == 0 || j == ny) f |= dnnmg::kVDir;
    if (!tf) f |= dnnmg::kPFix;
    flags[n] = f;
  }
}

}  // namespace

namespace dnnmg {
void set_thread_error(const char* msg);  // capi.cu
}

extern "C" int dnnmg_coarse_solve_noalloc(const dnnmg_config* cfg, const double* vbar,
                                          const double* b, double* x, void* stream) {
  using namespace dnnmg;
  if (!cfg || !vbar || !b || !x) {
    set_thread_error("dnnmg_coarse_solve_noalloc: null argument");
    return DNNMG_ERR_ARG;
  }
  if (!(cfg->nu > 0) || !(cfg->dt > 0) || !(cfg->alpha0 >= 0) || cfg->theta != 1.0) {
    set_thread_error("dnnmg_coarse_solve_noalloc: nu, dt, alpha0 or theta out of range");
    return DNNMG_ERR_ARG;
  }
  if (cfg->obstacle_level != 0) {
    set_thread_error("dnnmg_coarse_solve_noalloc: only level-0 obstacle blocks");
    return DNNMG_ERR_ARG;
  }
  if (cfg->obstacle_i0 >= 0 &&
      (cfg->obstacle_i0 < 1 || cfg->obstacle_i0 > 13 || cfg->obstacle_j0 != 1)) {
    set_thread_error("dnnmg_coarse_solve_noalloc: obstacle must be a 2x2 level-0 block, j0 = 1");
    return DNNMG_ERR_ARG;
  }
  const int ell = cfg->level_coarse;
  if (ell < 1 || ell > 9) {
    set_thread_error("dnnmg_coarse_solve_noalloc: level_coarse must be in 1..9");
    return DNNMG_ERR_ARG;
  }
  Grid g{};
  g.nx = 16 << ell;
  g.ny = 4 << ell;
  g.nnx = g.nx + 1;
  g.nny = g.ny + 1;
  g.nn = g.nnx * g.nny;
  g.h = 4.0 / g.nx;
  const size_t band_b = align256(coarse_band_doubles(g) * sizeof(double));
  const size_t piv_b = align256((size_t)3 * g.nn * sizeof(int));
  const size_t solid_b = align256((size_t)g.nx * g.ny);
  const size_t flags_b = align256((size_t)g.nn);
  const size_t need = band_b + piv_b + solid_b + flags_b + 256;
  if (need > kScratchBytes || !coarse_supported(g)) {
    set_thread_error("dnnmg_coarse_solve_noalloc: the coarse level needs more than the 2 MiB "
                     "of static scratch (only level 1 fits)");
    return DNNMG_ERR_ARG;
  }
  // an error left pending by earlier, unrelated work of this thread is not
  // ours to report or to clear: refuse to run on top of it
  if (cudaPeekAtLastError() != cudaSuccess) {
    set_thread_error("dnnmg_coarse_solve_noalloc: a CUDA error was pending before the call");
    return DNNMG_ERR_CUDA;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_thread_error("dnnmg_coarse_solve_noalloc: no usable CUDA device");
    return DNNMG_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    // once per device, with that device current: the symbol's device address
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        set_thread_error("dnnmg_coarse_solve_noalloc: cudaGetSymbolAddress failed");
        return DNNMG_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* band = reinterpret_cast<double*>(base);
  int* piv = reinterpret_cast<int*>(base + band_b);
  uint8_t* solid = base + band_b + piv_b;
  uint8_t* flags = solid + solid_b;
  int* status = reinterpret_cast<int*>(flags + flags_b);
  g.solid = solid;
  g.flags = flags;
  auto fail = [](const char* what) {
    set_thread_error(what);
    return DNNMG_ERR_CUDA;
  };
  // the status word keeps the previous call's value: clear it
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: clearing the status word failed");
  note_launch();
  level_masks_kernel<<<cdiv(g.nn, 256), 256, 0, st>>>(ell, cfg->obstacle_i0, cfg->obstacle_j0,
                                                     g.nx, g.ny, solid, flags);
  if (cudaGetLastError() != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: launch of the mask kernel failed");
  const Sten<double> s = make_sten<double>(g.h, *cfg);
  launch_coarse_lu(g, s, vbar, band, piv, status, st);
  if (cudaGetLastError() != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: launch of the coarse LU failed");
  launch_coarse_lu_solve(g, band, piv, b, x, st);
  if (cudaGetLastError() != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: launch of the coarse solve failed");
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: reading the status word failed");
  if (cudaStreamSynchronize(st) != cudaSuccess)
    return fail("dnnmg_coarse_solve_noalloc: the solve failed on the device");
  if (h_status) {
    set_thread_error("dnnmg_coarse_solve_noalloc: singular coarse-level matrix");
    return DNNMG_ERR_NUMERICAL;
  }
  set_thread_error("");
  return DNNMG_OK;
}
