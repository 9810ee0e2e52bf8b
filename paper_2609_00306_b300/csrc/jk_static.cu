// jk_static.cu -- Coulomb matrix J for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool or
// arena that owns all device memory, or a host application whose allocator
// must not be bypassed.  cd_jk_coulomb_static computes the same J as
// cd_jk(..., CD_JK_FP64 | CD_JK_DEVICE | CD_JK_ONLY_J) but takes its scratch
// (the packed density, the projected density v_P and the packed J) from one
// file-scope __device__ array of fixed size instead of allocating it.  Every
// GPU that loads this library holds that array until the process exits.
#include <mutex>
#include <string>
#include <unordered_map>
#include "internal.cuh"
#include "pivot.cuh"
#include "../../include/cderi_static.h"

namespace {

constexpr int64_t kStaticMaxRows = 1 << 20;      // screened pairs (rows)
constexpr int64_t kStaticMaxVectors = 1 << 15;   // Cholesky vectors M

// [0, rows): packed density d; [kStaticMaxRows, kStaticMaxRows + rows): packed J;
// [2 kStaticMaxRows, 2 kStaticMaxRows + M): v_P = sum_r L^P_r d_r.
// 2 x 2^20 + 2^15 doubles = 16.25 MiB.
static __device__ __align__(256) double g_coulomb_scratch[2 * kStaticMaxRows + kStaticMaxVectors];

std::mutex g_mu;
std::unordered_map<int, double*> g_scratch_addr;  // device ordinal -> device address of the array

// Device address of the scratch array on the current device.  In host code
// the symbol g_coulomb_scratch is only a host-side stand-in, so the address
// is obtained once per device with cudaGetSymbolAddress while that device is
// current.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cd::set_error(std::string("cd_jk_coulomb_static: cudaGetDevice failed: ") + cudaGetErrorString(e));
    return CD_ECUDA;
  }
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_scratch_addr.find(dev);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return CD_OK;
  }
  double* p = nullptr;
  e = cudaGetSymbolAddress((void**)&p, g_coulomb_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cd::set_error(std::string("cd_jk_coulomb_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return CD_ECUDA;
  }
  g_scratch_addr[dev] = p;
  *out = p;
  return CD_OK;
}

}  // namespace

extern "C" int cd_jk_coulomb_static(const cd_factor_t* f, const double* C_occ_dev, int32_t n_occ, double* J_dev,
                                    void* stream) {
  using namespace cd;
  if (!f || !C_occ_dev || !J_dev || n_occ <= 0) {
    set_error("cd_jk_coulomb_static: bad argument");
    return CD_EINVAL;
  }
  if (f->n > kStaticMaxRows || f->M > kStaticMaxVectors) {
    set_error("cd_jk_coulomb_static: factor too large for the static scratch (rows " + std::to_string(f->n) +
              " > " + std::to_string(kStaticMaxRows) + " or vectors " + std::to_string(f->M) + " > " +
              std::to_string(kStaticMaxVectors) + "); use cd_jk");
    return CD_EINVAL;
  }
  double* base = nullptr;
  CD_TRY(scratch_address(&base));
  cudaStream_t st = (cudaStream_t)stream;
  double* d = base;
  double* Jp = base + kStaticMaxRows;
  double* v = base + 2 * kStaticMaxRows;
  const int N = f->sys->hb.nbf;
  const int32_t* mu = f->sys->row_mu_dev;
  const int32_t* nu = f->sys->row_nu_dev;
  // d and v are fully overwritten; every entry of Jp is written by
  // launch_gemv_cols (stored by a single slab of vectors, or cleared and then
  // accumulated by several; cleared when there is no vector), and J is cleared
  // inside launch_unpack_sym.
  CD_TRY(launch_density_packed(C_occ_dev, N, n_occ, mu, nu, f->n, d, st));
  if (f->L) {
    CD_TRY(launch_gemv_rows<double>(f->L, f->ld, f->M, f->n, d, v, st));
    CD_TRY(launch_gemv_cols<double>(f->L, f->ld, f->M, f->n, v, Jp, st));
  } else {  // FP32-stored vectors (CD_VEC_FP32), FP64 accumulation
    CD_TRY(launch_gemv_rows<float>(f->L32, f->ld, f->M, f->n, d, v, st));
    CD_TRY(launch_gemv_cols<float>(f->L32, f->ld, f->M, f->n, v, Jp, st));
  }
  CD_TRY(launch_unpack_sym(Jp, mu, nu, f->n, N, J_dev, st));
  return CD_OK;
}
