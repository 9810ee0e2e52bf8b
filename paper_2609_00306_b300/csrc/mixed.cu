// mixed.cu -- mixed-precision J/K: vectors stored FP32 (rounded once after the
// FP64 factorisation); J accumulates FP32 vector entries against an FP64
// density in FP64; K runs on the tensor cores (see kexchange.cu).
#include "internal.cuh"
#include "pivot.cuh"

namespace cd {
namespace {
__global__ void to_fp32_kernel(const double* __restrict__ src, int64_t ld, int64_t total, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}
}  // namespace

int launch_to_fp32(const double* src, int64_t ld, int64_t M, int64_t n, float* dst, cudaStream_t st) {
  const int64_t total = M * ld;
  if (total <= 0) return CD_OK;
  (void)n;
  to_fp32_kernel<<<148 * 8, 256, 0, st>>>(src, ld, total, dst);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int jk_mixed(const float* L32, int64_t ld, int64_t M, int64_t n, int N, int O, const double* C_dev,
             const int32_t* mu, const int32_t* nu, double* J_dev, double* K_dev, bool wantJ, bool wantK,
             cudaStream_t st) {
  if (wantK) {
    set_error("cd_jk: the BF16x3 exchange kernel is not available in this build");
    return CD_EINVAL;
  }
  if (wantJ) {
    double *d = nullptr, *v = nullptr, *Jp = nullptr;
    CD_CUDA(cudaMalloc(&d, sizeof(double) * std::max<int64_t>(n, 1)));
    CD_CUDA(cudaMalloc(&v, sizeof(double) * std::max<int64_t>(M, 1)));
    CD_CUDA(cudaMalloc(&Jp, sizeof(double) * std::max<int64_t>(n, 1)));
    int rc = launch_density_packed(C_dev, N, O, mu, nu, n, d, st);
    if (rc == CD_OK) rc = launch_gemv_rows<float>(L32, ld, M, n, d, v, st);
    if (rc == CD_OK) rc = launch_gemv_cols<float>(L32, ld, M, n, v, Jp, st);
    if (rc == CD_OK) rc = launch_unpack_sym(Jp, mu, nu, n, N, J_dev, st);
    cudaStreamSynchronize(st);
    cudaFree(d); cudaFree(v); cudaFree(Jp);
    if (rc != CD_OK) return rc;
  }
  return CD_OK;
}

}  // namespace cd
