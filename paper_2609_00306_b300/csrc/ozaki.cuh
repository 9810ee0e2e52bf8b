// ozaki.cuh -- exact-slice GEMM on the BF16 tensor cores (interface).
//
// A real matrix X is represented, row by row, as X[m][k] = 2^e[m] * x[m][k]
// with |x| <= 1 and x ~ sum_{s=1..S} a_s 2^-(8s-1), a_s integers in
// [-128, 128] (exact in BF16).  A product of two such matrices is
//   sum_k X[m][k] Y[n][k] = 2^(e_m + f_n) sum_{s,t} 2^-(8(s+t)-2) sum_k a_s b_t .
// Each inner sum over at most `kc` values of k is an integer below 2^24 in
// magnitude, so the tensor cores' FP32 accumulation of it is exact (this is the
// error-free splitting of Ozaki et al., Numer. Algorithms 59 (2012) 95).
// Products with s + t <= KEEP are formed; products of equal s + t share one
// tensor-memory accumulator; after every kc values of k the accumulators are
// drained into a signed 64-bit fixed-point sum with unit 2^-F.  The result is
// exact up to the dropped slice products and the rounding at 2^-F.
#pragma once
#include <cuda.h>
#include "internal.cuh"

namespace cd {

// Slices of one entry: v = round(x 2^(8S-1)) for |x| <= 1 (|v| <= 2^(8S-1)),
// written as v = sum_s a_s 2^(8(S-1-s)) with balanced base-256 digits: the
// low digits in [-128, 127], taken from the least significant end with
// integer operations, the top digit the remainder (|a_0| <= 128).  Every digit
// is an integer of at most 8 bits, exact in BF16.  (No FP64 arithmetic: the
// FP64 pipe of this GPU is the scarce unit.)
template <int S>
__device__ __forceinline__ void fixed_digits(long long v, float (&a)[S]) {
  // every digit fits a 32-bit int; converting from int32 keeps the
  // conversion off the FP64 pipe (a 64-bit integer conversion runs there)
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const long long d = ((v + 128) & 255) - 128;
    a[s] = (float)(int)d;
    v = (v - d) >> 8;
  }
  a[0] = (float)(int)v;
}
// round(x * 2^k) for a finite double x with |x * 2^k| < 2^62, by integer
// operations on the bit pattern (ties away from zero).  A direct double ->
// int64 conversion would occupy the FP64 pipe, the scarce unit of this GPU.
__device__ __forceinline__ long long scaled_double_to_ll(double x, int k) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal: below any fixed-point unit used here
  const long long man = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
  const int sh = ex - 1075 + k;  // value = man * 2^sh
  long long v;
  if (sh >= 0) v = man << sh;
  else if (sh > -63) v = (man + (1ll << (-sh - 1))) >> (-sh);
  else v = 0;
  return bits < 0 ? -v : v;
}
__device__ __forceinline__ long long scaled_double_to_ll(float x, int k) {
  const int bits = __float_as_int(x);
  const int ex = (bits >> 23) & 0xFF;
  if (ex == 0) return 0;
  const long long man = (long long)((bits & 0x7FFFFF) | (1 << 23));
  const int sh = ex - 150 + k;
  long long v;
  if (sh >= 0) v = man << sh;
  else if (sh > -63) v = (man + (1ll << (-sh - 1))) >> (-sh);
  else v = 0;
  return bits < 0 ? -v : v;
}

// 64-byte swizzled K-major descriptor: rows of 32 bf16 (64 B), 8-row groups 512 B apart
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused: swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                   // version
  d |= (uint64_t)4 << 61;                   // 64-byte swizzle
  return d;
}

// An FP32 accumulator value that is an exact integer with |x| <= 2^24, as a
// 64-bit integer, using only FP32 adds/FMAs and integer adds: x = 4096 h + l
// with h = round(x / 4096) (|h| <= 4096) and |l| <= 2048, each turned into an
// int by the 1.5 * 2^23 mantissa trick.  (A direct float -> int64 conversion
// executes on the FP64 pipe of this GPU, which would bound the drain.)
__device__ __forceinline__ long long exact_float_to_ll(float x) {
  constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
  const float h = __fadd_rn(__fmaf_rn(x, 1.0f / 4096.0f, kMagic), -kMagic);
  const float l = __fmaf_rn(-h, 4096.0f, x);
  const int hi = __float_as_int(__fadd_rn(h, kMagic)) - 0x4B400000;
  const int lo = __float_as_int(__fadd_rn(l, kMagic)) - 0x4B400000;
  return ((long long)hi << 12) + (long long)lo;
}

// largest |a_s * b_t| used for the exactness bound of the FP32 accumulation
constexpr double kSliceProdMax = 129.0 * 129.0;

struct OzakiPlan {
  int SA = 3, SB = 3, KEEP = 4;   // slices of A and B, largest s + t kept
  int F = 40;                     // fixed-point fraction bits of the output
};

// Slice tensors: bf16 [S][rows][kpitch] (k contiguous).  Output: int64
// D[n][m] (leading dimension ldd, column n = row of B) accumulated with
// atomicAdd over k in [0, kdim) split into `ksplit` CTA slabs.
// sym: A and B are the same matrix; tiles entirely below the diagonal
// (column tile end <= row tile start) are skipped, so only D[n][m] with m <= n
// (and some near the diagonal) is written.
// a_chunked: A is stored in k-chunks of 32 instead, [kdim/32][SA][a_rows][32]
// (the growable slice store of the decomposition; a_kpitch is then unused).
int ozaki_gemm(const OzakiPlan& plan, const void* As, int64_t a_rows, int64_t a_kpitch,
               const void* Bs, int64_t b_rows, int64_t b_kpitch, int64_t kdim,
               unsigned long long* D, int64_t ldd, int ksplit, int* err_dev, cudaStream_t st, bool sym = false,
               bool a_chunked = false);

// Slicing: x = X / 2^e (row exponent e given) -> S bf16 integer slices.
// src element (r, k) at src[r * src_rs + k * src_ks]; dst[s][r][k0 + k] with pitch kpitch.
// chunked: dst in k-chunks of 32, [k/32][S][dst_rows][32] (kpitch unused).
int launch_slice_rows_f64(const double* src, int64_t src_rs, int64_t src_ks, int64_t rows, int64_t kcount,
                          const int32_t* row_exp, int S, void* dst, int64_t dst_rows, int64_t kpitch, int64_t k0,
                          cudaStream_t st, bool chunked = false);

int launch_row_exp_sqrt(const double* d, int64_t n, int32_t* e, cudaStream_t st);
// registers one CTA of the column-update GEMM occupies on its SM
int update_cta_registers(int* regs);
// Ls in k-chunks of 32 ([K/32][S][n][32], the decomposition's slice store);
// Bs flat [S][nb][bpitch]
int launch_gather_slices(const void* Ls, int64_t n, const int64_t* rows, const int64_t* valid, int nb,
                         int S, int64_t K, void* Bs, int64_t bpitch, cudaStream_t st);
// elements of one k-chunk of 32 slices of one row: the chunk layout's row pitch is 64 bytes
constexpr int kSliceChunk = 32;
int launch_colupd_finalize(const unsigned long long* D, int64_t ldd, int64_t n, int nb, const int32_t* e,
                           const int64_t* rows, const int32_t* slots, int F, double* cols, int64_t ld, cudaStream_t st);

}  // namespace cd
