// pf_peak.cu -- diagnostics: the measured fused multiply-add throughput of this
// GPU, FP32 and FP64 (the roofline denominators of the filter's kernels, which
// are FP32 and FP64 ALU work, not a tensor contraction), the propagate
// kernels' weight exponential on given arguments, and the invariant counters
// of a checked build.  None has a counterpart in the paper.
#include <algorithm>
#include <type_traits>
#include <cuda_runtime.h>

#include "pf.h"
#include "pf_internal.h"
#include "pf_runtime.h"

namespace {

constexpr int ACC = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chain(R* out, int iters, R b, R c) {
  R a[ACC];
#pragma unroll
  for (int k = 0; k < ACC; ++k) a[k] = R(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < ACC; ++k) a[k] = fma(a[k], b, c);
  }
  R s = 0;
#pragma unroll
  for (int k = 0; k < ACC; ++k) s += a[k];
  if (s == R(-1.2345)) out[blockIdx.x] = s;  // never true; keeps the chains alive
}

// The same chains on packed FP32 pairs (fma.rn.f32x2: one instruction, two
// lanes' fused multiply-adds), four flops per instruction.
struct Packed {};

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}

__global__ void __launch_bounds__(256) k_fma_chain2(float* out, int iters, float b, float c) {
  unsigned long long a[ACC];
#pragma unroll
  for (int k = 0; k < ACC; ++k) a[k] = pk2(float(threadIdx.x + k), float(threadIdx.x - k));
  const unsigned long long bb = pk2(b, b), cc = pk2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < ACC; ++k) a[k] = fma2(a[k], bb, cc);
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < ACC; ++k) s ^= a[k];
  if (s == 0x123456789abcdefull) out[blockIdx.x] = float(s);  // keeps the chains alive
}

template <typename R>
struct Kernel {
  static void* fn() { return reinterpret_cast<void*>(k_fma_chain<R>); }
  static void launch(int blocks, R* out, int iters) {
    k_fma_chain<R><<<blocks, 256>>>(out, iters, R(0.999999), R(1e-7));
  }
  static constexpr double flops_per_fma = 2.0;
  using Buf = R;
};
template <>
struct Kernel<Packed> {
  static void* fn() { return reinterpret_cast<void*>(k_fma_chain2); }
  static void launch(int blocks, float* out, int iters) {
    k_fma_chain2<<<blocks, 256>>>(out, iters, 0.999999f, 1e-7f);
  }
  static constexpr double flops_per_fma = 4.0;
  using Buf = float;
};

template <typename R>
pf_status measure(double* flops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return pfb::fail(PF_ECUDA, "no CUDA device");
  }
  using K = Kernel<R>;
  using B = typename K::Buf;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K::fn(), 256, 0);
  const int blocks = sms * std::max(per_sm, 1) * 4;
  B* out = nullptr;
  if (cudaMalloc(&out, sizeof(B) * blocks) != cudaSuccess) {
    cudaGetLastError();
    return pfb::fail(PF_ENOMEM, "peak measurement buffer");
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int iters = std::is_same<R, double>::value ? 64 : 1024;
  double best = 0.0, best_ms = 0.0;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(a);
    K::launch(blocks, out, iters);
    cudaEventRecord(b);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double f =
        K::flops_per_fma * ACC * double(iters) * double(blocks) * 256.0 / (double(ms) * 1e-3);
    if (rep >= 2 && f > best) {
      best = f;
      best_ms = ms;
    }
    if (rep < 2)  // size the kernel to about 40 ms
      iters = int(std::min<double>(double(iters) * 40.0 / std::max(double(ms), 0.01), 1 << 24));
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "peak kernel: %s", cudaGetErrorString(e));
  *flops = best;
  if (ms_out) *ms_out = best_ms;
  return PF_OK;
}

}  // namespace

extern "C" pf_status pf_measure_fma_peak(int32_t prec, double* flops_per_s, double* ms) {
  if (!flops_per_s) return pfb::fail(PF_EINVAL, "flops_per_s is NULL");
  if (prec == PF_FP64) return measure<double>(flops_per_s, ms);
  if (prec == PF_MIXED) return measure<float>(flops_per_s, ms);
  if (prec == 2) return measure<Packed>(flops_per_s, ms);
  return pfb::fail(PF_EINVAL, "prec must be PF_FP64, PF_MIXED or 2 (packed FP32 pairs)");
}

extern "C" pf_status pf_weight_exp(const double* d, double* w, int64_t n) {
  if (n < 0) return pfb::fail(PF_EINVAL, "n = %lld < 0", static_cast<long long>(n));
  if (n == 0) return PF_OK;
  if (!d || !w) return pfb::fail(PF_EINVAL, "d or w is NULL");
  if (n > (int64_t(1) << 28)) return pfb::fail(PF_EINVAL, "n = %lld > 2^28", static_cast<long long>(n));
  double* buf = nullptr;
  const size_t bytes = size_t(n) * sizeof(double);
  cudaError_t e = cudaMalloc(&buf, 2 * bytes);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  e = cudaMemcpy(buf, d, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pfb::launch_weight_exp(buf, buf + n, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(w, buf + n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "weight exponential: %s", cudaGetErrorString(e));
  return PF_OK;
}

extern "C" pf_status pf_weight_prefix(const double* w, double* prefix, double* totals,
                                      int64_t n) {
  if (n < 0) return pfb::fail(PF_EINVAL, "n = %lld < 0", static_cast<long long>(n));
  if (n == 0) return PF_OK;
  if (!w || !prefix || !totals) return pfb::fail(PF_EINVAL, "w, prefix or totals is NULL");
  if (n > (int64_t(1) << 28)) return pfb::fail(PF_EINVAL, "n = %lld > 2^28", static_cast<long long>(n));
  for (int64_t k = 0; k < n; ++k)
    if (!(w[k] >= 0.0 && w[k] <= 1.0))
      return pfb::fail(PF_EINVAL, "w[%lld] is not in [0, 1]", static_cast<long long>(k));
  const int64_t nt = (n + pfb::TILE - 1) / pfb::TILE;
  double* buf = nullptr;
  const size_t bytes = size_t(n) * sizeof(double);
  cudaError_t e = cudaMalloc(&buf, 2 * bytes + size_t(nt) * sizeof(double));
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  e = cudaMemcpy(buf, w, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pfb::launch_tile_prefix(buf, buf + n, buf + 2 * n, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(prefix, buf + n, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(totals, buf + 2 * n, size_t(nt) * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "tile prefix: %s", cudaGetErrorString(e));
  return PF_OK;
}

extern "C" pf_status pf_weight_sum_log(const double* s, double* y, int64_t n) {
  if (n < 0) return pfb::fail(PF_EINVAL, "n = %lld < 0", static_cast<long long>(n));
  if (n == 0) return PF_OK;
  if (!s || !y) return pfb::fail(PF_EINVAL, "s or y is NULL");
  if (n > (int64_t(1) << 28)) return pfb::fail(PF_EINVAL, "n = %lld > 2^28", static_cast<long long>(n));
  double* buf = nullptr;
  const size_t bytes = size_t(n) * sizeof(double);
  cudaError_t e = cudaMalloc(&buf, 2 * bytes);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  e = cudaMemcpy(buf, s, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pfb::launch_log_sum(buf, buf + n, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(y, buf + n, bytes, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "weight-sum logarithm: %s", cudaGetErrorString(e));
  return PF_OK;
}

extern "C" pf_status pf_debug_check_counts(uint64_t* counts, int32_t* checked) {
  if (!counts) return pfb::fail(PF_EINVAL, "counts is NULL");
  unsigned long long c[pfb::CHK_KINDS];
  const cudaError_t e = pfb::read_checks(c);
  if (e != cudaSuccess) return pfb::fail(PF_ECUDA, "check counters: %s", cudaGetErrorString(e));
  for (int k = 0; k < pfb::CHK_KINDS; ++k) counts[k] = c[k];
  if (checked) *checked = PF_CHECKED;
  return PF_OK;
}
