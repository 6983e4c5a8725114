// diag.cu -- diagnostic entry points: the flight logarithm and the
// integer-pipe reciprocal and 2u - 1 of the fp64 transport path evaluated on
// the host and on the device, and the CUDA library's log and division for
// comparison.  Not used by the transport itself.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "fp_exact.cuh"
#include "mc_log.cuh"

namespace {

__global__ void log1m_kernel(const double* __restrict__ u, double* __restrict__ out, uint64_t n, int which) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += nt) out[i] = which == 0 ? mclog::log1m(u[i]) : log(1.0 - u[i]);
}

__global__ void recip_kernel(const double* __restrict__ y, double* __restrict__ out, uint64_t n, int which) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += nt) out[i] = which == 0 ? mcx::recip_rn(y[i]) : 1.0 / y[i];
}

}  // namespace

extern "C" {

MC_API double mc_recip_rn(double y) { return mcx::recip_rn(y); }

MC_API double mc_two_u_minus_1(uint64_t n) { return n < (1ull << 53) ? mcx::two_u_minus_1(n) : 0.0; }

MC_API long long mc_llrint_nonneg(double v) { return mcx::llrint_nonneg(v); }

MC_API int mc_d_lt(double a, double b) { return mcx::d_lt(a, b) ? 1 : 0; }

MC_API double mc_mul_small(uint32_t j, double h) { return mcx::mul_small(j, h); }

MC_API int mc_recip_rn_device(const double* d_y, double* d_out, uint64_t n, int which, void* stream) {
  if ((n && (!d_y || !d_out)) || (which != 0 && which != 1)) {
    mci::set_error("mc_recip_rn_device: NULL buffer or which not in {0, 1}");
    return MC_ERR_ARG;
  }
  if (n == 0) return MC_OK;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  recip_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_y, d_out, n, which);
  return mci::cuda_status(cudaGetLastError(), "recip_kernel launch");
}

MC_API double mc_log1m(double u) { return mclog::log1m(u); }

MC_API int mc_log1m_device(const double* d_u, double* d_out, uint64_t n, int which, void* stream) {
  if ((n && (!d_u || !d_out)) || (which != 0 && which != 1)) {
    mci::set_error("mc_log1m_device: NULL buffer or which not in {0, 1}");
    return MC_ERR_ARG;
  }
  if (n == 0) return MC_OK;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  log1m_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_u, d_out, n, which);
  return mci::cuda_status(cudaGetLastError(), "log1m_kernel launch");
}

}  // extern "C"
