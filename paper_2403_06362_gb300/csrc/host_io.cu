// host_io.cu -- mc_lcg_draw_host: fused seeding and draws on host buffers.
//
// The id range is cut into slices of kSlice streams.  Two device slots
// (context-owned) alternate: while the draw kernel of slice j runs on the
// caller's stream, a private copy stream returns slice j - 1's final states
// and digests to the host, and a slot is reused only after its last copy
// has finished (events, no host waits inside the loop).  The call returns
// when every result is in host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace {

constexpr uint64_t kSlice = 1ull << 22;  // streams per slice (32 MiB per array)

int io_setup(mc_ctx* ctx) {
  if (!ctx->io_stream) MC_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->io_stream, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k) {
    if (!ctx->io_computed[k]) MC_TRY_CUDA(cudaEventCreateWithFlags(&ctx->io_computed[k], cudaEventDisableTiming));
    if (!ctx->io_copied[k]) MC_TRY_CUDA(cudaEventCreateWithFlags(&ctx->io_copied[k], cudaEventDisableTiming));
  }
  return ctx->host_io.reserve(2 * kSlice * 2 * sizeof(uint64_t));
}

}  // namespace

extern "C" MC_API int mc_lcg_draw_host(mc_ctx* ctx, const mc_lcg* lcg, const mc_seed_spec* seed, uint64_t id_begin,
                                       uint64_t* h_states, uint64_t n_streams, uint32_t draws, uint64_t* h_digest,
                                       void* stream) {
  if (!ctx) {
    mci::set_error("mc_lcg_draw_host: ctx is NULL");
    return MC_ERR_ARG;
  }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  if (n_streams == 0) return MC_OK;
  if (!seed && !h_states) {
    mci::set_error("mc_lcg_draw_host: h_states is NULL and no seed spec is given");
    return MC_ERR_ARG;
  }
  if (!h_states && !h_digest) {
    mci::set_error("mc_lcg_draw_host: no output (h_states and h_digest are NULL)");
    return MC_ERR_ARG;
  }
  MC_TRY_CUDA(cudaSetDevice(ctx->device));
  st = io_setup(ctx);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* base = static_cast<uint64_t*>(ctx->host_io.ptr);
  const uint64_t nslices = (n_streams + kSlice - 1) / kSlice;
  for (uint64_t j = 0; j < nslices; ++j) {
    const int k = (int)(j & 1u);
    const uint64_t lo = j * kSlice, cnt = std::min<uint64_t>(kSlice, n_streams - lo);
    uint64_t* d_st = base + (size_t)k * 2 * kSlice;
    uint64_t* d_dg = d_st + kSlice;
    if (j >= 2) MC_TRY_CUDA(cudaStreamWaitEvent(s, ctx->io_copied[k], 0));  // slot free again
    if (!seed)
      MC_TRY_CUDA(cudaMemcpyAsync(d_st, h_states + lo, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    st = mc_lcg_draw(ctx, lcg, seed, id_begin + lo, h_states ? d_st : nullptr, cnt, draws, nullptr,
                     h_digest ? d_dg : nullptr, stream);
    if (st != MC_OK) return st;
    MC_TRY_CUDA(cudaEventRecord(ctx->io_computed[k], s));
    MC_TRY_CUDA(cudaStreamWaitEvent(ctx->io_stream, ctx->io_computed[k], 0));
    if (h_states)
      MC_TRY_CUDA(cudaMemcpyAsync(h_states + lo, d_st, cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                  ctx->io_stream));
    if (h_digest)
      MC_TRY_CUDA(cudaMemcpyAsync(h_digest + lo, d_dg, cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                  ctx->io_stream));
    MC_TRY_CUDA(cudaEventRecord(ctx->io_copied[k], ctx->io_stream));
  }
  MC_TRY_CUDA(cudaStreamSynchronize(ctx->io_stream));
  return MC_OK;
}
