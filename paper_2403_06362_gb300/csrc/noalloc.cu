// noalloc.cu -- mc_transport_run_static: the slab transport for callers that
// must not allocate device memory.
//
// mc_transport_run keeps its scratch (the work ticket and the device copy of
// the problem list) in an mc_ctx, whose creation calls cudaMalloc.  Some
// callers cannot do that: code in a process whose device memory is owned by
// another allocator (a framework's caching allocator or a fixed memory pool
// that must account for every byte), and code that must not grow its
// footprint or take cudaMalloc's implicit device synchronisation after
// start-up (a latency-bound service, a plugin inside a host application).
// This entry point takes its scratch from one file-scope __device__ array
// instead.  The array is part of the module image: every device that loads
// libmc holds kStaticBytes of it until the process exits.
//
// Set-up: on the first call on a device (with that device current) the
// host looks up the array's device address with cudaGetSymbolAddress and
// caches it; make that first call before any stream capture begins.  The
// cached address belongs to the device's context at that time, so a device
// reset after the first call is not supported.
// Sharing: every call uses the same array, which keeps the previous call's
// contents; the upload kernel rewrites the problem list and zeroes the
// ticket on every call.  Two calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "slab.cuh"
#include "transport.h"

namespace {

constexpr uint32_t kStaticMaxProblems = 256;
constexpr size_t kTicketBytes = 256;  // the ticket, padded to keep the problem list 256-aligned
constexpr size_t kStaticBytes = kTicketBytes + kStaticMaxProblems * sizeof(mcs::SlabDev);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
struct DeviceSlot {
  void* scratch = nullptr;  // device address of g_static_scratch on this device
  int num_sms = 0;
  int smem_optin = 0;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

// Problems travel to the device as kernel parameters, 16 per launch.
constexpr uint32_t kUploadChunk = 16;
struct UploadChunk {
  mcs::SlabDev p[kUploadChunk];
};

__global__ void static_upload_kernel(const UploadChunk chunk, uint32_t first, uint32_t count,
                                     mcs::SlabDev* __restrict__ dst, unsigned long long* __restrict__ ticket) {
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) dst[first + i] = chunk.p[i];
  if (first == 0 && threadIdx.x == 0) *ticket = 0ull;
}

int device_slot(DeviceSlot** out) {
  int dev = 0;
  MC_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    mci::set_error("mc_transport_run_static: device %d beyond the %d supported", dev, kMaxDevices);
    return MC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_slots_mu);
  DeviceSlot& s = g_slots[dev];
  if (!s.scratch) {
    void* p = nullptr;
    MC_TRY_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    MC_TRY_CUDA(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev));
    MC_TRY_CUDA(cudaDeviceGetAttribute(&s.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    s.scratch = p;
  }
  *out = &s;
  return MC_OK;
}

// The checks of mc_transport_run (shared with api.cu), then this entry
// point's own limits: slab problems only, at most kStaticMaxProblems, the
// history schedule.
int check_static_args(const mc_problem* p, uint32_t n, const mc_run_config* cfg, const mc_tally* t,
                      uint64_t* total) {
  if (n > kStaticMaxProblems) {
    mci::set_error("mc_transport_run_static: %u problems exceed the static maximum of %u", n,
                   kStaticMaxProblems);
    return MC_ERR_ARG;
  }
  for (uint32_t i = 0; i < n; ++i) {
    if (p[i].geometry != MC_GEOM_SLAB) {
      mci::set_error("mc_transport_run_static: problem %u is not a slab problem (box and pulse geometries need "
                     "mc_transport_run)", i);
      return MC_ERR_ARG;
    }
  }
  int st = mci::check_problems(p, n, t, total);
  if (st != MC_OK) return st;
  st = mci::check_run_config(cfg, "mc_transport_run_static");
  if (st != MC_OK) return st;
  if (cfg->schedule == MC_SCHED_EVENT) {
    mci::set_error("mc_transport_run_static: the history schedule only (its bank would need an allocation)");
    return MC_ERR_ARG;
  }
  return MC_OK;
}

}  // namespace

extern "C" MC_API int mc_transport_run_static(const mc_lcg* lcg, const mc_problem* problems,
                                              uint32_t n_problems, const mc_run_config* cfg,
                                              const mc_tally* tally, void* stream) {
  if (!problems || n_problems == 0 || !cfg || !tally || !tally->d_bins || !tally->d_counts) {
    mci::set_error("mc_transport_run_static: NULL argument or no problems");
    return MC_ERR_ARG;
  }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  uint64_t total = 0;
  st = check_static_args(problems, n_problems, cfg, tally, &total);
  if (st != MC_OK) return st;
  const uint64_t rb = cfg->range_begin, re = cfg->range_end == 0 ? total : cfg->range_end;
  if (rb > re || re > total) {
    mci::set_error("mc_transport_run_static: range outside the %llu histories", (unsigned long long)total);
    return MC_ERR_ARG;
  }
  DeviceSlot* slot = nullptr;
  st = device_slot(&slot);
  if (st != MC_OK) return st;
  uint32_t slots = 0;  // checked before anything is enqueued
  st = mci::slab_staged_slots(cfg, tally, (size_t)slot->smem_optin, "mc_transport_run_static", &slots);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  auto* ticket = static_cast<unsigned long long*>(slot->scratch);
  auto* dprobs = reinterpret_cast<mcs::SlabDev*>(static_cast<unsigned char*>(slot->scratch) + kTicketBytes);

  // Upload (also zeroes the ticket left by the previous call) and prepare.
  for (uint32_t first = 0; first < n_problems; first += kUploadChunk) {
    const uint32_t count = n_problems - first < kUploadChunk ? n_problems - first : kUploadChunk;
    UploadChunk chunk;
    std::memset(&chunk, 0, sizeof chunk);
    mci::slab_fill_host(problems + first, count, chunk.p);
    static_upload_kernel<<<1, 32, 0, s>>>(chunk, first, count, dprobs, ticket);
    MC_TRY_CUDA(cudaGetLastError());
  }
  st = mci::slab_prep(dprobs, n_problems, s);
  if (st != MC_OK) return st;
  if (!cfg->accumulate) {
    MC_TRY_CUDA(cudaMemsetAsync(tally->d_bins, 0, tally->n_slots * sizeof(int64_t), s));
    MC_TRY_CUDA(cudaMemsetAsync(tally->d_counts, 0, (size_t)n_problems * MC_NCOUNT * sizeof(uint64_t), s));
  }
  if (re == rb) return MC_OK;

  mci::SlabLaunch L{};
  L.d_probs = dprobs;
  L.n_problems = n_problems;
  L.chunk = cfg->chunk ? cfg->chunk : mci::slab_default_chunk(re - rb, slot->num_sms);
  L.range_begin = rb;
  L.total = re - rb;
  L.d_ticket = ticket;
  L.tally = tally;
  L.lcg = *lcg;
  L.event_cap = cfg->event_cap ? cfg->event_cap : (1ull << 40);
  L.smem_slots = slots;
  L.single_n_bins = n_problems == 1 ? problems[0].n_bins : 0u;
  L.f32 = cfg->precision == MC_FP32_GUARDED;
  L.block = cfg->block ? (int)cfg->block : mci::slab_default_block(L.total, L.chunk, slot->num_sms);
  L.blocks_per_sm = (int)cfg->blocks_per_sm;
  L.num_sms = slot->num_sms;
  L.tally_agg = mci::tally_agg_of(cfg->tally_atomics, mci::kSlabAggDefault);
  return mci::slab_history_launch(L, s);
}
