// transport.h -- internal interface between the transport front end
// (api.cu) and the schedule back ends (slab.cu, box.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mc.h"

namespace mci {

// One launch of a slab schedule over the device problem list.
struct SlabLaunch {
  const void* d_probs;         // device SlabDev[n_problems], prepared
  uint32_t n_problems;
  uint32_t chunk;              // histories per ticket grab (per warp)
  uint64_t range_begin, total; // global histories [range_begin, range_begin + total)
  unsigned long long* d_ticket;
  const mc_tally* tally;
  mc_lcg lcg;
  uint64_t event_cap;
  uint32_t smem_slots;         // 0 = global atomics; else slots staged in smem
  bool f32;
  int block, blocks_per_sm, num_sms;
};

size_t slab_dev_size();
void slab_fill_host(const mc_problem* src, uint32_t n, void* dst);
int slab_prep(void* d_probs, uint32_t n, cudaStream_t s);
int slab_history_launch(const SlabLaunch& L, cudaStream_t s);

// Event-based schedule (slab_event.cu): bank of `cap` particles in d_bank
// (slab_bank_bytes(cap) bytes); h_done is pinned host memory.  Synchronises
// `s` between batches of iterations.  capture_stream non-null: each batch is
// captured once on it into a graph, which is then launched on `s`.
size_t slab_bank_bytes(uint32_t cap);
int slab_event_run(const SlabLaunch& L, void* d_bank, uint32_t cap, unsigned int* h_done,
                   cudaStream_t capture_stream, cudaStream_t s);

}  // namespace mci
