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
  uint32_t single_n_bins;      // n_bins of the problem when n_problems == 1
  const void* d_tables = nullptr;  // per-problem edge and width tables (nullable; see slab_prep)
  bool f32;
  int block, blocks_per_sm, num_sms;
  uint32_t pool_lock_attempts = 1u << 20;  // compaction-pool lock (mc_limits)
  // processing order of several problems (slab_prep's d_order area; null: id order)
  const uint32_t* d_order = nullptr;
  const uint64_t* d_order_begin = nullptr;
  bool tally_agg = true;                   // warp-aggregated tally atomics
  uint64_t event_iterations = ~0ull;       // event schedule bound (mc_limits; ~0: derived)
};

size_t slab_dev_size();
void slab_fill_host(const mc_problem* src, uint32_t n, void* dst);
// d_tables (nullable): room for slab_table_doubles(...) doubles, filled
// with every problem's bin edges and widths.  d_order (nullable):
// slab_order_bytes(n) bytes, filled for 2..kMaxOrderedProblems problems with
// their processing order (slab_order_ptrs gives the two arrays).
constexpr uint32_t kMaxOrderedProblems = 4096;
int slab_prep(void* d_probs, uint32_t n, cudaStream_t s, void* d_tables = nullptr, void* d_order = nullptr);
inline size_t slab_order_bytes(uint32_t n) { return (size_t)((n + 1u) & ~1u) * 4u + (size_t)(n + 1u) * 8u; }
inline void slab_order_ptrs(void* d_order, uint32_t n, const uint32_t** order, const uint64_t** begin) {
  *order = static_cast<const uint32_t*>(d_order);
  *begin = reinterpret_cast<const uint64_t*>(*order + ((n + 1u) & ~1u));
}
uint64_t slab_table_doubles(const mc_problem* src, uint32_t n);
int slab_history_launch(const SlabLaunch& L, cudaStream_t s);

// Event-based schedule (slab_event.cu): bank of `cap` particles in d_bank
// (slab_bank_bytes(cap) bytes); h_done is pinned host memory.  Synchronises
// `s` between batches of iterations.  capture_stream non-null: each batch is
// captured once on it into a graph, which is then launched on `s`.
size_t slab_bank_bytes(uint32_t cap);
int slab_event_run(const SlabLaunch& L, void* d_bank, uint32_t cap, unsigned int* h_done,
                   cudaStream_t capture_stream, cudaStream_t s);

// One run of the box transport (box.cu history schedule, box_event.cu event
// schedule).  Primaries are processed in chunks of primary_chunk; split
// children wait in two device banks of child_cap records each
// (generation ping-pong); d_child_count holds the two bank counts and
// h_count is pinned host memory for reading them back.
struct BoxLaunch {
  const void* d_probs;
  uint32_t n_problems;
  uint32_t chunk;
  uint64_t range_begin, total;
  uint64_t primary_chunk;
  unsigned long long* d_ticket;
  void* d_child[2];
  unsigned long long* d_child_count;
  unsigned long long* h_count;
  uint64_t child_cap;
  const mc_tally* tally;
  mc_lcg lcg;
  uint64_t event_cap;
  bool f32;
  int block, blocks_per_sm, num_sms;
  // event schedule only
  void* d_bank;
  uint32_t bank_cap;
  unsigned int* h_done;
  cudaStream_t capture_stream;
  uint32_t max_generations = 10000u;  // child generations (mc_limits)
  bool tally_agg = true;              // warp-aggregated mesh atomics
  uint64_t event_iterations = ~0ull;  // per generation (mc_limits; ~0: derived)
};

// One run of the pulse problem (pulse.cu).
struct PulseLaunch {
  const void* d_prob;
  uint64_t range_begin, total;
  uint32_t chunk;
  unsigned long long* d_ticket;
  const mc_tally* tally;
  mc_lcg lcg;
  uint64_t event_cap;
  int block, num_sms;
  uint32_t seeding;              // MC_SEED_*: selects the kernel variant
  uint32_t stack_depth;          // 1..256
  // Lane stacks of pending secondaries: pulse_stack_bytes(...) bytes.
  void* d_stack;
  size_t stack_bytes;
  // Overflow bank (hash modes; pulse_ovf_bytes(ovf_cap) bytes; nullptr: a
  // full stack drops, MC_ERR_CAPACITY) and a pinned count for the host loop.
  void* d_ovf;
  uint64_t ovf_cap;
  unsigned long long* h_count;
  uint32_t max_generations = 100000u;  // overflow generations (mc_limits)
  bool tally_agg = true;               // warp-aggregated tally atomics
};
size_t pulse_ovf_bytes(uint64_t cap);

size_t pulse_dev_size();
int pulse_fill_host(const mc_problem* src, void* dst);
int pulse_prep(void* d_prob, cudaStream_t s);
int pulse_run(const PulseLaunch& L, cudaStream_t s);
int pulse_stack_bytes(const PulseLaunch& L, size_t* bytes);

// Census phases with population control (pulse_census.cu).  d_buf holds
// pulse_census_bytes(groups, cap) bytes; the histories of `base` cover
// whole groups starting at group_begin.
struct PulseCensusLaunch {
  PulseLaunch base;
  const mc_pulse_spec* spec;
  void* d_buf;
  uint64_t groups, group_begin, cap;
};
uint64_t pulse_census_cap(const mc_pulse_spec& s, uint64_t groups);
size_t pulse_census_bytes(uint64_t groups, uint64_t cap);
int pulse_census_run(const PulseCensusLaunch& L, cudaStream_t s);

size_t box_dev_size();
size_t box_child_rec_size();
int box_fill_host(const mc_problem* src, uint32_t n, void* dst);
int box_prep(void* d_probs, uint32_t n, cudaStream_t s);
int box_history_run(const BoxLaunch& L, cudaStream_t s);
size_t box_bank_bytes(uint32_t cap);
int box_event_run(const BoxLaunch& L, cudaStream_t s);

}  // namespace mci
