// internal.h -- shared host-side plumbing of libmc (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/mc.h"

namespace mci {

// Thread-local message of the last failing call (returned by mc_last_error).
void set_error(const char* fmt, ...);

// Returns MC_ERR_CUDA with a message if `e` is an error, else MC_OK.
int cuda_status(cudaError_t e, const char* what);

#define MC_TRY_CUDA(expr)                                   \
  do {                                                      \
    int _st = ::mci::cuda_status((expr), #expr);            \
    if (_st != MC_OK) return _st;                           \
  } while (0)

// Validates an mc_lcg; fills `m`, `mask`.  Returns MC_OK or MC_ERR_ARG.
int check_lcg(const mc_lcg* lcg);

// Validates the problems of one mc_transport_run call against the tally and
// returns their total history count (MC_ERR_ARG with a message otherwise).
int check_problems(const mc_problem* p, uint32_t n, const mc_tally* t, uint64_t* total);
// Validates the fields of a run config; `who` prefixes the message.
int check_run_config(const mc_run_config* cfg, const char* who);
// Slab history launch defaults: histories per warp grab and block size.
uint32_t slab_default_chunk(uint64_t total, int num_sms);
int slab_default_block(uint64_t total, uint32_t chunk, int num_sms);
// Tally slots staged in shared memory for cfg->tally_mode (MC_ERR_ARG when
// mode 1 asks for more than fits).
int slab_staged_slots(const mc_run_config* cfg, const mc_tally* tally, size_t smem_optin, const char* who,
                      uint32_t* slots);

// Device scratch owned by a context.  Sizes only grow, and only outside
// the launch of a run (never inside a captured region).
struct DeviceBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int reserve(size_t want);  // grows with cudaMalloc; contents not kept
  void release();
};

// Default bounds on the waits of a run (mc_limits).
inline mc_limits default_limits() {
  mc_limits l{};
  l.pool_lock_attempts = 1u << 20;
  l.box_generations = 10000u;
  l.pulse_generations = 100000u;
  l.reserved = 0u;
  l.event_iterations = ~0ull;
  return l;
}

// Warp-aggregated tally atomics for a run: mc_run_config.tally_atomics 1
// (per lane) or 2 (aggregated), else the kernel's default.
inline bool tally_agg_of(uint32_t tally_atomics, bool kernel_default) {
  return tally_atomics == 0 ? kernel_default : tally_atomics == 2;
}
// Defaults (measured): one atomic per lane in every kernel.  The atomics are
// not the bound of any of them, so the grouping (a match, three reductions
// and a branch per contribution) costs more issue slots than it saves.
constexpr bool kSlabAggDefault = false;
constexpr bool kBoxAggDefault = false;
constexpr bool kPulseAggDefault = false;

// Instantiated launch graphs of the history schedule, keyed by launch shape.
struct GraphCache {
  std::unordered_map<uint64_t, cudaGraphExec_t> m;
};

}  // namespace mci

struct mc_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;  // max dynamic shared memory per block (opt-in)
  mc_limits limits = mci::default_limits();  // bounds on the waits of a run
  // Small scratch: work tickets, status word, count staging.
  mci::DeviceBuf scratch;
  // Device copy of the problem list and per-problem derived constants.
  mci::DeviceBuf problems;
  // Pinned host staging of the problem list (uploaded with cudaMemcpyAsync).
  void* h_problems = nullptr;
  size_t h_problems_bytes = 0;
  cudaEvent_t staged = nullptr;  // recorded after the last upload from h_problems
  // Host image of the problem records last uploaded and prepared: a call with
  // the same records (same kind and count) finds the device copy current and
  // skips the upload and the prep kernel.
  std::vector<unsigned char>* staged_image = nullptr;
  std::vector<unsigned char>* fill_scratch = nullptr;
  int staged_kind = -1;
  uint32_t staged_n = 0;
  // Event-based schedule: particle bank and a pinned completion flag.
  mci::DeviceBuf bank;
  unsigned int* h_done = nullptr;
  // Box transport: two banks of split children and a pinned count.
  mci::DeviceBuf children;
  unsigned long long* h_count = nullptr;
  // Pulse problem: two generation banks of secondaries that overflowed the
  // lane stacks (hash modes).
  mci::DeviceBuf overflow;
  // Pulse problem: the lane stacks of pending secondaries.
  mci::DeviceBuf pulse_stack;
  // Pulse census phases: bank counts, group weight totals and two banks.
  mci::DeviceBuf census;
  // Private stream used only to capture graphs (the caller's stream may be
  // the legacy default stream, which cannot be captured).
  cudaStream_t capture_stream = nullptr;
  mci::GraphCache* graphs = nullptr;
  // mc_lcg_draw_host: two device slots of a slice's states and digests, a
  // copy stream and the events that order the slots' reuse.
  mci::DeviceBuf host_io;
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_computed[2] = {nullptr, nullptr};
  cudaEvent_t io_copied[2] = {nullptr, nullptr};
  // Autotuner: scratch tally and the best configuration per workload shape.
  mci::DeviceBuf tune_tally;
  std::unordered_map<uint64_t, mc_run_config>* tune_cache = nullptr;
};
