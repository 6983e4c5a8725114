// api.cu -- contexts, errors, the transport front end and the tally read-back
// of libmc.  The device work lives in rng.cu and slab.cu; this file is host
// logic only: argument checks, staging of the problem list, launch sequence
// and conversion of int64 fixed-point tallies to flux.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstddef>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "internal.h"
#include "mc_device.cuh"
#include "transport.h"

namespace mci {

namespace {
thread_local std::string g_last_error;
}

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MC_OK;
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return MC_ERR_CUDA;
}

int check_lcg(const mc_lcg* lcg) {
  if (!lcg) {
    set_error("lcg is NULL");
    return MC_ERR_ARG;
  }
  if (lcg->m < 1 || lcg->m > 64 || lcg->reserved != 0) {
    set_error("lcg: m = %u outside 1..64 (or reserved != 0)", lcg->m);
    return MC_ERR_ARG;
  }
  if ((lcg->g & 1ull) == 0) {
    set_error("lcg: g must be odd");
    return MC_ERR_ARG;
  }
  return MC_OK;
}

int DeviceBuf::reserve(size_t want) {
  if (want <= bytes) return MC_OK;
  release();
  void* p = nullptr;
  int st = cuda_status(cudaMalloc(&p, want), "cudaMalloc(context scratch)");
  if (st != MC_OK) return st;
  ptr = p;
  bytes = want;
  return MC_OK;
}

void DeviceBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

}  // namespace mci

namespace {

// Layout of the small scratch block.
constexpr size_t kTicketOff = 0;     // unsigned long long ticket
constexpr size_t kScratchBytes = 256;

// Slab records are followed, 256-byte aligned, by every problem's bin edge
// and width tables (filled on the device by slab_prep).
// The tables are followed, 256-byte aligned, by the processing order of a
// launch of several problems (also filled by slab_prep).
size_t slab_tables_offset(uint32_t n) { return ((size_t)n * mci::slab_dev_size() + 255u) & ~(size_t)255u; }
size_t slab_order_offset(const mc_problem* problems, uint32_t n) {
  return (slab_tables_offset(n) + (size_t)mci::slab_table_doubles(problems, n) * sizeof(double) + 255u) &
         ~(size_t)255u;
}
size_t slab_stage_bytes(const mc_problem* problems, uint32_t n) {
  return slab_order_offset(problems, n) + mci::slab_order_bytes(n);
}
void* slab_tables_of(mc_ctx* ctx, uint32_t n) { return static_cast<char*>(ctx->problems.ptr) + slab_tables_offset(n); }
void* slab_order_of(mc_ctx* ctx, const mc_problem* problems, uint32_t n) {
  return static_cast<char*>(ctx->problems.ptr) + slab_order_offset(problems, n);
}

// Host half of staging: waits until the pinned buffer is free, sizes the
// buffers and writes the problem records into pinned memory.
int stage_host(mc_ctx* ctx, const mc_problem* problems, uint32_t n, size_t* bytes_out) {
  const bool box = problems[0].geometry == MC_GEOM_BOX;
  const size_t bytes = (size_t)n * (box ? mci::box_dev_size() : mci::slab_dev_size());
  if (problems[0].geometry == MC_GEOM_PULSE) {
    mci::set_error("graph replay covers the slab history schedule only");
    return MC_ERR_ARG;
  }
  if (ctx->staged) MC_TRY_CUDA(cudaEventSynchronize(ctx->staged));
  if (bytes > ctx->h_problems_bytes) {
    if (ctx->h_problems) cudaFreeHost(ctx->h_problems);
    ctx->h_problems = nullptr;
    ctx->h_problems_bytes = 0;
    MC_TRY_CUDA(cudaMallocHost(&ctx->h_problems, bytes));
    ctx->h_problems_bytes = bytes;
  }
  int st = ctx->problems.reserve(box ? bytes : slab_stage_bytes(problems, n));
  if (st != MC_OK) return st;
  if (box) mci::box_fill_host(problems, n, ctx->h_problems);
  else mci::slab_fill_host(problems, n, ctx->h_problems);
  ctx->staged_kind = -1;  // the graph uploads these records itself: the staging image no longer holds
  if (!ctx->staged) MC_TRY_CUDA(cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming));
  *bytes_out = bytes;
  return MC_OK;
}

int stage_problems(mc_ctx* ctx, const mc_problem* problems, uint32_t n, cudaStream_t s) {
  const bool box = problems[0].geometry == MC_GEOM_BOX;
  const bool pulse = problems[0].geometry == MC_GEOM_PULSE;
  const size_t bytes = pulse ? mci::pulse_dev_size()
                             : (size_t)n * (box ? mci::box_dev_size() : mci::slab_dev_size());
  const size_t dev_bytes = (pulse || box) ? bytes : slab_stage_bytes(problems, n);
  // Fill a host image first: if it equals the image last uploaded, the
  // device copy (base fields and the derived ones the prep kernel computes
  // from them) is still current.
  const int kind = pulse ? MC_GEOM_PULSE : (box ? MC_GEOM_BOX : MC_GEOM_SLAB);
  if (!ctx->fill_scratch) ctx->fill_scratch = new std::vector<unsigned char>();
  if (!ctx->staged_image) ctx->staged_image = new std::vector<unsigned char>();
  std::vector<unsigned char>& img = *ctx->fill_scratch;
  img.assign(bytes, 0);
  if (pulse) mci::pulse_fill_host(problems, img.data());
  else if (box) mci::box_fill_host(problems, n, img.data());
  else mci::slab_fill_host(problems, n, img.data());
  if (kind == ctx->staged_kind && n == ctx->staged_n && ctx->problems.bytes >= dev_bytes &&
      *ctx->staged_image == img)
    return MC_OK;
  cudaEvent_t* ev = &ctx->staged;
  if (*ev) MC_TRY_CUDA(cudaEventSynchronize(*ev));
  if (bytes > ctx->h_problems_bytes) {
    if (ctx->h_problems) cudaFreeHost(ctx->h_problems);
    ctx->h_problems = nullptr;
    ctx->h_problems_bytes = 0;
    MC_TRY_CUDA(cudaMallocHost(&ctx->h_problems, bytes));
    ctx->h_problems_bytes = bytes;
  }
  ctx->staged_kind = -1;  // until the upload below is enqueued
  int st = ctx->problems.reserve(dev_bytes);
  if (st != MC_OK) return st;
  std::memcpy(ctx->h_problems, img.data(), bytes);
  MC_TRY_CUDA(cudaMemcpyAsync(ctx->problems.ptr, ctx->h_problems, bytes, cudaMemcpyHostToDevice, s));
  if (!*ev) MC_TRY_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  MC_TRY_CUDA(cudaEventRecord(*ev, s));
  st = pulse ? mci::pulse_prep(ctx->problems.ptr, s)
             : (box ? mci::box_prep(ctx->problems.ptr, n, s)
                    : mci::slab_prep(ctx->problems.ptr, n, s, slab_tables_of(ctx, n),
                                     slab_order_of(ctx, problems, n)));
  if (st != MC_OK) return st;
  ctx->staged_image->swap(img);
  ctx->staged_kind = kind;
  ctx->staged_n = n;
  return MC_OK;
}

int check_box(const mc_problem& q, uint32_t i) {
  const mc_box_spec* b = q.box;
  if (!b) {
    mci::set_error("problem %u: box geometry without a box spec", i);
    return MC_ERR_ARG;
  }
  bool ok = b->side > 0.0 && std::isfinite(b->side) && b->inner_lo >= 0.0 && b->inner_lo < b->inner_hi &&
            b->inner_hi <= b->side && b->n_groups >= 1 && b->n_groups <= MC_BOX_MAX_GROUPS && b->mesh >= 1 &&
            b->mesh <= MC_BOX_MAX_MESH && b->max_split >= 1 && b->reserved == 0 &&
            (uint64_t)q.n_bins == (uint64_t)b->mesh * b->mesh * b->mesh;
  for (int r = 0; r < 2 && ok; ++r) {
    ok = b->sigma_t[r] > 0.0 && std::isfinite(b->sigma_t[r]) && b->c[r] >= 0.0 && b->c[r] <= 1.0 &&
         b->ww_low[r] >= 0.0 && b->ww_survive[r] > 0.0 && b->ww_high[r] > 0.0;
    for (uint32_t g = 0; g < b->n_groups && ok; ++g) ok = b->scatter_cdf[r][g][b->n_groups - 1] == 1.0;
  }
  if (!ok) {
    mci::set_error("problem %u: invalid box spec (extents, groups, mesh, windows, or a CDF row not ending at 1)",
                   i);
    return MC_ERR_ARG;
  }
  return MC_OK;
}

int check_problems(const mc_problem* p, uint32_t n, const mc_tally* t, uint64_t* total) {
  uint64_t acc = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const mc_problem& q = p[i];
    if (q.geometry != p[0].geometry || q.geometry > MC_GEOM_PULSE) {
      mci::set_error("problem %u: all problems of one call must share one geometry (slab, box or pulse)", i);
      return MC_ERR_ARG;
    }
    if (q.geometry == MC_GEOM_PULSE) {
      const mc_pulse_spec* ps = q.pulse;
      const bool ok = n == 1 && ps && ps->sigma_t > 0.0 && std::isfinite(ps->sigma_t) && ps->c >= 0.0 &&
                      ps->c <= 1.0 && ps->nu >= 1.0 && ps->nu <= 64.0 && ps->t_end > 0.0 &&
                      ps->t_end <= 1.0e6 && ps->x_half >= 0.0 && ps->n_reps >= 1 && ps->n_batches >= 1 &&
                      ps->per_batch >= 1 && ps->n_time_bins >= 1 && q.n_bins == ps->n_time_bins &&
                      (uint64_t)q.n_batches == (uint64_t)ps->n_reps * ps->n_batches &&
                      q.n_histories == (uint64_t)ps->n_reps * ps->n_batches * ps->per_batch &&
                      q.seeding <= MC_SEED_HASH_HIER && q.reserved == 0 &&
                      (ps->n_census < 2 || (q.seeding != MC_SEED_STRIDE && ps->n_census <= (1u << 20) &&
                                            ps->pc_target <= (1u << 30) &&
                                            (uint64_t)ps->n_reps * ps->n_batches < (1ull << 32)));
      if (!ok) {
        mci::set_error("problem %u: invalid pulse problem (one problem per call; spec, n_bins = n_time_bins, "
                       "n_batches = reps * batches, n_histories = reps * batches * per_batch; census phases "
                       "need hash seeding, n_census <= 2^20, pc_target <= 2^30)", i);
        return MC_ERR_ARG;
      }
      const uint64_t slots = (uint64_t)q.n_bins * q.n_batches;
      if (q.tally_offset > t->n_slots || slots > t->n_slots - q.tally_offset) {
        mci::set_error("problem %u: pulse tally slots outside the tally", i);
        return MC_ERR_ARG;
      }
      acc += q.n_histories;
      continue;
    }
    if (q.geometry == MC_GEOM_BOX) {
      int st = check_box(q, i);
      if (st != MC_OK) return st;
      if (q.n_batches == 0 || q.source != MC_SRC_ISOTROPIC || q.seeding > MC_SEED_HASH_HIER || q.reserved != 0) {
        mci::set_error("problem %u: bad n_batches/source/seeding for a box", i);
        return MC_ERR_ARG;
      }
      const uint64_t slots = (uint64_t)q.n_bins * q.n_batches;
      if (q.tally_offset > t->n_slots || slots > t->n_slots - q.tally_offset) {
        mci::set_error("problem %u: mesh slots outside the tally", i);
        return MC_ERR_ARG;
      }
      acc += q.n_histories;
      continue;
    }
    if (!(q.L > 0.0) || !(q.sigma_t > 0.0) || !(q.c >= 0.0 && q.c <= 1.0) || !std::isfinite(q.L) ||
        !std::isfinite(q.sigma_t)) {
      mci::set_error("problem %u: need L > 0, sigma_t > 0, 0 <= c <= 1", i);
      return MC_ERR_ARG;
    }
    if (q.n_bins == 0 || q.n_batches == 0 || q.source > MC_SRC_BEAM || q.seeding > MC_SEED_HASH_HIER ||
        q.reserved != 0) {
      mci::set_error("problem %u: bad n_bins/n_batches/source/seeding", i);
      return MC_ERR_ARG;
    }
    const uint64_t slots = (uint64_t)q.n_bins * q.n_batches;
    if (q.tally_offset > t->n_slots || slots > t->n_slots - q.tally_offset) {
      mci::set_error("problem %u: tally slots [%llu, +%llu) outside the tally (%llu slots)", i,
                     (unsigned long long)q.tally_offset, (unsigned long long)slots,
                     (unsigned long long)t->n_slots);
      return MC_ERR_ARG;
    }
    acc += q.n_histories;
  }
  *total = acc;
  return MC_OK;
}

constexpr uint64_t kChildCap = 1ull << 22;      // child records per bank
constexpr uint64_t kPrimaryChunk = 1ull << 22;  // source histories per generation-0 launch

int run_box(mc_ctx* ctx, const mc_lcg* lcg, uint32_t n_problems, const mc_run_config* cfg, const mc_tally* tally,
            uint64_t rb, uint64_t re, unsigned long long* ticket, cudaStream_t s) {
  const size_t rec = mci::box_child_rec_size();
  int st = ctx->children.reserve(2 * kChildCap * rec);
  if (st != MC_OK) return st;
  if (!ctx->h_count) MC_TRY_CUDA(cudaMallocHost(&ctx->h_count, sizeof(unsigned long long)));
  mci::BoxLaunch L{};
  L.d_probs = ctx->problems.ptr;
  L.n_problems = n_problems;
  L.chunk = cfg->chunk ? cfg->chunk : 32u;
  L.range_begin = rb;
  L.total = re - rb;
  L.primary_chunk = kPrimaryChunk;
  L.d_ticket = ticket;
  L.d_child[0] = ctx->children.ptr;
  L.d_child[1] = static_cast<char*>(ctx->children.ptr) + kChildCap * rec;
  L.d_child_count = ticket + 1;  // scratch words 1 and 2
  L.h_count = ctx->h_count;
  L.child_cap = kChildCap;
  L.tally = tally;
  L.lcg = *lcg;
  // Box particles end by leaking or by roulette within a few hundred flights;
  // the default cap of 2^22 flights per particle only bounds pathologies.
  L.event_cap = cfg->event_cap ? cfg->event_cap : (1ull << 22);
  L.f32 = cfg->precision == MC_FP32_GUARDED;
  // the box kernel is built for at most 256 threads per block (3 blocks per SM)
  L.block = cfg->block ? (int)std::min<uint32_t>(cfg->block, 256u) : 256;
  L.blocks_per_sm = (int)cfg->blocks_per_sm;
  L.num_sms = ctx->num_sms;
  L.max_generations = ctx->limits.box_generations;
  L.tally_agg = mci::tally_agg_of(cfg->tally_atomics, mci::kBoxAggDefault);
  L.event_iterations = ctx->limits.event_iterations;
  if (cfg->schedule == MC_SCHED_EVENT) {
    // Two banks of up to 2^21 particles (about 0.55 GiB fp64); allocated on first use.
    const uint32_t cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(L.total, 1), 1u << 21);
    st = ctx->bank.reserve(mci::box_bank_bytes(cap));
    if (st != MC_OK) return st;
    if (!ctx->h_done) MC_TRY_CUDA(cudaMallocHost(&ctx->h_done, sizeof(unsigned int)));
    if (cfg->use_graph && !ctx->capture_stream)
      MC_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    L.d_bank = ctx->bank.ptr;
    L.bank_cap = cap;
    L.h_done = ctx->h_done;
    L.capture_stream = cfg->use_graph ? ctx->capture_stream : nullptr;
    return mci::box_event_run(L, s);
  }
  return mci::box_history_run(L, s);
}

}  // namespace

namespace mci {

int check_problems(const mc_problem* p, uint32_t n, const mc_tally* t, uint64_t* total) {
  return ::check_problems(p, n, t, total);
}

int check_run_config(const mc_run_config* cfg, const char* who) {
  if (cfg->schedule > MC_SCHED_AUTO || cfg->precision > MC_FP32_GUARDED || cfg->tally_mode > 2 ||
      (cfg->block != 0 && (cfg->block % 32 != 0 || cfg->block > 512)) || cfg->stack_depth > 256 ||
      cfg->tally_atomics > 2) {
    set_error("%s: bad run config (schedule/precision/tally_mode/block/stack_depth/tally_atomics)", who);
    return MC_ERR_ARG;
  }
  return MC_OK;
}

// About four grabs per resident warp: fine-grained enough to balance
// long-tailed histories, coarse enough that lanes rarely change problem in
// a batched launch; within [32, 1024].
uint32_t slab_default_chunk(uint64_t total, int num_sms) {
  return (uint32_t)std::min<uint64_t>(1024, std::max<uint64_t>(32, total / ((uint64_t)num_sms * 256)));
}

// 256 threads, except that a run too small to give every SM a block of 256
// is spread over all SMs in smaller blocks: its time is the latency of its
// longest warps, which run faster with fewer warps per sub-partition.
int slab_default_block(uint64_t total, uint32_t chunk, int num_sms) {
  const uint64_t warps = (total + chunk - 1) / chunk;
  if (warps * 32 < (uint64_t)num_sms * 256)
    return (int)std::max<uint64_t>(32, 32 * std::max<uint64_t>(1, warps / (uint64_t)num_sms));
  return 256;
}

// Slots staged in shared memory: all of them (tally_mode 1, an error when
// they do not fit beside 2 KiB of the kernel's own static shared memory),
// none (mode 2), or all when at most 8192 (64 KiB; mode 0, "auto").
int slab_staged_slots(const mc_run_config* cfg, const mc_tally* tally, size_t smem_optin, const char* who,
                      uint32_t* slots) {
  const bool fits = tally->n_slots * 8u + 2048u <= smem_optin;
  if (cfg->tally_mode == 1 && !fits) {
    set_error("%s: %llu tally slots do not fit in shared memory", who, (unsigned long long)tally->n_slots);
    return MC_ERR_ARG;
  }
  const bool stage = cfg->tally_mode == 1 || (cfg->tally_mode == 0 && tally->n_slots <= 8192u);
  *slots = stage ? (uint32_t)tally->n_slots : 0u;
  return MC_OK;
}

}  // namespace mci

extern "C" {

MC_API const char* mc_last_error(void) { return mci::g_last_error.c_str(); }

MC_API int mc_ctx_create(mc_ctx** out, int device) {
  if (!out) {
    mci::set_error("mc_ctx_create: out is NULL");
    return MC_ERR_ARG;
  }
  *out = nullptr;
  MC_TRY_CUDA(cudaSetDevice(device));
  mc_ctx* c = new mc_ctx();
  c->device = device;
  c->tune_cache = new std::unordered_map<uint64_t, mc_run_config>();
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = (size_t)optin;
  int st = c->scratch.reserve(kScratchBytes);
  if (st != MC_OK) {
    delete c;
    return st;
  }
  st = mci::cuda_status(cudaMemset(c->scratch.ptr, 0, kScratchBytes), "cudaMemset(scratch)");
  if (st != MC_OK) {
    c->scratch.release();
    delete c;
    return st;
  }
  *out = c;
  return MC_OK;
}

MC_API int mc_ctx_set_limits(mc_ctx* ctx, const mc_limits* limits) {
  if (!ctx) {
    mci::set_error("mc_ctx_set_limits: ctx is NULL");
    return MC_ERR_ARG;
  }
  if (limits && limits->reserved != 0) {
    mci::set_error("mc_ctx_set_limits: reserved field must be 0");
    return MC_ERR_ARG;
  }
  ctx->limits = limits ? *limits : mci::default_limits();
  return MC_OK;
}

MC_API int mc_ctx_get_limits(const mc_ctx* ctx, mc_limits* out) {
  if (!ctx || !out) {
    mci::set_error("mc_ctx_get_limits: NULL argument");
    return MC_ERR_ARG;
  }
  *out = ctx->limits;
  return MC_OK;
}

MC_API void mc_ctx_destroy(mc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->staged) cudaEventDestroy(ctx->staged);
  ctx->scratch.release();
  ctx->problems.release();
  ctx->bank.release();
  if (ctx->h_problems) cudaFreeHost(ctx->h_problems);
  if (ctx->h_done) cudaFreeHost(ctx->h_done);
  if (ctx->h_count) cudaFreeHost(ctx->h_count);
  ctx->children.release();
  ctx->census.release();
  delete ctx->staged_image;
  delete ctx->fill_scratch;
  ctx->overflow.release();
  ctx->pulse_stack.release();
  ctx->tune_tally.release();
  delete ctx->tune_cache;
  if (ctx->graphs) {
    for (auto& kv : ctx->graphs->m) cudaGraphExecDestroy(kv.second);
    delete ctx->graphs;
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  ctx->host_io.release();
  if (ctx->io_stream) cudaStreamDestroy(ctx->io_stream);
  for (int k = 0; k < 2; ++k) {
    if (ctx->io_computed[k]) cudaEventDestroy(ctx->io_computed[k]);
    if (ctx->io_copied[k]) cudaEventDestroy(ctx->io_copied[k]);
  }
  delete ctx;
}

MC_API uint64_t mc_hash64(uint64_t k, uint64_t s) { return mcd::hash64(k, s); }

}  // extern "C"

namespace {

// Validates a call; returns the total history count in *total.
int validate_run(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                 const mc_run_config* cfg, const mc_tally* tally, uint64_t* total) {
  if (!ctx || !problems || n_problems == 0 || !cfg || !tally || !tally->d_bins || !tally->d_counts) {
    mci::set_error("mc_transport_run: NULL argument or no problems");
    return MC_ERR_ARG;
  }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  st = check_problems(problems, n_problems, tally, total);
  if (st != MC_OK) return st;
  st = mci::check_run_config(cfg, "mc_transport_run");
  if (st != MC_OK) return st;
  const uint64_t rb = cfg->range_begin, re = cfg->range_end == 0 ? *total : cfg->range_end;
  if (rb > re || re > *total) {
    mci::set_error("mc_transport_run: range [%llu, %llu) outside the %llu histories", (unsigned long long)rb,
                   (unsigned long long)re, (unsigned long long)*total);
    return MC_ERR_ARG;
  }
  if (problems[0].geometry == MC_GEOM_PULSE && problems[0].pulse->n_census >= 2 &&
      (rb % problems[0].pulse->per_batch != 0 || re % problems[0].pulse->per_batch != 0)) {
    mci::set_error("pulse census phases: the history range must cover whole (rep, batch) groups");
    return MC_ERR_ARG;
  }
  return MC_OK;
}

uint64_t total_histories(const mc_problem* p, uint32_t n) {
  uint64_t t = 0;
  for (uint32_t i = 0; i < n; ++i) t += p[i].n_histories;
  return t;
}

int make_slab_launch(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                     const mc_run_config* cfg, const mc_tally* tally, uint64_t rb, uint64_t re,
                     unsigned long long* ticket, mci::SlabLaunch* out) {
  mci::SlabLaunch L{};
  L.single_n_bins = n_problems == 1 ? problems[0].n_bins : 0u;
  L.d_probs = ctx->problems.ptr;
  L.d_tables = slab_tables_of(ctx, n_problems);
  L.n_problems = n_problems;
  // A launch of all the histories of 2..kMaxOrderedProblems problems takes
  // them in the order the prep kernel ranked (longest expected chains first).
  if (n_problems >= 2 && n_problems <= mci::kMaxOrderedProblems && rb == 0 && re == total_histories(problems, n_problems))
    mci::slab_order_ptrs(slab_order_of(ctx, problems, n_problems), n_problems, &L.d_order, &L.d_order_begin);
  L.chunk = cfg->chunk ? cfg->chunk : mci::slab_default_chunk(re - rb, ctx->num_sms);
  L.range_begin = rb;
  L.total = re - rb;
  L.d_ticket = ticket;
  L.tally = tally;
  L.lcg = *lcg;
  L.event_cap = cfg->event_cap ? cfg->event_cap : (1ull << 40);
  uint32_t slots = 0;
  int st = mci::slab_staged_slots(cfg, tally, ctx->smem_optin, "mc_transport_run", &slots);
  if (st != MC_OK) return st;
  L.smem_slots = slots;
  L.f32 = cfg->precision == MC_FP32_GUARDED;
  L.block = cfg->block ? (int)cfg->block : mci::slab_default_block(L.total, L.chunk, ctx->num_sms);
  L.blocks_per_sm = (int)cfg->blocks_per_sm;
  L.num_sms = ctx->num_sms;
  L.pool_lock_attempts = ctx->limits.pool_lock_attempts;
  L.event_iterations = ctx->limits.event_iterations;
  L.tally_agg = mci::tally_agg_of(cfg->tally_atomics, mci::kSlabAggDefault);
  *out = L;
  return MC_OK;
}

uint64_t fnv(uint64_t h, const void* p, size_t n);

// History schedule as one CUDA graph per launch shape: problem upload from
// the pinned staging buffer, prep kernel, memsets and the persistent kernel
// are captured once; later calls refresh the pinned records and replay.
int run_slab_graph(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                   const mc_run_config* cfg, const mc_tally* tally, uint64_t rb, uint64_t re, cudaStream_t s) {
  size_t bytes = 0;
  int st = stage_host(ctx, problems, n_problems, &bytes);
  if (st != MC_OK) return st;
  auto* ticket = reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->scratch.ptr) + kTicketOff);
  mci::SlabLaunch L{};
  st = make_slab_launch(ctx, lcg, problems, n_problems, cfg, tally, rb, re, ticket, &L);
  if (st != MC_OK) return st;
  uint64_t key = 1469598103934665603ull;
  const void* ptrs[] = {ctx->problems.ptr, ctx->h_problems, tally->d_bins, tally->d_counts, tally->d_hist_state,
                        tally->d_hist_draws};
  key = fnv(key, ptrs, sizeof ptrs);
  key = fnv(key, cfg, sizeof *cfg);
  key = fnv(key, &ctx->limits, sizeof ctx->limits);  // the lock bound is a kernel argument
  key = fnv(key, lcg, sizeof *lcg);
  key = fnv(key, &n_problems, sizeof n_problems);
  key = fnv(key, &bytes, sizeof bytes);
  key = fnv(key, &tally->n_slots, sizeof tally->n_slots);
  // the history range and the launch's shape are baked into the graph (the
  // kernel's ticket bound, its grid, chunk and block): a call whose problems
  // hold another number of histories captures a graph of its own
  key = fnv(key, &L.range_begin, sizeof L.range_begin);
  key = fnv(key, &L.total, sizeof L.total);
  key = fnv(key, &L.chunk, sizeof L.chunk);
  key = fnv(key, &L.block, sizeof L.block);
  key = fnv(key, &L.single_n_bins, sizeof L.single_n_bins);
  if (!ctx->graphs) ctx->graphs = new mci::GraphCache();
  auto it = ctx->graphs->m.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it != ctx->graphs->m.end()) {
    exec = it->second;
  } else {
    if (!ctx->capture_stream) MC_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    if (ctx->graphs->m.size() >= 16) {
      for (auto& kv : ctx->graphs->m) cudaGraphExecDestroy(kv.second);
      ctx->graphs->m.clear();
    }
    cudaStream_t cs = ctx->capture_stream;
    cudaGraph_t g = nullptr;
    MC_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaMemcpyAsync(ctx->problems.ptr, ctx->h_problems, bytes, cudaMemcpyHostToDevice, cs);
    mci::slab_prep(ctx->problems.ptr, n_problems, cs, slab_tables_of(ctx, n_problems),
                   slab_order_of(ctx, problems, n_problems));
    if (!cfg->accumulate) {
      cudaMemsetAsync(tally->d_bins, 0, tally->n_slots * sizeof(int64_t), cs);
      cudaMemsetAsync(tally->d_counts, 0, (size_t)n_problems * MC_NCOUNT * sizeof(uint64_t), cs);
    }
    cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), cs);
    const int lst = mci::slab_history_launch(L, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (lst != MC_OK) {
      if (g) cudaGraphDestroy(g);
      return lst;
    }
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaStreamEndCapture(history run)");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaGraphInstantiate(history run)");
    ctx->graphs->m[key] = exec;
  }
  MC_TRY_CUDA(cudaGraphLaunch(exec, s));
  MC_TRY_CUDA(cudaEventRecord(ctx->staged, s));
  return MC_OK;
}

// Runs a validated call whose schedule is HISTORY or EVENT.
int transport_run_impl(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                       const mc_run_config* cfg, const mc_tally* tally, uint64_t total, cudaStream_t s) {
  int st = MC_OK;
  const uint64_t rb = cfg->range_begin, re = cfg->range_end == 0 ? total : cfg->range_end;
  MC_TRY_CUDA(cudaSetDevice(ctx->device));
  if (cfg->use_graph && cfg->schedule == MC_SCHED_HISTORY && problems[0].geometry == MC_GEOM_SLAB && re > rb)
    return run_slab_graph(ctx, lcg, problems, n_problems, cfg, tally, rb, re, s);

  st = stage_problems(ctx, problems, n_problems, s);
  if (st != MC_OK) return st;
  if (!cfg->accumulate) {
    MC_TRY_CUDA(cudaMemsetAsync(tally->d_bins, 0, tally->n_slots * sizeof(int64_t), s));
    MC_TRY_CUDA(cudaMemsetAsync(tally->d_counts, 0, (size_t)n_problems * MC_NCOUNT * sizeof(uint64_t), s));
  }
  auto* ticket = reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->scratch.ptr) + kTicketOff);
  MC_TRY_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
  if (re == rb) return MC_OK;

  if (problems[0].geometry == MC_GEOM_BOX) return run_box(ctx, lcg, n_problems, cfg, tally, rb, re, ticket, s);
  if (problems[0].geometry == MC_GEOM_PULSE) {
    mci::PulseLaunch P{};
    P.d_prob = ctx->problems.ptr;
    P.range_begin = rb;
    P.total = re - rb;
    P.chunk = cfg->chunk ? cfg->chunk : 32u;
    P.d_ticket = ticket;
    P.tally = tally;
    P.lcg = *lcg;
    P.event_cap = cfg->event_cap ? cfg->event_cap : (1ull << 24);
    P.block = cfg->block ? (int)std::min<uint32_t>(cfg->block, 256u) : 128;
    P.num_sms = ctx->num_sms;
    P.stack_depth = cfg->stack_depth ? cfg->stack_depth : 256u;
    P.seeding = problems[0].seeding;
    P.max_generations = ctx->limits.pulse_generations;
    P.tally_agg = mci::tally_agg_of(cfg->tally_atomics, mci::kPulseAggDefault);
    if (problems[0].seeding != MC_SEED_STRIDE) {
      // overflow bank of 2^20 secondaries (32 MiB per generation bank)
      P.ovf_cap = 1ull << 20;
      st = ctx->overflow.reserve(mci::pulse_ovf_bytes(P.ovf_cap));
      if (st != MC_OK) return st;
      if (!ctx->h_count) MC_TRY_CUDA(cudaMallocHost(&ctx->h_count, sizeof(unsigned long long)));
      P.d_ovf = ctx->overflow.ptr;
      P.h_count = ctx->h_count;
    }
    const mc_pulse_spec* ps = problems[0].pulse;
    if (ps->n_census < 2) {
      size_t sb = 0;
      st = mci::pulse_stack_bytes(P, &sb);
      if (st != MC_OK) return st;
      st = ctx->pulse_stack.reserve(sb);
      if (st != MC_OK) return st;
      P.d_stack = ctx->pulse_stack.ptr;
      P.stack_bytes = sb;
      return mci::pulse_run(P, s);
    }
    if (rb % ps->per_batch != 0 || re % ps->per_batch != 0) {  // (also checked by validate_run)
      mci::set_error("pulse census phases: the history range must cover whole (rep, batch) groups");
      return MC_ERR_ARG;
    }
    mci::PulseCensusLaunch C{};
    C.base = P;
    C.spec = ps;
    C.groups = (re - rb) / ps->per_batch;
    C.group_begin = rb / ps->per_batch;
    C.cap = mci::pulse_census_cap(*ps, C.groups);
    st = ctx->census.reserve(mci::pulse_census_bytes(C.groups, C.cap));
    if (st != MC_OK) return st;
    C.d_buf = ctx->census.ptr;
    return mci::pulse_census_run(C, s);
  }

  mci::SlabLaunch L{};
  st = make_slab_launch(ctx, lcg, problems, n_problems, cfg, tally, rb, re, ticket, &L);
  if (st != MC_OK) return st;
  if (cfg->schedule == MC_SCHED_EVENT) {
    // Two banks of up to 2^21 particles (about 0.35 GiB fp64); allocated on first use.
    const uint32_t cap = (uint32_t)std::min<uint64_t>(L.total, 1u << 21);
    st = ctx->bank.reserve(mci::slab_bank_bytes(cap));
    if (st != MC_OK) return st;
    if (!ctx->h_done) MC_TRY_CUDA(cudaMallocHost(&ctx->h_done, sizeof(unsigned int)));
    if (cfg->use_graph && !ctx->capture_stream)
      MC_TRY_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    return mci::slab_event_run(L, ctx->bank.ptr, cap, ctx->h_done, cfg->use_graph ? ctx->capture_stream : nullptr,
                               s);
  }
  return mci::slab_history_launch(L, s);
}

// FNV-1a over the bytes that decide the best launch shape.
uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t tune_key(const mc_problem* problems, uint32_t n, const mc_run_config* cfg, const mc_tally* tally,
                  uint64_t total) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &n, sizeof n);
  h = fnv(h, &total, sizeof total);
  h = fnv(h, &cfg->precision, sizeof cfg->precision);
  h = fnv(h, &cfg->tally_mode, sizeof cfg->tally_mode);
  h = fnv(h, &tally->n_slots, sizeof tally->n_slots);
  for (uint32_t i = 0; i < n; ++i) {
    const mc_problem& q = problems[i];
    h = fnv(h, &q, offsetof(mc_problem, box));
    if (q.box) h = fnv(h, q.box, sizeof(mc_box_spec));
  }
  return h;
}

int autotune_impl(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                  const mc_run_config* base, const mc_tally* tally, uint64_t total, mc_run_config* best,
                  float* best_ms, cudaStream_t s) {
  // Scratch tally: the caller's tally is never written while tuning.
  const size_t bins = tally->n_slots * sizeof(int64_t), cnts = (size_t)n_problems * MC_NCOUNT * sizeof(uint64_t);
  int st = ctx->tune_tally.reserve(bins + cnts);
  if (st != MC_OK) return st;
  mc_tally t2{};
  t2.d_bins = static_cast<int64_t*>(ctx->tune_tally.ptr);
  t2.n_slots = tally->n_slots;
  t2.d_counts = reinterpret_cast<uint64_t*>(static_cast<char*>(ctx->tune_tally.ptr) + bins);
  // A sample from the middle of the concatenated history list: all of it up
  // to 2^17 histories, else a quarter (at least 2^17).
  uint64_t S = total <= (1ull << 17) ? total : std::max<uint64_t>(1ull << 17, total / 4);
  uint64_t start = (total - S) / 2;
  if (problems[0].geometry == MC_GEOM_PULSE) {  // whole (rep, batch) groups (census phases need them)
    const uint64_t pb = problems[0].pulse->per_batch;
    start -= start % pb;
    S = std::min<uint64_t>(total - start, (S + pb - 1) / pb * pb);
  }
  struct Cand { uint32_t schedule, block, chunk, graph; };
  const bool box = problems[0].geometry == MC_GEOM_BOX;
  // Chunks relative to the default for the full run (histories per warp
  // grab; see transport_run_impl), so the sample ranks them as the run would.
  const uint64_t c0 = std::min<uint64_t>(1024, std::max<uint64_t>(32, total / ((uint64_t)ctx->num_sms * 256)));
  std::vector<Cand> cands;
  for (uint32_t b : box ? std::vector<uint32_t>{128u, 256u} : std::vector<uint32_t>{128u, 256u, 512u})
    for (uint64_t c : {c0 / 4, c0, c0 * 4})
      cands.push_back({MC_SCHED_HISTORY, b, (uint32_t)std::max<uint64_t>(8, c), 0u});
  cands.push_back({MC_SCHED_EVENT, 256u, 0u, 1u});
  cudaEvent_t e0, e1;
  MC_TRY_CUDA(cudaEventCreate(&e0));
  MC_TRY_CUDA(cudaEventCreate(&e1));
  // a warm-up run, then one timed run of r
  auto time_run = [&](mc_run_config& r, float* ms) {
    int rs = transport_run_impl(ctx, lcg, problems, n_problems, &r, &t2, total, s);
    if (rs == MC_OK) rs = mci::cuda_status(cudaEventRecord(e0, s), "cudaEventRecord");
    if (rs == MC_OK) rs = transport_run_impl(ctx, lcg, problems, n_problems, &r, &t2, total, s);
    if (rs == MC_OK) rs = mci::cuda_status(cudaEventRecord(e1, s), "cudaEventRecord");
    if (rs == MC_OK) rs = mci::cuda_status(cudaEventSynchronize(e1), "cudaEventSynchronize");
    if (rs == MC_OK) cudaEventElapsedTime(ms, e0, e1);
    return rs;
  };
  float best_t = 0.0f;
  bool have = false;
  mc_run_config best_hist{}, event{};
  float best_hist_t = 0.0f;
  bool have_hist = false, have_event = false;
  for (const Cand& c : cands) {
    mc_run_config r = *base;
    r.schedule = c.schedule;
    r.block = c.block;
    r.chunk = c.chunk;
    r.use_graph = c.graph;
    r.accumulate = 0;
    r.range_begin = start;
    r.range_end = start + S;
    float ms = 0.0f;
    st = time_run(r, &ms);
    if (st != MC_OK) break;
    if (!have || ms < best_t) {
      best_t = ms;
      *best = r;
      have = true;
    }
    if (c.schedule == MC_SCHED_HISTORY && (!have_hist || ms < best_hist_t)) {
      best_hist_t = ms;
      best_hist = r;
      have_hist = true;
    }
    if (c.schedule == MC_SCHED_EVENT) {
      event = r;
      have_event = true;
    }
  }
  // A sample ranks shapes as they behave on a quarter of the histories, not
  // on the whole: the history schedule's tail is a larger share of a small
  // run, and a chunk that balances a quarter can be too fine or too coarse
  // for the whole (256 batched problems: chunks of 1/4 or 4 times the
  // default take 45-50 ms against 20 ms).  So, whenever the sample is not
  // the whole range, the sample's winner, the best history shape and the
  // library's default shape are timed again on the whole range and the
  // fastest of them is kept.
  if (st == MC_OK && have && S < total) {
    mc_run_config dflt = *base;
    dflt.schedule = MC_SCHED_HISTORY;
    dflt.block = 0;
    dflt.chunk = 0;
    dflt.use_graph = 0;
    dflt.accumulate = 0;
    std::vector<mc_run_config> finals{*best, dflt};
    if (have_hist) finals.push_back(best_hist);
    float best_full = 0.0f;
    mc_run_config pick = *best;
    for (size_t i = 0; i < finals.size() && st == MC_OK; ++i) {
      mc_run_config r = finals[i];
      r.range_begin = 0;
      r.range_end = total;
      // the better of two timings: shapes within a few per cent of each
      // other trade places from one run to the next
      float ms = 0.0f, ms2 = 0.0f;
      st = time_run(r, &ms);
      if (st == MC_OK) st = time_run(r, &ms2);
      ms = std::min(ms, ms2);
      if (st == MC_OK && (i == 0 || ms < best_full)) {
        best_full = ms;
        pick = finals[i];
      }
    }
    if (st == MC_OK) {
      *best = pick;
      best_t = best_full;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MC_OK) return st;
  best->range_begin = base->range_begin;
  best->range_end = base->range_end;
  best->accumulate = base->accumulate;
  if (best_ms) *best_ms = best_t;
  (*ctx->tune_cache)[tune_key(problems, n_problems, base, tally, total)] = *best;
  return MC_OK;
}

}  // namespace

extern "C" {

MC_API int mc_transport_run(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems,
                            uint32_t n_problems, const mc_run_config* cfg, const mc_tally* tally,
                            void* stream) {
  uint64_t total = 0;
  int st = validate_run(ctx, lcg, problems, n_problems, cfg, tally, &total);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (cfg->schedule != MC_SCHED_AUTO) return transport_run_impl(ctx, lcg, problems, n_problems, cfg, tally, total, s);
  MC_TRY_CUDA(cudaSetDevice(ctx->device));
  mc_run_config r{};
  auto it = ctx->tune_cache->find(tune_key(problems, n_problems, cfg, tally, total));
  if (it != ctx->tune_cache->end()) {
    r = it->second;
  } else {
    st = autotune_impl(ctx, lcg, problems, n_problems, cfg, tally, total, &r, nullptr, s);
    if (st != MC_OK) return st;
  }
  r.range_begin = cfg->range_begin;
  r.range_end = cfg->range_end;
  r.accumulate = cfg->accumulate;
  r.event_cap = cfg->event_cap;
  return transport_run_impl(ctx, lcg, problems, n_problems, &r, tally, total, s);
}

MC_API int mc_autotune(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                       const mc_run_config* base, const mc_tally* tally, mc_run_config* best, float* best_ms,
                       void* stream) {
  uint64_t total = 0;
  int st = validate_run(ctx, lcg, problems, n_problems, base, tally, &total);
  if (st != MC_OK) return st;
  if (!best) {
    mci::set_error("mc_autotune: best is NULL");
    return MC_ERR_ARG;
  }
  if (total == 0) {
    *best = *base;
    best->schedule = MC_SCHED_HISTORY;
    if (best_ms) *best_ms = 0.0f;
    return MC_OK;
  }
  MC_TRY_CUDA(cudaSetDevice(ctx->device));
  return autotune_impl(ctx, lcg, problems, n_problems, base, tally, total, best, best_ms, (cudaStream_t)stream);
}

MC_API int mc_tally_read(mc_ctx* ctx, const mc_problem* problems, uint32_t problem, const mc_tally* tally,
                         double* h_flux, double* h_rel_err, double* h_batch, int64_t* h_raw,
                         uint64_t* h_counts, void* stream) {
  if (!ctx || !problems || !tally || !tally->d_bins || !tally->d_counts || !h_flux) {
    mci::set_error("mc_tally_read: NULL argument");
    return MC_ERR_ARG;
  }
  const mc_problem& p = problems[problem];
  const uint32_t nb = p.n_bins, nbat = p.n_batches;
  const uint64_t slots = (uint64_t)nb * nbat;
  if (nb == 0 || nbat == 0 || p.tally_offset > tally->n_slots || slots > tally->n_slots - p.tally_offset) {
    mci::set_error("mc_tally_read: problem %u does not fit the tally", problem);
    return MC_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  MC_TRY_CUDA(cudaSetDevice(ctx->device));
  std::vector<int64_t> raw(slots);
  std::vector<uint64_t> cnt(MC_NCOUNT);
  MC_TRY_CUDA(cudaMemcpyAsync(raw.data(), tally->d_bins + p.tally_offset, slots * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
  MC_TRY_CUDA(cudaMemcpyAsync(cnt.data(), tally->d_counts + (size_t)problem * MC_NCOUNT,
                              MC_NCOUNT * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  MC_TRY_CUDA(cudaStreamSynchronize(s));
  if (h_raw) std::memcpy(h_raw, raw.data(), slots * sizeof(int64_t));
  if (h_counts) std::memcpy(h_counts, cnt.data(), MC_NCOUNT * sizeof(uint64_t));

  // Cell volume per bin: slab width L/n_bins, or the cube of the mesh pitch.
  double vol = p.L / (double)nb;
  if (p.geometry == MC_GEOM_BOX && p.box) {
    const double h = p.box->side / (double)p.box->mesh;
    vol = h * h * h;
  }
  if (p.geometry == MC_GEOM_PULSE && p.pulse) vol = 2.0 * p.pulse->x_half;  // unit time bins
  const double scale = std::ldexp(1.0, -32);
  const uint64_t N = p.n_histories;
  bool overflow = false;
  std::vector<double> total(nb, 0.0);
  std::vector<double> batch(slots, 0.0);
  for (uint32_t k = 0; k < nbat; ++k) {
    // Batch k holds the ids with floor(id * nbat / N) == k.
    const uint64_t lo = (uint64_t)(((unsigned __int128)k * N + nbat - 1) / nbat);
    const uint64_t hi = (uint64_t)(((unsigned __int128)(k + 1) * N + nbat - 1) / nbat);
    const double nk = (double)(hi - lo);
    for (uint32_t b = 0; b < nb; ++b) {
      const int64_t v = raw[(size_t)k * nb + b];
      if (v >= (1ll << 62) || v <= -(1ll << 62)) overflow = true;
      total[b] += (double)v;
      batch[(size_t)k * nb + b] = nk > 0 ? (double)v * scale / (nk * vol) : 0.0;
    }
  }
  for (uint32_t b = 0; b < nb; ++b) h_flux[b] = N > 0 ? total[b] * scale / ((double)N * vol) : 0.0;
  if (h_batch) std::memcpy(h_batch, batch.data(), slots * sizeof(double));
  if (h_rel_err) {
    for (uint32_t b = 0; b < nb; ++b) {
      if (nbat < 2 || h_flux[b] == 0.0) {
        h_rel_err[b] = 0.0;
        continue;
      }
      double mean = 0.0;
      for (uint32_t k = 0; k < nbat; ++k) mean += batch[(size_t)k * nb + b];
      mean /= nbat;
      double var = 0.0;
      for (uint32_t k = 0; k < nbat; ++k) {
        const double d = batch[(size_t)k * nb + b] - mean;
        var += d * d;
      }
      var /= (nbat - 1);
      h_rel_err[b] = std::sqrt(var / nbat) / std::fabs(h_flux[b]);
    }
  }
  if (overflow) {
    mci::set_error("mc_tally_read: a bin of problem %u reached the int64 headroom 2^62", problem);
    return MC_ERR_OVERFLOW;
  }
  if (cnt[MC_C_DROPPED] != 0) {
    mci::set_error("mc_tally_read: %llu secondaries of problem %u were dropped (full stack)",
                   (unsigned long long)cnt[MC_C_DROPPED], problem);
    return MC_ERR_CAPACITY;
  }
  if (cnt[MC_C_CAPPED] != 0) {
    mci::set_error("mc_tally_read: %llu histories of problem %u hit the event cap",
                   (unsigned long long)cnt[MC_C_CAPPED], problem);
    return MC_ERR_EVENT_CAP;
  }
  return MC_OK;
}

}  // extern "C"
