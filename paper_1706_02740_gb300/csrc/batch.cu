// Batches: the transforms of many plans with one launch per stage.
//
// A batch holds device copies of its plans' records, the per-stage block prefixes (which blocks of
// each launch belong to which signal) and device arrays of the per-execution input and output
// pointers.  Each execution copies the pointers in from a pinned staging ring (so back-to-back
// executions on one stream never overwrite a staging slot the GPU has not read yet) and then runs
// the same stage sequence as a single plan, each stage launched once for the whole batch, either
// directly or as the replay of a CUDA graph captured once.  The launch geometry (sft_tuning) sets
// the block prefixes; the autotuner times candidate geometries on the batch itself.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "alloc_hook.h"
#include "guard.h"
#include "sft_internal.h"
#include "tuning_table.h"

namespace sft {

namespace {
constexpr int kRing = 8;
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

struct Batch {
  std::vector<Plan*> plans;
  int n = 0;
  DevPlan d0;
  LaunchSet ls;
  char* dev = nullptr;
  size_t device_bytes = 0;
  DevPlan* d_plans = nullptr;
  int32_t* d_prefix = nullptr;        // [kStCount][n + 1]
  void** d_ptrs = nullptr;            // [4][n]: f, out_w, out_c, out_n
  void** pinned = nullptr;            // [kRing][4][n]
  cudaEvent_t ring_ev[kRing] = {};
  bool ring_used[kRing] = {};
  int ring_pos = 0;
  Profiler prof;
  int64_t launches = 0;
  // CUDA graph of the stage launches
  bool graph_on = false;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr;         // private capture stream
  int graph_launched = 0;
};

namespace {

// The shape class of a batch whose plans all share one (the tuning table's key).
bool batch_key(const std::vector<Plan*>& ps, TuneKey* k) {
  for (size_t i = 0; i < ps.size(); ++i) {
    const DevPlan& d = ps[i]->d;
    const TuneKey ki = tune_key(d.N, d.s, d.kappa, d.prec);
    if (i == 0) *k = ki;
    else if (!same_key(*k, ki)) return false;
  }
  return !ps.empty();
}

void drop_graph(Batch& B) {
  if (B.gexec) cudaGraphExecDestroy(B.gexec);
  B.gexec = nullptr;
  B.graph_launched = 0;
}

void free_batch(Batch& B) {
  drop_graph(B);
  if (B.cap) cudaStreamDestroy(B.cap);
  B.cap = nullptr;
  profile_release(B.prof);
  for (int i = 0; i < kRing; ++i)
    if (B.ring_ev[i]) cudaEventDestroy(B.ring_ev[i]);
  if (B.pinned) cudaFreeHost(B.pinned);
  if (B.dev) cudaFree(B.dev);
  B.pinned = nullptr;
  B.dev = nullptr;
}

// Block prefixes of every stage under tuning t; false when a launch would exceed 2^31 - 1 blocks.
bool make_prefixes(const std::vector<Plan*>& ps, const sft_tuning& t, std::vector<int32_t>& prefix,
                   int32_t* blocks) {
  const int n = (int)ps.size();
  prefix.assign((size_t)kStCount * (n + 1), 0);
  for (int k = 0; k < kStCount; ++k) {
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      prefix[(size_t)k * (n + 1) + i] = (int32_t)acc;
      acc += signal_blocks(ps[i]->d, k, t);
    }
    if (acc > 0x7fffffff) return false;
    prefix[(size_t)k * (n + 1) + n] = (int32_t)acc;
    blocks[k] = (int32_t)acc;
  }
  return true;
}

// Apply a (validated) tuning: wait for the device, rewrite the prefixes, drop the graph.
sft_status apply_tuning(Batch& B, const sft_tuning& t) {
  std::vector<int32_t> prefix;
  int32_t blocks[kStCount];
  if (!make_prefixes(B.plans, t, prefix, blocks)) {
    set_error("batch too large for this tuning (a launch would exceed 2^31 - 1 blocks)");
    return SFT_EINVAL;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(B.d_prefix, prefix.data(), prefix.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("tuning upload failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  drop_graph(B);
  B.ls.tune = t;
  for (int k = 0; k < kStCount; ++k) B.ls.blocks[k] = blocks[k];
  return SFT_OK;
}

sft_status check_buffers(const Batch& B, const void* const* f_devs, int64_t* const* out_freqs_devs,
                         void* const* out_coefs_devs, int32_t* const* out_count_devs) {
  if (!f_devs || !out_freqs_devs || !out_coefs_devs || !out_count_devs) {
    set_error("batch execution: NULL argument");
    return SFT_EINVAL;
  }
  const size_t align = B.d0.input == SFT_IN_C64 ? 8 : 16;
  for (int i = 0; i < B.n; ++i) {
    if (!f_devs[i] || ((uintptr_t)f_devs[i] % align) || !out_freqs_devs[i] || !out_coefs_devs[i] ||
        !out_count_devs[i]) {
      set_error("batch execution: NULL or misaligned pointer for signal " + std::to_string(i));
      return SFT_EINVAL;
    }
  }
  return SFT_OK;
}

// The plans of a batch: non-NULL, each once, sharing precision, input type, kappa and the
// refinement switch.
sft_status check_plans(const char* who, const sft_plan_t* plans, int32_t n, std::vector<Plan*>& ps) {
  if (!plans || n < 1 || n > (1 << 20)) {
    set_error(std::string(who) + ": need plans and 1 <= n <= 2^20");
    return SFT_EINVAL;
  }
  ps.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) { set_error(std::string(who) + ": NULL plan"); return SFT_EINVAL; }
    ps[i] = sft_plan_internal(plans[i]);
  }
  const DevPlan& a = ps[0]->d;
  for (int i = 0; i < n; ++i) {
    const DevPlan& b = ps[i]->d;
    if (b.prec != a.prec || b.input != a.input || b.kappa != a.kappa || b.refine != a.refine) {
      set_error(std::string(who) + ": plans must share precision, input type, kappa and refine_fp64");
      return SFT_EINVAL;
    }
  }
  std::vector<Plan*> sorted(ps);
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_error(std::string(who) + ": a plan may appear once (its scratch serves one signal)");
    return SFT_EINVAL;
  }
  return SFT_OK;
}

sft_status execute(Batch& B, const void* const* f_devs, int64_t* const* out_freqs_devs,
                   void* const* out_coefs_devs, int32_t* const* out_count_devs, cudaStream_t st) {
  const int n = B.n;
  const int slot = B.ring_pos;
  B.ring_pos = (B.ring_pos + 1) % kRing;
  if (B.ring_used[slot]) cudaEventSynchronize(B.ring_ev[slot]);
  void** stage = B.pinned + (size_t)slot * 4 * n;
  for (int i = 0; i < n; ++i) {
    stage[i] = const_cast<void*>(f_devs[i]);
    stage[n + i] = out_freqs_devs[i];
    stage[2 * n + i] = out_coefs_devs[i];
    stage[3 * n + i] = out_count_devs[i];
  }
  cudaError_t e = cudaMemcpyAsync(B.d_ptrs, stage, 4 * (size_t)n * sizeof(void*),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(B.ring_ev[slot], st);
  B.ring_used[slot] = true;
  if (e != cudaSuccess) {
    set_error(std::string("batch execution: pointer upload failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  BatchView bv;
  memset(&bv, 0, sizeof(bv));
  bv.plans = B.d_plans;
  bv.n = n;
  bv.f = const_cast<const void* const*>(B.d_ptrs);
  bv.out_w = reinterpret_cast<int64_t* const*>(B.d_ptrs + n);
  bv.out_c = reinterpret_cast<double2* const*>(B.d_ptrs + 2 * n);
  bv.out_n = reinterpret_cast<int32_t* const*>(B.d_ptrs + 3 * n);
  if (!B.graph_on) {
    int launched = 0;
    e = run_stages(B.d0, bv, B.ls, st, profile_slot(B.prof), &launched);
    B.launches += launched;
    if (e != cudaSuccess) {
      set_error(std::string("batch execution: launch failed: ") + cudaGetErrorString(e));
      return SFT_ECUDA;
    }
    return SFT_OK;
  }
  if (!B.gexec) {
    // capture on the private stream: the captured launches run only when the graph is launched
    if (!B.cap) e = cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      int launched = 0;
      const cudaError_t e1 = run_stages(B.d0, bv, B.ls, B.cap, nullptr, &launched);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(B.cap, &g);
      e = e1 != cudaSuccess ? e1 : e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&B.gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) B.graph_launched = launched;
      else B.gexec = nullptr;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("batch execution: graph capture failed: ") + cudaGetErrorString(e));
      return SFT_ECUDA;
    }
  }
  e = cudaGraphLaunch(B.gexec, st);
  if (e != cudaSuccess) {
    set_error(std::string("batch execution: graph launch failed: ") + cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  B.launches += B.graph_launched;
  return SFT_OK;
}

}  // namespace

}  // namespace sft

struct sft_batch_s {
  sft::Batch B;
};

extern "C" {

sft_status sft_batch_create(sft_batch_t* out, const sft_plan_t* plans, int32_t n) {
  return sft::guarded("sft_batch_create", [&]() -> sft_status {
    using namespace sft;
    if (!out) {
      set_error("sft_batch_create: out is NULL");
      return SFT_EINVAL;
    }
    *out = nullptr;
    std::vector<Plan*> ps;
    const sft_status chk = check_plans("sft_batch_create", plans, n, ps);
    if (chk != SFT_OK) return chk;
    const DevPlan& a = ps[0]->d;
    sft_batch_s* h = new (std::nothrow) sft_batch_s();
    if (!h) { set_error("host allocation failed"); return SFT_ENOMEM; }
    Batch& B = h->B;
    B.plans = ps;
    B.n = n;
    B.d0 = a;
    B.ls.tune = default_tuning();
    {
      TuneKey key;
      sft_tuning stored;
      if (batch_key(ps, &key) && tuning_table_find(key, &stored)) B.ls.tune = stored;
    }
    B.ls.pmax = 0;
    B.ls.rlmax = 0;
    B.ls.rtpt = 0;
    B.ls.kmax = 0;
    for (int i = 0; i < n; ++i) {
      B.ls.pmax = std::max(B.ls.pmax, ps[i]->d.pmax);
      if (ps[i]->d.rader) B.ls.rlmax = std::max(B.ls.rlmax, ps[i]->d.rLmax);
      if (ps[i]->d.rader) B.ls.rtpt = std::max(B.ls.rtpt, ps[i]->d.rTpt);
      B.ls.kmax = std::max(B.ls.kmax, ps[i]->d.K);
    }
    std::vector<int32_t> prefix;
    if (!make_prefixes(ps, B.ls.tune, prefix, B.ls.blocks)) {
      delete h;
      set_error("sft_batch_create: batch too large (a launch would exceed 2^31 - 1 blocks)");
      return SFT_EINVAL;
    }
    const size_t o_plans = 0;
    const size_t o_prefix = align256(o_plans + sizeof(DevPlan) * (size_t)n);
    const size_t o_ptrs = align256(o_prefix + prefix.size() * sizeof(int32_t));
    const size_t total = align256(o_ptrs + 4 * (size_t)n * sizeof(void*));
    cudaError_t e = dev_malloc((void**)&B.dev, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      set_error(std::string("sft_batch_create: cudaMalloc failed: ") + cudaGetErrorString(e));
      return SFT_ENOMEM;
    }
    B.device_bytes = total;
    std::vector<char> blob(o_ptrs, 0);
    for (int i = 0; i < n; ++i) memcpy(blob.data() + o_plans + sizeof(DevPlan) * i, &ps[i]->d, sizeof(DevPlan));
    memcpy(blob.data() + o_prefix, prefix.data(), prefix.size() * sizeof(int32_t));
    e = cudaMemcpy(B.dev, blob.data(), o_ptrs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = host_alloc((void**)&B.pinned, (size_t)kRing * 4 * n * sizeof(void*));
    for (int i = 0; e == cudaSuccess && i < kRing; ++i)
      e = cudaEventCreateWithFlags(&B.ring_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_batch(B);
      delete h;
      set_error(std::string("sft_batch_create: set-up failed: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
    }
    B.d_plans = reinterpret_cast<DevPlan*>(B.dev + o_plans);
    B.d_prefix = reinterpret_cast<int32_t*>(B.dev + o_prefix);
    B.d_ptrs = reinterpret_cast<void**>(B.dev + o_ptrs);
    for (int k = 0; k < kStCount; ++k) B.ls.blk[k] = B.d_prefix + (size_t)k * (n + 1);
    *out = h;
    return SFT_OK;
  });
}

sft_status sft_batch_execute(sft_batch_t batch, const void* const* f_devs,
                             int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                             int32_t* const* out_count_devs, void* stream) {
  return sft::guarded("sft_batch_execute", [&]() -> sft_status {
    using namespace sft;
    if (!batch) { set_error("sft_batch_execute: batch is NULL"); return SFT_EINVAL; }
    Batch& B = batch->B;
    sft_status s = check_buffers(B, f_devs, out_freqs_devs, out_coefs_devs, out_count_devs);
    if (s != SFT_OK) return s;
    return execute(B, f_devs, out_freqs_devs, out_coefs_devs, out_count_devs, (cudaStream_t)stream);
  });
}

sft_status sft_batch_set_tuning(sft_batch_t batch, const sft_tuning* t) {
  using namespace sft;
  if (!batch || !t) { set_error("sft_batch_set_tuning: NULL argument"); return SFT_EINVAL; }
  std::string why;
  if (!tuning_valid(*t, &why)) { set_error("sft_batch_set_tuning: " + why); return SFT_EINVAL; }
  return apply_tuning(batch->B, *t);
}

sft_status sft_batch_get_tuning(sft_batch_t batch, sft_tuning* t) {
  if (!batch || !t) { sft::set_error("sft_batch_get_tuning: NULL argument"); return SFT_EINVAL; }
  *t = batch->B.ls.tune;
  return SFT_OK;
}

sft_status sft_batch_autotune(sft_batch_t batch, const void* const* f_devs,
                              int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                              int32_t* const* out_count_devs, void* stream, int32_t reps,
                              sft_tuning* chosen) {
  return sft::guarded("sft_batch_autotune", [&]() -> sft_status {
    using namespace sft;
    if (!batch || reps < 1) { set_error("sft_batch_autotune: need a batch and reps >= 1"); return SFT_EINVAL; }
    Batch& B = batch->B;
    sft_status s = check_buffers(B, f_devs, out_freqs_devs, out_coefs_devs, out_count_devs);
    if (s != SFT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const bool prof_was = B.prof.on, graph_was = B.graph_on;
    B.graph_on = false;
    drop_graph(B);
    s = profile_enable(B.prof, 1);
    if (s != SFT_OK) return s;

    // Mean milliseconds per execution of the stages s0..s1 under tuning t.
    auto measure = [&](const sft_tuning& t, int s0, int s1, double* ms) -> sft_status {
      sft_status r = apply_tuning(B, t);
      double stage[kStages];
      int32_t cnt = 0;
      for (int pass = 0; pass < 2 && r == SFT_OK; ++pass) {
        const int runs = pass == 0 ? 1 : reps;
        for (int i = 0; i < runs && r == SFT_OK; ++i)
          r = execute(B, f_devs, out_freqs_devs, out_coefs_devs, out_count_devs, st);
        if (r != SFT_OK) break;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
          set_error("sft_batch_autotune: execution failed");
          r = SFT_ECUDA;
          break;
        }
        r = profile_read(B.prof, stage, &cnt);
      }
      if (r == SFT_OK) {
        double sum = 0;
        for (int k = s0; k <= s1; ++k) sum += stage[k];
        *ms = sum / (cnt > 0 ? cnt : 1);
      }
      return r;
    };
    // Keep the fastest of best and the candidates for stages s0..s1.
    auto try_knob = [&](sft_tuning& best, const std::vector<sft_tuning>& cands, int s0,
                        int s1) -> sft_status {
      double best_ms = 0;
      sft_status r = measure(best, s0, s1, &best_ms);
      for (size_t i = 0; i < cands.size() && r == SFT_OK; ++i) {
        std::string why;
        if (!tuning_valid(cands[i], &why)) continue;
        double ms = 0;
        r = measure(cands[i], s0, s1, &ms);
        if (r == SFT_OK && ms < best_ms) {
          best_ms = ms;
          best = cands[i];
        }
      }
      return r;
    };

    sft_tuning best = B.ls.tune;
    std::vector<sft_tuning> cands;
    // resampling: CTA size and register cap (kappa 4 and 6 only)
    if (B.d0.kappa == 4 || B.d0.kappa == 6) {
      for (int th : {128, 256, 512})
        for (int cap : {0, 1}) {
          sft_tuning t = best;
          t.resample_threads = th;
          t.resample_regcap = cap;
          cands.push_back(t);
        }
      s = try_knob(best, cands, 0, 0);
    }
    // chirp convolution: transforms per CTA of every length class present, then the FP32 8192 build
    // (one or two CTAs per SM)
    for (int c = 0; c < 9 && s == SFT_OK; ++c) {
      // the lengths with as many threads per transform as 2^(c+6) (2^k and r 2^k share an entry)
      bool present = false;
      for (int k = kStBluestein0; k < kStCount; ++k)
        present |= B.ls.blocks[k] > 0 && fft_tune_class(fft_stage_length(k)) == c;
      if (!present) continue;
      const int M = 64 << c, hi = M >= 4096 ? 1 : 4096 / M;
      if (hi == 1) continue;
      cands.clear();
      for (int g = 1; g <= hi; g *= 2) {
        sft_tuning t = best;
        t.dft_per_cta[c] = g;
        cands.push_back(t);
      }
      s = try_knob(best, cands, 1, 1);
    }
    if (s == SFT_OK && B.d0.prec == SFT_FP32 && B.ls.blocks[kStBluestein0 + 7] > 0) {
      cands.clear();
      sft_tuning t = best;
      t.dft_two_ctas = 1 - best.dft_two_ctas;
      cands.push_back(t);
      s = try_knob(best, cands, 1, 1);
    }
    // residues, CRT and vote: bins per CTA
    if (s == SFT_OK) {
      cands.clear();
      for (int th : {128, 256, 512}) {
        sft_tuning t = best;
        t.bin_threads = th;
        cands.push_back(t);
      }
      s = try_knob(best, cands, 2, 3);
    }
    const sft_status s2 = apply_tuning(B, best);
    if (s == SFT_OK) s = s2;
    TuneKey key;
    if (s == SFT_OK && batch_key(B.plans, &key)) tuning_table_store(key, best);
    profile_enable(B.prof, prof_was ? 1 : 0);
    B.graph_on = graph_was;
    if (s == SFT_OK && chosen) *chosen = best;
    return s;
  });
}

sft_status sft_batch_graph(sft_batch_t batch, int32_t enable) {
  if (!batch) { sft::set_error("sft_batch_graph: batch is NULL"); return SFT_EINVAL; }
  sft::Batch& B = batch->B;
  B.graph_on = enable != 0;
  if (!B.graph_on) sft::drop_graph(B);
  return SFT_OK;
}

sft_status sft_batch_destroy(sft_batch_t batch) {
  if (!batch) return SFT_OK;
  sft::free_batch(batch->B);
  delete batch;
  return SFT_OK;
}

sft_status sft_execute_batch(const sft_plan_t* plans, const void* const* f_devs,
                             int64_t* const* out_freqs_devs, void* const* out_coefs_devs,
                             int32_t* const* out_count_devs, int32_t n, void* stream) {
  return sft::guarded("sft_execute_batch", [&]() -> sft_status {
    using namespace sft;
    std::vector<Plan*> ps;
    sft_status s = check_plans("sft_execute_batch", plans, n, ps);
    if (s != SFT_OK) return s;
    if (!f_devs || !out_freqs_devs || !out_coefs_devs || !out_count_devs) {
      set_error("sft_execute_batch: NULL argument");
      return SFT_EINVAL;
    }
    const DevPlan& d0 = ps[0]->d;
    const size_t align = d0.input == SFT_IN_C64 ? 8 : 16;
    for (int i = 0; i < n; ++i) {
      if (!f_devs[i] || ((uintptr_t)f_devs[i] % align) || !out_freqs_devs[i] || !out_coefs_devs[i] ||
          !out_count_devs[i]) {
        set_error("sft_execute_batch: NULL or misaligned pointer for signal " + std::to_string(i));
        return SFT_EINVAL;
      }
    }
    LaunchSet ls;
    memset(&ls, 0, sizeof(ls));
    ls.tune = default_tuning();
    for (int i = 0; i < n; ++i) {
      ls.pmax = std::max(ls.pmax, ps[i]->d.pmax);
      if (ps[i]->d.rader) ls.rlmax = std::max(ls.rlmax, ps[i]->d.rLmax);
      if (ps[i]->d.rader) ls.rtpt = std::max(ls.rtpt, ps[i]->d.rTpt);
      ls.kmax = std::max(ls.kmax, ps[i]->d.K);
    }
    std::vector<int32_t> prefix;
    if (!make_prefixes(ps, ls.tune, prefix, ls.blocks)) {
      set_error("sft_execute_batch: batch too large (a launch would exceed 2^31 - 1 blocks)");
      return SFT_EINVAL;
    }
    // one device array: records | block prefixes | pointer tables, filled from one host image by a
    // stream-ordered copy (pageable source: staged before the copy call returns)
    const size_t o_prefix = align256(sizeof(DevPlan) * (size_t)n);
    const size_t o_ptrs = align256(o_prefix + prefix.size() * sizeof(int32_t));
    const size_t total = o_ptrs + 4 * (size_t)n * sizeof(void*);
    std::vector<char> blob(total, 0);
    for (int i = 0; i < n; ++i) memcpy(blob.data() + sizeof(DevPlan) * i, &ps[i]->d, sizeof(DevPlan));
    memcpy(blob.data() + o_prefix, prefix.data(), prefix.size() * sizeof(int32_t));
    void** hp = reinterpret_cast<void**>(blob.data() + o_ptrs);
    for (int i = 0; i < n; ++i) {
      hp[i] = const_cast<void*>(f_devs[i]);
      hp[n + i] = out_freqs_devs[i];
      hp[2 * n + i] = out_coefs_devs[i];
      hp[3 * n + i] = out_count_devs[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* dev = nullptr;
    cudaError_t e = dev_malloc_async((void**)&dev, total, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("sft_execute_batch: cudaMallocAsync failed: ") + cudaGetErrorString(e));
      return SFT_ENOMEM;
    }
    e = cudaMemcpyAsync(dev, blob.data(), total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      for (int k = 0; k < kStCount; ++k)
        ls.blk[k] = reinterpret_cast<int32_t*>(dev + o_prefix) + (size_t)k * (n + 1);
      void** dp = reinterpret_cast<void**>(dev + o_ptrs);
      BatchView bv;
      memset(&bv, 0, sizeof(bv));
      bv.plans = reinterpret_cast<DevPlan*>(dev);
      bv.n = n;
      bv.f = const_cast<const void* const*>(dp);
      bv.out_w = reinterpret_cast<int64_t* const*>(dp + n);
      bv.out_c = reinterpret_cast<double2* const*>(dp + 2 * n);
      bv.out_n = reinterpret_cast<int32_t* const*>(dp + 3 * n);
      int launched = 0;
      e = run_stages(d0, bv, ls, st, nullptr, &launched);
    }
    const cudaError_t ef = cudaFreeAsync(dev, st);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) {
      set_error(std::string("sft_execute_batch: ") + cudaGetErrorString(e));
      return SFT_ECUDA;
    }
    return SFT_OK;
  });
}

sft_status sft_batch_profile(sft_batch_t batch, int32_t enable) {
  if (!batch) { sft::set_error("batch is NULL"); return SFT_EINVAL; }
  return sft::profile_enable(batch->B.prof, enable);
}

sft_status sft_batch_profile_read(sft_batch_t batch, double* stage_ms, int32_t* n_executions) {
  if (!batch || !stage_ms || !n_executions) { sft::set_error("NULL argument"); return SFT_EINVAL; }
  return sft::profile_read(batch->B.prof, stage_ms, n_executions);
}

int64_t sft_batch_launches(sft_batch_t batch) { return batch ? batch->B.launches : 0; }

size_t sft_batch_device_bytes(sft_batch_t batch) { return batch ? batch->B.device_bytes : 0; }

}  // extern "C"
