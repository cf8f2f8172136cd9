// Continuous batching of design iterations: one phase of the design loop of
// several jobs (contexts of any sizes and precisions) runs as one CUDA graph
// launch.  Each job's kernels form one branch of the graph, captured from
// the job's own stream with its own buffers and in its own order, so a job
// computes bitwise what it computes alone; the branches run concurrently on
// the device and the host issues one launch per phase instead of one per
// kernel per job.  Graphs are cached per job table and replayed while the
// table (jobs, buffers, and the alternation of each job's two modulus
// buffers, which both phases read) repeats, which it does every other
// iteration of a steady set of jobs.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"

namespace {

using namespace topo;

struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<const to_ctx*> ctxs;
  std::vector<long long> launches;   // kernels per job branch
  unsigned long long last_use = 0;
};

constexpr size_t MAX_GRAPHS = 64;
std::mutex g_mu;
std::map<std::vector<uintptr_t>, BatchGraph> g_graphs;
unsigned long long g_clock = 0;

uintptr_t bits(double v) {
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (uintptr_t)u;
}

to_status err(const std::string& msg, to_status st = TO_E_INVALID) {
  set_global_error(msg);
  return st;
}

// the host-side state change of to_set_density without its launches (the
// modulus buffers alternate; the hierarchy must be rebuilt)
void density_state(to_ctx* c) {
  if (c->have_density) std::swap(c->E64, c->Eprev64);
  c->have_density = true;
  c->hier_stale = true;
}

// one job's work of a phase, enqueued on its context stream
to_status enqueue_phase(const to_batch_job& j, int phase) {
  to_ctx* c = j.ctx;
  if (phase == TO_PHASE_DENSITY) {
    to_status st = to_filter(c, TO_FILTER_DENSITY, j.rho, j.rho_phys);
    if (st != TO_OK) return st;
    return to_set_density(c, j.rho_phys);
  }
  to_status st = to_sensitivity(c, j.u, j.compliance_dev, j.dc);
  if (st != TO_OK) return st;
  if ((st = to_filter(c, TO_FILTER_SENS, j.dc, j.dc_f)) != TO_OK) return st;
  return oc_update_enqueue(c, j.volfrac, j.move, j.dc_f, j.dv_f, j.rho, j.change_dev);
}

void evict_oldest_locked() {
  auto old = g_graphs.begin();
  for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it)
    if (it->second.last_use < old->second.last_use) old = it;
  cudaGraphExecDestroy(old->second.exec);
  g_graphs.erase(old);
}

}  // namespace

void batch_forget(const to_ctx* c) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    const auto& v = it->second.ctxs;
    if (std::find(v.begin(), v.end(), c) != v.end()) {
      cudaGraphExecDestroy(it->second.exec);
      it = g_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

extern "C" to_status to_batch_step(const to_batch_job* jobs, int32_t n, int32_t phase,
                                   void* stream) {
  if (!jobs || n < 1 || n > TO_BATCH_MAX_JOBS) return err("n must be in [1, TO_BATCH_MAX_JOBS]");
  if (phase != TO_PHASE_DENSITY && phase != TO_PHASE_UPDATE) return err("bad phase");
  std::vector<const to_ctx*> seen;
  for (int i = 0; i < n; ++i) {
    const to_batch_job& j = jobs[i];
    if (!j.ctx || !j.rho) return err("NULL context or design field");
    if (phase == TO_PHASE_DENSITY && !j.rho_phys) return err("NULL rho_phys");
    if (phase == TO_PHASE_UPDATE &&
        (!j.u || !j.dc || !j.dc_f || !j.dv_f || !j.compliance_dev || !j.ctx->have_density))
      return err("NULL argument, or a context without a density");
    if (phase == TO_PHASE_UPDATE &&
        !(j.volfrac > 0.0 && j.volfrac <= 1.0 && j.move > 0.0 && j.move <= 1.0))
      return err("bad volfrac/move");
    if (std::find(seen.begin(), seen.end(), j.ctx) != seen.end())
      return err("a context appears twice in the batch");
    seen.push_back(j.ctx);
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the job table (and, for the density phase, which modulus buffer each
  // job writes next) identifies the graph
  std::vector<uintptr_t> key{(uintptr_t)phase, (uintptr_t)n, (uintptr_t)s};
  for (int i = 0; i < n; ++i) {
    const to_batch_job& j = jobs[i];
    for (uintptr_t v : {(uintptr_t)j.ctx, (uintptr_t)j.rho, (uintptr_t)j.rho_phys, (uintptr_t)j.u,
                        (uintptr_t)j.dc, (uintptr_t)j.dc_f, (uintptr_t)j.dv_f,
                        (uintptr_t)j.compliance_dev, (uintptr_t)j.change_dev, bits(j.volfrac),
                        bits(j.move)})
      key.push_back(v);
    // the captured kernels address the context's modulus buffers, which
    // trade places at every density update: both phases depend on them
    key.push_back((uintptr_t)j.ctx->E64);
    key.push_back((uintptr_t)j.ctx->Eprev64);
    key.push_back((uintptr_t)j.ctx->have_density);
  }
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_graphs.find(key);
  if (it == g_graphs.end()) {
    // capture: fork every job's stream from s, enqueue its work there, join
    BatchGraph bg;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins(n, nullptr);
    std::vector<unsigned> keep_prof(n);
    std::vector<long long> keep_launches(n);
    // host state the density phase changes while it is captured; restored
    // afterwards, so that every launch (fresh or cached) applies it once
    struct HostState {
      double *E64, *Eprev64;
      bool have_density, hier_stale;
    };
    std::vector<HostState> keep_state(n);
    for (int i = 0; i < n; ++i) {
      const to_ctx* c = jobs[i].ctx;
      keep_state[i] = {c->E64, c->Eprev64, c->have_density, c->hier_stale};
    }
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (fork) cudaEventDestroy(fork);
      for (auto ev : joins)
        if (ev) cudaEventDestroy(ev);
      return err(std::string("batch events: ") + cudaGetErrorString(e), TO_E_CUDA);
    }
    to_status st = TO_OK;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, s);
    int started = 0;
    for (int i = 0; i < n && e == cudaSuccess && st == TO_OK; ++i) {
      to_ctx* c = jobs[i].ctx;
      keep_prof[i] = c->prof_mask;
      keep_launches[i] = c->launches;
      c->prof_mask = 0u;   // no profiling events inside the graph
      ++started;
      if (c->stream != s) e = cudaStreamWaitEvent(c->stream, fork, 0);
      if (e == cudaSuccess) st = enqueue_phase(jobs[i], phase);
      if (e == cudaSuccess && st == TO_OK && c->stream != s) {
        e = cudaEventRecord(joins[i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, joins[i], 0);
      }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = e2;
    for (int i = 0; i < started; ++i) {
      to_ctx* c = jobs[i].ctx;
      c->prof_mask = keep_prof[i];
      bg.launches.push_back(c->launches - keep_launches[i]);
      c->launches = keep_launches[i];
      c->E64 = keep_state[i].E64;
      c->Eprev64 = keep_state[i].Eprev64;
      c->have_density = keep_state[i].have_density;
      c->hier_stale = keep_state[i].hier_stale;
    }
    cudaEventDestroy(fork);
    for (auto ev : joins) cudaEventDestroy(ev);
    if (e == cudaSuccess && st == TO_OK) e = cudaGraphInstantiate(&bg.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != TO_OK) return st;   // nothing ran: a capture executes no kernel
    if (e != cudaSuccess) return err(std::string("batch graph: ") + cudaGetErrorString(e), TO_E_CUDA);
    bg.ctxs.assign(seen.begin(), seen.end());
    if (g_graphs.size() >= MAX_GRAPHS) evict_oldest_locked();
    it = g_graphs.emplace(key, std::move(bg)).first;
  }
  it->second.last_use = ++g_clock;
  const cudaError_t e = cudaGraphLaunch(it->second.exec, s);
  if (e != cudaSuccess) return err(std::string("batch launch: ") + cudaGetErrorString(e), TO_E_CUDA);
  for (int i = 0; i < n; ++i) {
    to_ctx* c = jobs[i].ctx;
    c->launches += it->second.launches[i];
    if (phase == TO_PHASE_DENSITY) density_state(c);
  }
  return TO_OK;
}
