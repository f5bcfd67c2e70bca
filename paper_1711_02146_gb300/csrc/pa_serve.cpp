// pa_serve.cpp — many population annealing runs on one GPU: a batch that
// advances a fixed set of runs together, and a continuous-batching server that
// admits submitted runs while device memory allows.
//
// Each run lives on its own non-blocking stream, so the kernels of different
// runs overlap on the device while the host issues their steps round-robin
// (pa_step of an explicit schedule does not wait for the device); a server run's
// stream priority is set by its work, smaller runs higher.  Memory is
// stream-ordered (per run one allocation from the runs' memory pool in pa_create
// and one cudaFreeAsync in pa_destroy), so admitting or retiring a run never
// synchronises the other runs.  Results of a run depend only on its
// configuration, never on what else is running.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.h"

namespace {

// Deep copy of a configuration (the schedule arrays are owned).
struct OwnedConfig {
  pa_config cfg{};
  std::vector<double> betas;
  std::vector<int32_t> sweeps;
  void set(const pa_config& c) {
    cfg = c;
    if (c.betas) {
      betas.assign(c.betas, c.betas + c.n_temps);
      cfg.betas = betas.data();
    }
    if (c.sweeps_per_step) {
      sweeps.assign(c.sweeps_per_step, c.sweeps_per_step + c.n_temps);
      cfg.sweeps_per_step = sweeps.data();
    }
  }
  OwnedConfig() = default;
  OwnedConfig(const OwnedConfig& o) { set(o.cfg); }
  OwnedConfig& operator=(const OwnedConfig& o) {
    if (this != &o) set(o.cfg);
    return *this;
  }
};

int make_stream(cudaStream_t* s, int priority) {
  return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, priority) == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

// Metropolis updates a run will do (its schedule's sweeps times N R per population;
// an adaptive schedule counts its step limit).
double run_work(const pa_config& c) {
  double sweeps = 0.0;
  for (int t = 1; t < c.n_temps; ++t) sweeps += c.sweeps_per_step ? (double)c.sweeps_per_step[t] : (double)c.n_sweeps;
  return sweeps * (double)c.L * c.L * c.L * (double)c.R * (double)c.n_pop;
}

// The device's stream priorities: least (numerically largest) and greatest.
void priority_range(int* least, int* greatest) {
  *least = 0;
  *greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(least, greatest) != cudaSuccess) {
    cudaGetLastError();
    *least = *greatest = 0;
  }
}

// Server requests: the smaller the run, the higher its stream's priority, one level
// per decade of work (shortest job first, so short requests are not held up behind
// long ones); runs of 1e12 updates and more share the least priority.
int server_priority_level(const pa_config& c, int n_levels) {
  const double w = run_work(c);
  int decade = w < 1.0 ? 0 : (int)std::floor(std::log10(w));
  int level = 12 - decade;  // 0: least priority
  return std::max(0, std::min(n_levels - 1, level));
}

}  // namespace

struct pa_batch {
  std::vector<pa_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  int32_t mode = PA_BATCH_FUSED;
  int64_t kernel_launches = 0, graph_launches = 0;
};

struct pa_server {
  struct Request {
    uint64_t id;
    OwnedConfig cfg;
    size_t footprint;
  };
  struct Active {
    uint64_t id;
    pa_ctx* ctx;
    cudaStream_t stream;
    size_t footprint;
    cudaEvent_t done;
    bool all_issued;
    int n_pop;
    int model;
    int level;  // stream priority level
  };
  struct Finished {
    std::vector<pa_obs> obs;    // per population, last step (+-1 couplings)
    std::vector<pa_gobs> gobs;  // per population, last step (Gaussian couplings)
    int32_t last_step;
    int status;
  };
  size_t budget = 0, used = 0;
  int32_t max_active = 0, steps_per_poll = 1;
  uint64_t next_id = 1;
  std::deque<Request> queue;
  std::vector<Active> active;
  std::vector<std::vector<cudaStream_t>> free_streams;  // per priority level, 0 = least
  int least_priority = 0, n_levels = 1;
  std::vector<cudaEvent_t> free_events;
  std::map<uint64_t, Finished> finished;
};

extern "C" {

// ---------------------------------------------------------------- batch

int pa_batch_create(const pa_config* cfgs, int32_t n, pa_batch** out) try {
  if (!out || !cfgs || n < 1) return PA_ERR_INVALID;
  *out = nullptr;
  pa_batch* b = new (std::nothrow) pa_batch();
  if (!b) return PA_ERR_NOMEM;
  for (int32_t i = 0; i < n; ++i) {
    cudaStream_t s = nullptr;
    int rc = make_stream(&s, 0);  // default priority (largest-first priorities measured 2 % slower)
    pa_ctx* c = nullptr;
    if (rc == PA_OK) rc = pa::create_run(&cfgs[i], s, &c, false);
    if (rc == PA_OK) pa::use_chosen_shape(c);
    if (rc != PA_OK) {
      if (s) cudaStreamDestroy(s);
      pa_batch_destroy(b);
      return rc;
    }
    b->ctx.push_back(c);
    b->streams.push_back(s);
  }
  *out = b;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_batch_run(pa_batch* b) try {
  if (!b) return PA_ERR_INVALID;
  // fused mode: the runs that qualify advance by rounds of one graph launch each
  // (issued at once, asynchronously); the others step on their own streams meanwhile
  std::vector<pa_ctx*> fused;
  std::vector<char> live(b->ctx.size(), 1);
  if (b->mode == PA_BATCH_FUSED)
    for (size_t i = 0; i < b->ctx.size(); ++i)
      if (pa::group_eligible(b->ctx[i])) {
        fused.push_back(b->ctx[i]);
        live[i] = 0;
      }
  pa::Group* grp = nullptr;
  if (!fused.empty()) {
    int rc = pa::group_create(fused.data(), (int)fused.size(), &grp);
    if (rc == PA_OK) rc = pa::group_run(grp, &b->kernel_launches, &b->graph_launches);
    if (rc != PA_OK) {
      pa::group_destroy(grp);
      return rc;
    }
  }
  size_t n_live = 0;
  for (char l : live) n_live += l ? 1 : 0;
  std::vector<int64_t> before(b->ctx.size(), 0);
  for (size_t i = 0; i < b->ctx.size(); ++i) before[i] = pa::run_kernel_launches(b->ctx[i]);
  int rc = PA_OK;  // a run that fails stops; the others finish (the first error is returned)
  while (n_live > 0) {
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      if (!live[i]) continue;
      const int r = pa_step(b->ctx[i]);
      if (r != PA_OK) {
        live[i] = 0;
        --n_live;
        if (r != PA_DONE && rc == PA_OK) rc = r;
      }
    }
  }
  for (pa_ctx* c : b->ctx) {
    const int r = pa_sync(c);
    if (rc == PA_OK && r != PA_OK) rc = r;
  }
  for (size_t i = 0; i < b->ctx.size(); ++i) b->kernel_launches += pa::run_kernel_launches(b->ctx[i]) - before[i];
  pa::group_destroy(grp);
  return rc;
} catch (...) {
  return pa::exception_status();
}

int pa_batch_set_mode(pa_batch* b, int32_t mode) try {
  if (!b || (mode != PA_BATCH_FUSED && mode != PA_BATCH_STREAMS)) return PA_ERR_INVALID;
  b->mode = mode;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_batch_launches(const pa_batch* b, int64_t* kernel_launches, int64_t* graph_launches) try {
  if (!b || !kernel_launches || !graph_launches) return PA_ERR_INVALID;
  *kernel_launches = b->kernel_launches;
  *graph_launches = b->graph_launches;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_batch_ctx(pa_batch* b, int32_t i, pa_ctx** view) try {
  if (!b || !view || i < 0 || (size_t)i >= b->ctx.size()) return PA_ERR_INVALID;
  *view = b->ctx[(size_t)i];
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_batch_destroy(pa_batch* b) try {
  if (!b) return PA_ERR_INVALID;
  for (pa_ctx* c : b->ctx) pa_destroy(c);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete b;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

// ---------------------------------------------------------------- server

int pa_server_create(size_t mem_budget, int32_t max_active, int32_t steps_per_poll, pa_server** out) try {
  if (!out || mem_budget == 0 || max_active < 1 || steps_per_poll < 1) return PA_ERR_INVALID;
  pa_server* s = new (std::nothrow) pa_server();
  if (!s) return PA_ERR_NOMEM;
  s->budget = mem_budget;
  s->max_active = max_active;
  s->steps_per_poll = steps_per_poll;
  int least = 0, greatest = 0;
  priority_range(&least, &greatest);
  s->least_priority = least;
  s->n_levels = least - greatest + 1;
  s->free_streams.resize((size_t)s->n_levels);
  *out = s;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_server_submit(pa_server* s, const pa_config* cfg, uint64_t* id) try {
  if (!s || !cfg || !id) return PA_ERR_INVALID;
  size_t fp = 0;
  int rc = pa_footprint(cfg, &fp);
  if (rc != PA_OK) return rc;
  if (fp > s->budget) return PA_ERR_NOMEM;  // could never be admitted
  pa_server::Request r;
  r.id = s->next_id++;
  r.cfg.set(*cfg);
  r.footprint = fp;
  s->queue.push_back(std::move(r));
  *id = s->queue.back().id;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

namespace {

int admit(pa_server* s) {
  while (!s->queue.empty() && (int32_t)s->active.size() < s->max_active &&
         s->used + s->queue.front().footprint <= s->budget) {
    pa_server::Request& r = s->queue.front();
    const int level = server_priority_level(r.cfg.cfg, s->n_levels);
    std::vector<cudaStream_t>& pool = s->free_streams[(size_t)level];
    cudaStream_t st = nullptr;
    if (!pool.empty()) {
      st = pool.back();
      pool.pop_back();
    } else if (make_stream(&st, s->least_priority - level) != PA_OK) {
      return PA_ERR_CUDA;
    }
    cudaEvent_t ev = nullptr;
    if (!s->free_events.empty()) {
      ev = s->free_events.back();
      s->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      pool.push_back(st);
      return PA_ERR_CUDA;
    }
    pa_ctx* c = nullptr;
    const int rc = pa::create_run(&r.cfg.cfg, st, &c, false);
    if (rc == PA_OK) pa::use_chosen_shape(c);
    if (rc != PA_OK) {
      // the request fails on its own; the server keeps serving the others
      pa_server::Finished f;
      f.last_step = -1;
      f.status = rc;
      s->finished[r.id] = f;
      pool.push_back(st);
      s->free_events.push_back(ev);
      s->queue.pop_front();
      continue;
    }
    s->active.push_back({r.id, c, st, r.footprint, ev, false, r.cfg.cfg.n_pop, r.cfg.cfg.model, level});
    s->used += r.footprint;
    s->queue.pop_front();
  }
  return PA_OK;
}

}  // namespace

int pa_server_poll(pa_server* s, uint64_t* done_ids, int32_t cap, int32_t* n_done) try {
  if (!s || !n_done || cap < 0 || (cap > 0 && !done_ids)) return PA_ERR_INVALID;
  *n_done = 0;
  int rc = admit(s);
  if (rc != PA_OK) return rc;
  // issue steps
  for (auto& a : s->active) {
    if (a.all_issued) continue;
    for (int k = 0; k < s->steps_per_poll; ++k) {
      const int st = pa_step(a.ctx);
      if (st == PA_OK) continue;
      a.all_issued = true;  // PA_DONE, or an error recorded in the run
      cudaEventRecord(a.done, a.stream);
      break;
    }
  }
  // retire runs whose last step has completed on the device
  for (size_t i = 0; i < s->active.size();) {
    pa_server::Active& a = s->active[i];
    if (!a.all_issued || cudaEventQuery(a.done) != cudaSuccess || *n_done >= cap) {
      ++i;
      continue;
    }
    pa_server::Finished f;
    f.last_step = pa_current_step(a.ctx);
    f.status = pa_sync(a.ctx);
    if (a.model == PA_MODEL_GAUSS) {
      f.gobs.resize((size_t)a.n_pop);
      for (int p = 0; p < a.n_pop && f.status == PA_OK; ++p)
        f.status = pa_gobservables(a.ctx, f.last_step, p, &f.gobs[(size_t)p]);
    } else {
      f.obs.resize((size_t)a.n_pop);
      for (int p = 0; p < a.n_pop && f.status == PA_OK; ++p)
        f.status = pa_observables(a.ctx, f.last_step, p, &f.obs[(size_t)p]);
    }
    s->finished[a.id] = std::move(f);
    pa_destroy(a.ctx);
    // the run's work is done, so this waits only for its memory's release, after
    // which any stream may reuse that memory
    cudaStreamSynchronize(a.stream);
    s->free_streams[(size_t)a.level].push_back(a.stream);
    s->free_events.push_back(a.done);
    s->used -= a.footprint;
    done_ids[(*n_done)++] = a.id;
    s->active.erase(s->active.begin() + (long)i);
  }
  return admit(s);
} catch (...) {
  return pa::exception_status();
}

int pa_server_result(pa_server* s, uint64_t id, int32_t pop, pa_obs* out, int32_t* last_step) try {
  if (!s || !out) return PA_ERR_INVALID;
  auto it = s->finished.find(id);
  if (it == s->finished.end()) return PA_ERR_STATE;
  if (it->second.status != PA_OK) return it->second.status;
  if (pop < 0 || (size_t)pop >= it->second.obs.size()) return PA_ERR_INVALID;  // also: a Gaussian request
  *out = it->second.obs[(size_t)pop];
  if (last_step) *last_step = it->second.last_step;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_server_gresult(pa_server* s, uint64_t id, int32_t pop, pa_gobs* out, int32_t* last_step) try {
  if (!s || !out) return PA_ERR_INVALID;
  auto it = s->finished.find(id);
  if (it == s->finished.end()) return PA_ERR_STATE;
  if (it->second.status != PA_OK) return it->second.status;
  if (pop < 0 || (size_t)pop >= it->second.gobs.size()) return PA_ERR_INVALID;  // also: a +-1 request
  *out = it->second.gobs[(size_t)pop];
  if (last_step) *last_step = it->second.last_step;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_server_load(pa_server* s, int32_t* queued, int32_t* active) try {
  if (!s) return PA_ERR_INVALID;
  if (queued) *queued = (int32_t)s->queue.size();
  if (active) *active = (int32_t)s->active.size();
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

int pa_server_destroy(pa_server* s) try {
  if (!s) return PA_ERR_INVALID;
  for (auto& a : s->active) {
    pa_destroy(a.ctx);
    s->free_streams[(size_t)a.level].push_back(a.stream);
    s->free_events.push_back(a.done);
  }
  for (auto& pool : s->free_streams)
    for (cudaStream_t st : pool) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t ev : s->free_events) cudaEventDestroy(ev);
  delete s;
  return PA_OK;
} catch (...) {
  return pa::exception_status();
}

}  // extern "C"
