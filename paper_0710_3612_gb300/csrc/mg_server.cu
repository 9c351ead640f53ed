// Serving engine: solve requests over several gauge configurations with
// continuous batching and HBM-budget admission of resident set-ups (the
// contract is in include/mg_server.h).  Host code over the solver's C ABI;
// every arithmetic step runs in the solver's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mg.h"
#include "../../include/mg_server.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  int cfg = 0;
  double mass = 0.0, tol = 0.0;
  int solver = 0, nrhs = 0;
  const void* b = nullptr;
  void* x = nullptr;
  Clock::time_point t_submit;
  bool done = false;
  mg_status st = MG_OK;
  std::vector<mg_solve_info> info;
  double latency_ms = 0.0;
};

struct Config {
  int id = 0;
  mg_params p{};
  double setup_mass = 0.0;
  int Lx = 0, Lt = 0;
  void* gauge = nullptr;         // device copies owned by the server
  void* noise = nullptr;
  long long need = 0;            // peak bytes of a set-up + the batch buffers
  long long resident = 0;        // bytes while resident
  mg_handle* h = nullptr;
  double cur_mass = 0.0;
  cudaStream_t stream = nullptr;
  void* bbuf = nullptr;          // batch staging, [max_rhs][Lt][Lx][2] complex128 each
  void* xbuf = nullptr;
  std::deque<Request*> queue;
  bool busy = false;             // held by a worker
  long long last_used = 0;
};

}  // namespace

struct mg_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::unique_ptr<Config>> cfgs;
  std::unordered_map<long long, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> workers;
  long long budget = 0, resident = 0, peak_resident = 0;
  int max_rhs = 1, device = 0;
  bool stop = false;
  long long next_id = 1, tick = 0;
  long long submitted = 0, completed = 0, failed = 0, batches = 0, batched_rhs = 0;
  long long builds = 0, evictions = 0, remasses = 0;
  std::vector<double> latencies;
};

namespace {

// Releases a configuration's hierarchy and batch buffers (the caller holds
// the lock and the configuration is idle).
void evict(mg_server* s, Config* c) {
  mg_destroy(c->h);
  c->h = nullptr;
  cudaFree(c->bbuf);
  cudaFree(c->xbuf);
  c->bbuf = c->xbuf = nullptr;
  s->resident -= c->resident;
  c->resident = 0;
  ++s->evictions;
}

// Chooses the next configuration to run (the lock is held; never waits):
// candidates are the configurations no worker holds that have pending
// requests, oldest pending request first.  A resident candidate runs; one
// larger than the whole budget is returned to fail its requests; otherwise a
// candidate runs if idle hierarchies (no pending request, not held) can be
// evicted, least recently used first, to fit its set-up -- then *build is set
// and its peak is reserved.  nullptr if nothing can run now.
Config* choose(mg_server* s, bool* build) {
  *build = false;
  std::vector<Config*> cand;
  for (auto& c : s->cfgs)
    if (!c->busy && !c->queue.empty()) cand.push_back(c.get());
  std::sort(cand.begin(), cand.end(),
            [](const Config* a, const Config* b) { return a->queue.front()->id < b->queue.front()->id; });
  for (Config* c : cand) {
    if (c->h || c->need > s->budget) return c;
    std::vector<Config*> idle;
    long long freeable = 0;
    for (auto& o : s->cfgs)
      if (o->h && !o->busy && o->queue.empty()) {
        idle.push_back(o.get());
        freeable += o->resident;
      }
    if (s->resident - freeable + c->need > s->budget) continue;
    std::sort(idle.begin(), idle.end(),
              [](const Config* a, const Config* b) { return a->last_used < b->last_used; });
    for (Config* o : idle) {
      if (s->resident + c->need <= s->budget) break;
      evict(s, o);
    }
    s->resident += c->need;                   // reserve the set-up's peak
    s->peak_resident = std::max(s->peak_resident, s->resident);
    *build = true;
    return c;
  }
  return nullptr;
}

void finish(mg_server* s, std::vector<Request*>& batch, mg_status st,
            const std::vector<mg_solve_info>* infos) {
  const auto now = Clock::now();
  size_t k = 0;
  for (Request* r : batch) {
    r->st = st;
    if (infos) r->info.assign(infos->begin() + k, infos->begin() + k + r->nrhs);
    k += r->nrhs;
    r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    r->done = true;
    if (st == MG_OK || st == MG_ERR_NOCONV) {
      ++s->completed;
      s->latencies.push_back(r->latency_ms);
    } else {
      ++s->failed;
    }
  }
}

void worker_main(mg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool build = false;
    Config* c = choose(s, &build);
    if (!c) {
      if (s->stop) return;
      s->cv_work.wait(lk);
      continue;
    }
    if (!c->h && !build) {                    // larger than the whole budget
      std::vector<Request*> all(c->queue.begin(), c->queue.end());
      c->queue.clear();
      finish(s, all, MG_ERR_NOMEM, nullptr);
      s->cv_done.notify_all();
      continue;
    }
    c->busy = true;
    if (build) {
      lk.unlock();
      const size_t vb = (size_t)s->max_rhs * c->Lx * c->Lt * 2 * 16;
      mg_handle* h = nullptr;
      mg_status st = mg_setup(c->gauge, c->setup_mass, &c->p, c->stream, &h);
      if (st == MG_OK && (cudaMalloc(&c->bbuf, vb) != cudaSuccess ||
                          cudaMalloc(&c->xbuf, vb) != cudaSuccess)) {
        cudaGetLastError();
        st = MG_ERR_NOMEM;
      }
      long long bytes = 0;
      if (st == MG_OK) mg_device_bytes(h, &bytes);
      lk.lock();
      if (st != MG_OK) {
        if (h) mg_destroy(h);
        cudaFree(c->bbuf);
        cudaFree(c->xbuf);
        c->bbuf = c->xbuf = nullptr;
        s->resident -= c->need;
        std::vector<Request*> all(c->queue.begin(), c->queue.end());
        c->queue.clear();
        finish(s, all, st, nullptr);
        c->busy = false;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
        continue;
      }
      c->h = h;
      c->cur_mass = c->setup_mass;
      c->resident = bytes + 2 * (long long)vb;  // the set-up's temporaries are freed
      s->resident += c->resident - c->need;
      ++s->builds;
    }
    // one batch: the oldest pending request at the hierarchy's current mass
    // (re-massing rebuilds the Galerkin operators and the coarsest inverse),
    // else the oldest request; with it every pending request of the same
    // mass, solver and tolerance that fits in max_rhs
    std::vector<Request*> batch;
    int total = 0;
    const Request* head = c->queue.front();
    for (const Request* r : c->queue)
      if (r->mass == c->cur_mass) {
        head = r;
        break;
      }
    const double mass = head->mass, tol = head->tol;
    const int solver = head->solver;
    for (auto it = c->queue.begin(); it != c->queue.end();) {
      Request* r = *it;
      if (r->mass == mass && r->tol == tol && r->solver == solver && total + r->nrhs <= s->max_rhs) {
        batch.push_back(r);
        total += r->nrhs;
        it = c->queue.erase(it);
      } else {
        ++it;
      }
    }
    lk.unlock();
    mg_status st = MG_OK;
    bool remassed = false;
    if (c->cur_mass != mass) {
      st = mg_set_mass(c->h, mass);
      if (st == MG_OK) {
        c->cur_mass = mass;
        remassed = true;
      }
    }
    std::vector<mg_solve_info> infos(total);
    if (st == MG_OK) {
      const size_t n = (size_t)c->Lx * c->Lt * 2 * 16;     // bytes of one right-hand side
      const void* b = batch[0]->b;
      void* x = batch[0]->x;
      if (batch.size() > 1) {
        size_t off = 0;
        for (Request* r : batch) {
          cudaMemcpyAsync((char*)c->bbuf + off, r->b, r->nrhs * n, cudaMemcpyDeviceToDevice,
                          c->stream);
          off += r->nrhs * n;
        }
        b = c->bbuf;
        x = c->xbuf;
      }
      st = mg_solve(c->h, b, x, total, tol, 1000000, solver, infos.data());
      if (batch.size() > 1 && (st == MG_OK || st == MG_ERR_NOCONV)) {
        size_t off = 0;
        for (Request* r : batch) {
          cudaMemcpyAsync(r->x, (char*)c->xbuf + off, r->nrhs * n, cudaMemcpyDeviceToDevice,
                          c->stream);
          off += r->nrhs * n;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = MG_ERR_CUDA;
      }
    }
    lk.lock();
    if (remassed) ++s->remasses;
    ++s->batches;
    s->batched_rhs += total;
    finish(s, batch, st, &infos);
    c->busy = false;
    c->last_used = ++s->tick;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t k = (size_t)std::ceil(q * (double)v.size());
  k = std::min(std::max<size_t>(k, 1), v.size());
  return v[k - 1];
}

}  // namespace

extern "C" {

mg_status mg_server_create(long long budget_bytes, int max_rhs, int workers, mg_server** out) {
  if (!out || budget_bytes <= 0 || max_rhs < 1 || max_rhs > 64 || workers < 1 || workers > 16)
    return MG_ERR_ARG;
  mg_server* s = new (std::nothrow) mg_server();
  if (!s) return MG_ERR_NOMEM;
  s->budget = budget_bytes;
  s->max_rhs = max_rhs;
  cudaGetDevice(&s->device);
  for (int k = 0; k < workers; ++k) s->workers.emplace_back(worker_main, s);
  *out = s;
  return MG_OK;
}

mg_status mg_server_add_config(mg_server* s, const void* gauge, const mg_params* params,
                               double setup_mass, int* config_id) {
  if (!s || !gauge || !params || !config_id) return MG_ERR_ARG;
  auto c = std::make_unique<Config>();
  c->p = *params;
  c->p.max_rhs = s->max_rhs;
  long long peak = 0;
  mg_status st = mg_setup_bytes(&c->p, nullptr, &peak);
  if (st != MG_OK) return st;
  c->Lx = params->Lx;
  c->Lt = params->Lt;
  c->setup_mass = setup_mass;
  c->need = peak + 2LL * s->max_rhs * c->Lx * c->Lt * 2 * 16;
  const size_t gb = (size_t)2 * c->Lx * c->Lt * 16;
  const size_t nb = (size_t)mg_setup_noise_len(params) * 16;
  if (cudaMalloc(&c->gauge, gb) != cudaSuccess) { cudaGetLastError(); return MG_ERR_NOMEM; }
  if (nb && cudaMalloc(&c->noise, nb) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->gauge);
    return MG_ERR_NOMEM;
  }
  if (cudaMemcpy(c->gauge, gauge, gb, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      (nb && cudaMemcpy(c->noise, params->setup_noise, nb, cudaMemcpyDeviceToDevice) != cudaSuccess) ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->gauge);
    cudaFree(c->noise);
    return MG_ERR_CUDA;
  }
  c->p.setup_noise = c->noise;
  std::lock_guard<std::mutex> g(s->mu);
  c->id = (int)s->cfgs.size();
  *config_id = c->id;
  s->cfgs.push_back(std::move(c));
  return MG_OK;
}

mg_status mg_server_submit(mg_server* s, int config_id, double mass, const void* b, void* x,
                           int nrhs, double tol, int solver, long long* request_id) {
  if (!s || !b || !x || !request_id || !(tol > 0.0) || nrhs < 1) return MG_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (config_id < 0 || config_id >= (int)s->cfgs.size() || nrhs > s->max_rhs) return MG_ERR_ARG;
  auto r = std::make_unique<Request>();
  r->id = s->next_id++;
  r->cfg = config_id;
  r->mass = mass;
  r->b = b;
  r->x = x;
  r->nrhs = nrhs;
  r->tol = tol;
  r->solver = solver;
  r->t_submit = Clock::now();
  *request_id = r->id;
  s->cfgs[config_id]->queue.push_back(r.get());
  s->reqs.emplace(r->id, std::move(r));
  ++s->submitted;
  s->cv_work.notify_one();
  return MG_OK;
}

mg_status mg_server_wait(mg_server* s, long long request_id, mg_solve_info* info,
                         double* latency_ms) {
  if (!s) return MG_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return MG_ERR_ARG;
  Request* r = it->second.get();
  s->cv_done.wait(lk, [&] { return r->done; });
  const mg_status st = r->st;
  if (info && !r->info.empty()) std::memcpy(info, r->info.data(), r->info.size() * sizeof(mg_solve_info));
  if (latency_ms) *latency_ms = r->latency_ms;
  s->reqs.erase(it);
  return st;
}

mg_status mg_server_get_stats(mg_server* s, mg_server_stats* out) {
  if (!s || !out) return MG_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->batches = s->batches;
  out->batched_rhs = s->batched_rhs;
  out->builds = s->builds;
  out->evictions = s->evictions;
  out->remasses = s->remasses;
  out->resident_bytes = s->resident;
  out->peak_resident_bytes = s->peak_resident;
  out->budget_bytes = s->budget;
  out->p50_ms = percentile(s->latencies, 0.50);
  out->p99_ms = percentile(s->latencies, 0.99);
  out->max_ms = percentile(s->latencies, 1.0);
  return MG_OK;
}

void mg_server_destroy(mg_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] {
      for (auto& c : s->cfgs)
        if (c->busy || !c->queue.empty()) return false;
      return true;
    });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& c : s->cfgs) {
    if (c->h) evict(s, c.get());
    cudaFree(c->gauge);
    cudaFree(c->noise);
    if (c->stream) cudaStreamDestroy(c->stream);
  }
  delete s;
}

}  // extern "C"
