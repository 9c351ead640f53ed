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

// One resident hierarchy of a configuration at one mass, with its own
// stream and batch buffers.
struct Hier {
  double mass = 0.0;
  mg_handle* h = nullptr;
  cudaStream_t stream = nullptr;
  void* bbuf = nullptr;          // batch staging, [max_rhs][Lt][Lx][2] complex128 each
  void* xbuf = nullptr;
  long long bytes = 0;           // device bytes while resident
  bool busy = false;             // held by a worker (solving, or being built)
  bool ready = false;            // built (set under the lock when the build returns)
  int readers = 0;               // clones being made from it (not evictable meanwhile)
  long long last_used = 0;
};

struct Config {
  int id = 0;
  mg_params p{};
  double setup_mass = 0.0;
  int Lx = 0, Lt = 0;
  void* gauge = nullptr;         // device copies owned by the server
  void* noise = nullptr;
  long long need_setup = 0;      // peak bytes of a set-up + batch buffers
  long long need_clone = 0;      // resident bytes of a hierarchy + batch buffers
  std::vector<std::unique_ptr<Hier>> hs;
  std::deque<Request*> queue;
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
  long long builds = 0, clones = 0, evictions = 0, remasses = 0;
  int inject_build_failures = 0;   // host-side fault injection (mg_server_inject_build_failures)
  std::vector<double> latencies;
};

namespace {

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

void erase_hier(Config* c, const Hier* r) {
  for (auto it = c->hs.begin(); it != c->hs.end(); ++it)
    if (it->get() == r) {
      c->hs.erase(it);
      return;
    }
}

void free_hier(Hier* r) {
  mg_destroy(r->h);
  cudaFree(r->bbuf);
  cudaFree(r->xbuf);
  if (r->stream) cudaStreamDestroy(r->stream);
  r->h = nullptr;
  r->bbuf = r->xbuf = nullptr;
  r->stream = nullptr;
}

bool pending_at(const Config* c, double mass) {
  for (const Request* q : c->queue)
    if (q->mass == mass) return true;
  return false;
}

// Destroys idle hierarchies (not held, not a clone source, no pending request
// at their mass), least recently used first, until `need` more bytes fit;
// false if they cannot.  The lock is held.
bool make_room(mg_server* s, long long need) {
  if (s->resident + need <= s->budget) return true;
  std::vector<std::pair<Config*, Hier*>> idle;
  long long freeable = 0;
  for (auto& c : s->cfgs)
    for (auto& r : c->hs)
      if (!r->busy && !r->readers && !pending_at(c.get(), r->mass)) {
        idle.push_back({c.get(), r.get()});
        freeable += r->bytes;
      }
  if (s->resident - freeable + need > s->budget) return false;
  std::sort(idle.begin(), idle.end(),
            [](const auto& a, const auto& b) { return a.second->last_used < b.second->last_used; });
  for (auto& cr : idle) {
    if (s->resident + need <= s->budget) break;
    free_hier(cr.second);
    s->resident -= cr.second->bytes;
    ++s->evictions;
    erase_hier(cr.first, cr.second);
  }
  return true;
}

Hier* find_hier(Config* c, double mass) {
  for (auto& r : c->hs)
    if (r->mass == mass) return r.get();
  return nullptr;
}

// What a worker does next (chosen with the lock held; never waits).
struct Job {
  Config* c = nullptr;
  Hier* r = nullptr;             // the hierarchy that serves the batch
  double mass = 0.0;
  enum { RUN, BUILD, CLONE, REMASS, FAIL } kind = RUN;
  Hier* src = nullptr;           // clone source
};

// Pending (configuration, mass) groups in the order of their oldest request.
// A group whose hierarchy exists and is free runs.  One without a hierarchy
// gets a new one if memory allows (after evicting idle ones): a clone of a
// resident hierarchy of its configuration, else a set-up; otherwise an idle
// hierarchy of the same configuration is re-massed.  A configuration larger
// than the whole budget fails.
bool choose(mg_server* s, Job* job) {
  struct G { long long id; Config* c; double mass; };
  std::vector<G> groups;
  for (auto& c : s->cfgs)
    for (const Request* q : c->queue) {
      bool seen = false;
      for (const G& g : groups)
        if (g.c == c.get() && g.mass == q->mass) seen = true;
      if (!seen) groups.push_back({q->id, c.get(), q->mass});
    }
  std::sort(groups.begin(), groups.end(), [](const G& a, const G& b) { return a.id < b.id; });
  for (const G& g : groups) {
    Config* c = g.c;
    job->c = c;
    job->mass = g.mass;
    if (Hier* r = find_hier(c, g.mass)) {
      if (r->busy) continue;
      job->r = r;
      job->kind = Job::RUN;
      return true;
    }
    Hier* src = nullptr;
    for (auto& r : c->hs)
      if (r->ready && (!src || r->last_used > src->last_used)) src = r.get();
    if (!src && !c->hs.empty()) continue;      // its first hierarchy is being built: clone later
    const long long need = src ? c->need_clone : c->need_setup;
    if (!src && c->need_setup > s->budget) {
      job->kind = Job::FAIL;
      return true;
    }
    if (make_room(s, need)) {
      auto r = std::make_unique<Hier>();
      r->mass = g.mass;
      r->busy = true;
      r->bytes = need;                          // reserved; exact after the build
      s->resident += need;
      s->peak_resident = std::max(s->peak_resident, s->resident);
      job->r = r.get();
      job->src = src;
      job->kind = src ? Job::CLONE : Job::BUILD;
      if (src) ++src->readers;
      c->hs.push_back(std::move(r));
      return true;
    }
    for (auto& r : c->hs)                        // re-mass an idle hierarchy instead
      if (r->ready && !r->busy && !r->readers && !pending_at(c, r->mass)) {
        r->mass = g.mass;                          // serves this group from now on
        r->busy = true;
        job->r = r.get();
        job->kind = Job::REMASS;
        return true;
      }
  }
  return false;
}

// Fails the queued requests of configuration c; mass != nullptr: only those at
// that mass (a failed build or clone concerns its own group only).
void fail_queue(mg_server* s, Config* c, mg_status st, const double* mass = nullptr) {
  std::vector<Request*> out;
  for (auto it = c->queue.begin(); it != c->queue.end();) {
    if (!mass || (*it)->mass == *mass) {
      out.push_back(*it);
      it = c->queue.erase(it);
    } else {
      ++it;
    }
  }
  finish(s, out, st, nullptr);
}

void worker_main(mg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    Job job;
    if (!choose(s, &job)) {
      if (s->stop) return;
      s->cv_work.wait(lk);
      continue;
    }
    Config* c = job.c;
    Hier* r = job.r;
    if (job.kind == Job::FAIL) {
      fail_queue(s, c, MG_ERR_NOMEM);
      s->cv_done.notify_all();
      continue;
    }
    r->busy = true;
    const size_t vb = (size_t)s->max_rhs * c->Lx * c->Lt * 2 * 16;
    if (job.kind == Job::BUILD || job.kind == Job::CLONE) {
      const bool inject = s->inject_build_failures > 0;
      if (inject) --s->inject_build_failures;
      lk.unlock();
      mg_status st = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) == cudaSuccess
                         ? MG_OK : MG_ERR_CUDA;
      if (st == MG_OK && inject) {
        // stands in for a failing mg_setup / mg_clone, after a while so that
        // builds of other groups are in flight meanwhile
        std::this_thread::sleep_for(std::chrono::milliseconds(50));
        st = MG_ERR_CUDA;
      } else if (st == MG_OK) {
        if (job.kind == Job::CLONE) {
          st = mg_clone(job.src->h, job.mass, r->stream, &r->h);
        } else {
          st = mg_setup(c->gauge, c->setup_mass, &c->p, r->stream, &r->h);
          if (st == MG_OK && job.mass != c->setup_mass) st = mg_set_mass(r->h, job.mass);
        }
      }
      if (st == MG_OK && (cudaMalloc(&r->bbuf, vb) != cudaSuccess ||
                          cudaMalloc(&r->xbuf, vb) != cudaSuccess)) {
        cudaGetLastError();
        st = MG_ERR_NOMEM;
      }
      long long bytes = 0;
      if (st == MG_OK) mg_device_bytes(r->h, &bytes);
      lk.lock();
      if (job.src) --job.src->readers;
      if (st != MG_OK) {
        free_hier(r);
        s->resident -= r->bytes;
        erase_hier(c, r);
        fail_queue(s, c, st, &job.mass);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
        continue;
      }
      s->resident += bytes + 2 * (long long)vb - r->bytes;
      r->bytes = bytes + 2 * (long long)vb;
      r->ready = true;
      if (job.kind == Job::CLONE) ++s->clones; else ++s->builds;
    }
    // one batch: the oldest pending request at this mass and every other one
    // with the same solver and tolerance that fits in max_rhs
    std::vector<Request*> batch;
    int total = 0;
    const Request* head = nullptr;
    for (const Request* q : c->queue)
      if (q->mass == job.mass) {
        head = q;
        break;
      }
    if (!head) {                      // nothing left at this mass: release the hierarchy
      if (job.kind == Job::REMASS) {  // it was re-labelled but never re-massed
        free_hier(r);
        s->resident -= r->bytes;
        erase_hier(c, r);
      } else {
        r->busy = false;
        r->last_used = ++s->tick;
      }
      s->cv_done.notify_all();
      s->cv_work.notify_all();
      continue;
    }
    const double tol = head->tol;
    const int solver = head->solver;
    for (auto it = c->queue.begin(); it != c->queue.end();) {
      Request* q = *it;
      if (q->mass == job.mass && q->tol == tol && q->solver == solver &&
          total + q->nrhs <= s->max_rhs) {
        batch.push_back(q);
        total += q->nrhs;
        it = c->queue.erase(it);
      } else {
        ++it;
      }
    }
    lk.unlock();
    mg_status st = MG_OK;
    if (job.kind == Job::REMASS) st = mg_set_mass(r->h, job.mass);
    std::vector<mg_solve_info> infos(total);
    if (st == MG_OK) {
      const size_t n = (size_t)c->Lx * c->Lt * 2 * 16;     // bytes of one right-hand side
      const void* b = batch[0]->b;
      void* x = batch[0]->x;
      if (batch.size() > 1) {
        size_t off = 0;
        for (Request* q : batch) {
          cudaMemcpyAsync((char*)r->bbuf + off, q->b, q->nrhs * n, cudaMemcpyDeviceToDevice,
                          r->stream);
          off += q->nrhs * n;
        }
        b = r->bbuf;
        x = r->xbuf;
      }
      st = mg_solve(r->h, b, x, total, tol, 1000000, solver, infos.data());
      if (batch.size() > 1 && (st == MG_OK || st == MG_ERR_NOCONV)) {
        size_t off = 0;
        for (Request* q : batch) {
          cudaMemcpyAsync(q->x, (char*)r->xbuf + off, q->nrhs * n, cudaMemcpyDeviceToDevice,
                          r->stream);
          off += q->nrhs * n;
        }
        if (cudaStreamSynchronize(r->stream) != cudaSuccess) st = MG_ERR_CUDA;
      }
    }
    lk.lock();
    if (job.kind == Job::REMASS && st == MG_OK) ++s->remasses;
    ++s->batches;
    s->batched_rhs += total;
    finish(s, batch, st, &infos);
    r->busy = false;
    r->last_used = ++s->tick;
    if (job.kind == Job::REMASS && st != MG_OK) {   // state of a failed re-mass is unknown
      free_hier(r);
      s->resident -= r->bytes;
      erase_hier(c, r);
    }
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
  long long resident = 0, peak = 0;
  mg_status st = mg_setup_bytes(&c->p, &resident, &peak);
  if (st != MG_OK) return st;
  c->Lx = params->Lx;
  c->Lt = params->Lt;
  c->setup_mass = setup_mass;
  const long long vb = 2LL * s->max_rhs * c->Lx * c->Lt * 2 * 16;
  c->need_setup = peak + vb;
  c->need_clone = resident + vb;
  const size_t gb = (size_t)2 * c->Lx * c->Lt * 16;
  const size_t nb = (size_t)mg_setup_noise_len(params) * 16;
  if (cudaMalloc(&c->gauge, gb) != cudaSuccess) { cudaGetLastError(); return MG_ERR_NOMEM; }
  if (nb && cudaMalloc(&c->noise, nb) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->gauge);
    return MG_ERR_NOMEM;
  }
  if (cudaMemcpy(c->gauge, gauge, gb, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      (nb && cudaMemcpy(c->noise, params->setup_noise, nb, cudaMemcpyDeviceToDevice) != cudaSuccess)) {
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

mg_status mg_server_inject_build_failures(mg_server* s, int count) {
  if (!s || count < 0) return MG_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  s->inject_build_failures = count;
  return MG_OK;
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
  out->clones = s->clones;
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
      for (auto& c : s->cfgs) {
        if (!c->queue.empty()) return false;
        for (auto& r : c->hs)
          if (r->busy) return false;
      }
      return true;
    });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& c : s->cfgs) {
    for (auto& r : c->hs) free_hier(r.get());
    cudaFree(c->gauge);
    cudaFree(c->noise);
  }
  delete s;
}

}  // extern "C"
