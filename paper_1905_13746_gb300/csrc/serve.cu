// Serving loop: continuous batching of arriving file groups.
//
// The paper classifies the files of a group with the group's model (Sec. 3,
// Sec. 4); a server keeps the models resident and classifies groups as they
// arrive.  A host worker thread admits queued groups in arrival order while
// batch slots and device-memory budget are free, copies host inputs to the
// device on a copy stream, and at each step scores every admitted group in
// one batch (nb_batch_score, replaying a captured graph) while the previous
// step may still be running; finished steps return their slots and memory and
// complete their tickets.  All waits are bounded or time out.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "seg.cuh"

namespace nbg {

using Clock = std::chrono::steady_clock;

static double now_us() {
  return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

// first-fit allocator over [0, cap) with coalescing, 256-byte granules
class RangePool {
 public:
  explicit RangePool(size_t cap = 0) { reset(cap); }
  void reset(size_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t ticket;
  int model;
  const void* X;
  int64_t n;
  bool in_host = false;  // X is host memory: staged through the device pool
  int out_kind = 0;      // outputs: 0 device memory, 1 pinned host, 2 pageable host (staged)
  uint8_t* label;
  float* margin;
  float* logpost;
  double t_arrive = 0, t_done = 0;
  bool done = false;
  // staging
  size_t off = 0, bytes = 0;      // device pool (inputs from the host, outputs to the host)
  size_t hoff = 0, hbytes = 0;    // pinned host pool (outputs)
  char* dX = nullptr;
  uint8_t* dlabel = nullptr;
  float* dmargin = nullptr;
  float* dlogpost = nullptr;
  cudaEvent_t copied = nullptr;
};

struct Step {
  std::vector<Req*> reqs;
  cudaEvent_t done;
};

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace nbg

using namespace nbg;

struct nb_server {
  std::vector<const nb_model*> models;
  std::vector<int> C;
  nb_dtype dtype;
  int F = 0, es = 1, device = 0, max_slots = 1, want_lp = 0;
  nb_batch* batch = nullptr;
  cudaStream_t copy_st = nullptr, comp_st = nullptr;
  char* dpool = nullptr;
  char* hpool = nullptr;
  size_t budget = 0, hbudget = 0;
  RangePool pool, hpool_alloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::deque<Step> steps;
  std::vector<cudaEvent_t> event_cache;
  std::unordered_map<uint64_t, Req*> tickets;
  std::vector<double> lat_us;
  double first_arrival = -1, last_done = 0;
  uint64_t files_done = 0, next_ticket = 1;
  int slots_used = 0;
  bool stop = false;
  nb_status fault = NB_OK;
  std::thread worker;
  std::vector<nb_group> gbuf;
};

static cudaEvent_t take_event(nb_server* s) {
  if (!s->event_cache.empty()) {
    cudaEvent_t e = s->event_cache.back();
    s->event_cache.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

// device staging bytes of a request: its input when it comes from the host,
// its outputs when they go to the host
static size_t dev_stage_bytes(const nb_server* s, const Req* r) {
  if (r->n == 0) return 0;
  const size_t n = (size_t)r->n;
  size_t b = r->in_host ? round256(n * s->F * s->es) : 0;
  if (r->out_kind != 0)
    b += round256(n) + round256(n * 4) + (r->logpost ? round256(n * 4 * s->C[r->model]) : 0);
  return b;
}

static size_t out_bytes(const nb_server* s, const Req* r) {
  return (size_t)r->n * (1 + 4 + (r->logpost ? 4 * (size_t)s->C[r->model] : 0));
}

static void finish_req(nb_server* s, Req* r) {
  if (r->out_kind == 2 && r->n > 0) {
    const int C = s->C[r->model];
    const char* h = s->hpool + r->hoff;
    memcpy(r->label, h, (size_t)r->n);
    memcpy(r->margin, h + (size_t)r->n, (size_t)r->n * 4);
    if (r->logpost) memcpy(r->logpost, h + (size_t)r->n * 5, (size_t)r->n * 4 * C);
    s->hpool_alloc.release(r->hoff, r->hbytes);
  }
  if (r->bytes) s->pool.release(r->off, r->bytes);
  if (r->copied) s->event_cache.push_back(r->copied);
  r->copied = nullptr;
  r->t_done = now_us();
  r->done = true;
  s->lat_us.push_back(r->t_done - r->t_arrive);
  s->last_done = r->t_done;
  s->files_done += (uint64_t)r->n;
  --s->slots_used;
}

static void worker_loop(nb_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  std::vector<Req*> admitted;
  for (;;) {
    // 1. completions, oldest step first
    bool progressed = false;
    while (!s->steps.empty() && cudaEventQuery(s->steps.front().done) == cudaSuccess) {
      Step st = s->steps.front();
      s->steps.pop_front();
      for (Req* r : st.reqs) finish_req(s, r);
      s->event_cache.push_back(st.done);
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // 2. admission in arrival order
    // (a step takes at most max_slots groups; device memory is the admission limit)
    while (!s->queue.empty() && (int)admitted.size() < s->max_slots) {
      Req* r = s->queue.front();
      const size_t db = dev_stage_bytes(s, r);
      size_t off = 0, hoff = 0;
      if (db && !s->pool.alloc(db, &off)) break;
      if (r->out_kind == 2 && r->n > 0) {
        if (!s->hpool_alloc.alloc(out_bytes(s, r) + 256, &hoff)) {
          if (db) s->pool.release(off, db);
          break;
        }
        r->hoff = hoff;
        r->hbytes = out_bytes(s, r) + 256;
      }
      r->off = off;
      r->bytes = db;
      if (db) {
        const size_t n = (size_t)r->n;
        char* base = s->dpool + off;
        size_t o = 0;
        if (r->in_host) {
          r->dX = base;
          o = round256(n * s->F * s->es);
          cudaMemcpyAsync(r->dX, r->X, n * s->F * s->es, cudaMemcpyHostToDevice, s->copy_st);
          r->copied = take_event(s);
          cudaEventRecord(r->copied, s->copy_st);
        }
        if (r->out_kind != 0) {
          r->dlabel = reinterpret_cast<uint8_t*>(base + o);
          o += round256(n);
          r->dmargin = reinterpret_cast<float*>(base + o);
          o += round256(n * 4);
          r->dlogpost = r->logpost ? reinterpret_cast<float*>(base + o) : nullptr;
        }
      }
      ++s->slots_used;
      s->queue.pop_front();
      admitted.push_back(r);
    }
    // 3. one step over everything admitted (at most two steps in flight)
    if (!admitted.empty() && s->steps.size() < 2) {
      s->gbuf.clear();
      for (Req* r : admitted) {
        if (r->n == 0) continue;
        nb_group g{};
        g.model = r->model;
        g.n = r->n;
        g.ld = s->F;
        g.X = r->in_host ? r->dX : r->X;
        if (r->copied) cudaStreamWaitEvent(s->comp_st, r->copied, 0);
        if (r->out_kind == 0) {
          g.label = r->label;
          g.margin = r->margin;
          g.logpost = r->logpost;
        } else {
          g.label = r->dlabel;
          g.margin = r->dmargin;
          g.logpost = r->dlogpost;
        }
        s->gbuf.push_back(g);
      }
      if (!s->gbuf.empty()) {
        nb_status st = nb_batch_score(s->batch, s->gbuf.data(), (int)s->gbuf.size(),
                                      s->comp_st, nullptr);
        if (st != NB_OK && s->fault == NB_OK) s->fault = st;
      }
      for (Req* r : admitted) {
        if (r->out_kind == 0 || r->n == 0) continue;
        const size_t n = (size_t)r->n;
        const int C = s->C[r->model];
        uint8_t* hl = r->label;
        float* hm = r->margin;
        float* hp = r->logpost;
        if (r->out_kind == 2) {
          char* h = s->hpool + r->hoff;
          hl = reinterpret_cast<uint8_t*>(h);
          hm = reinterpret_cast<float*>(h + n);
          hp = reinterpret_cast<float*>(h + n * 5);
        }
        cudaMemcpyAsync(hl, r->dlabel, n, cudaMemcpyDeviceToHost, s->comp_st);
        cudaMemcpyAsync(hm, r->dmargin, n * 4, cudaMemcpyDeviceToHost, s->comp_st);
        if (r->logpost)
          cudaMemcpyAsync(hp, r->dlogpost, n * 4 * C, cudaMemcpyDeviceToHost, s->comp_st);
      }
      Step stp;
      stp.reqs = admitted;
      stp.done = take_event(s);
      cudaEventRecord(stp.done, s->comp_st);
      s->steps.push_back(stp);
      admitted.clear();
      continue;
    }
    if (s->stop && s->queue.empty() && admitted.empty() && s->steps.empty()) break;
    // 4. wait: poll briefly while the GPU works, else sleep until a submission
    if (!s->steps.empty()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else if (admitted.empty()) {
      s->cv_work.wait_for(lk, s->queue.empty() ? std::chrono::microseconds(2000)
                                               : std::chrono::microseconds(50));
    }
  }
}

extern "C" nb_status nb_server_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                                      size_t mem_budget, int max_slots, const nb_score_opts* opts,
                                      nb_server** out) {
  if (!out || !models || n_models < 1 || n_models > kSegMaxModels || max_slots < 1 ||
      elem_size(dtype) == 0) {
    set_error("nb_server_create: need 1..8 models, max_slots >= 1, a valid dtype");
    return NB_EINVAL;
  }
  *out = nullptr;
  nb_server* s = new (std::nothrow) nb_server();
  if (!s) {
    set_error("nb_server_create: out of host memory");
    return NB_ENOMEM;
  }
  s->dtype = dtype;
  s->es = elem_size(dtype);
  s->F = models[0]->F;
  s->max_slots = max_slots;
  s->want_lp = opts ? opts->want_logpost : 0;
  for (int i = 0; i < n_models; ++i) {
    s->models.push_back(models[i]);
    s->C.push_back(models[i]->C);
  }
  cudaGetDevice(&s->device);
  auto fail = [&](nb_status st) {
    nb_server_destroy(s);
    return st;
  };
  nb_status st = nb_batch_create(models, n_models, dtype, s->F, max_slots, opts, &s->batch);
  if (st != NB_OK) return fail(st);
  cudaError_t e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->comp_st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaStreamCreate"));
  s->budget = mem_budget ? mem_budget : (size_t(1) << 30);
  e = cudaMalloc(reinterpret_cast<void**>(&s->dpool), s->budget);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc(server budget)"));
  int cmax = 2;
  for (int c : s->C) cmax = std::max(cmax, c);
  // outputs of everything the device budget can stage, in pinned host memory
  s->hbudget = s->budget / (size_t)(s->F * s->es) * (size_t)(1 + 4 + 4 * cmax) + (1 << 20);
  e = cudaMallocHost(reinterpret_cast<void**>(&s->hpool), s->hbudget);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMallocHost(server)"));
  s->pool.reset(s->budget);
  s->hpool_alloc.reset(s->hbudget);
  st = nb_batch_capture(s->batch, s->comp_st);
  if (st != NB_OK) return fail(st);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return NB_OK;
}

// validates one submission and builds its request (arrival = t_arrive)
static nb_status make_req(nb_server* s, int model_id, const void* X, int64_t n, uint8_t* label,
                          float* margin, float* logpost, double t_arrive, Req** out) {
  if (model_id < 0 || model_id >= (int)s->models.size() || n < 0 ||
      (n > 0 && (!X || !label || !margin || (s->want_lp && !logpost)))) {
    set_error("nb_classify_stream: bad model id, sizes or pointers");
    return NB_EINVAL;
  }
  // 0 device, 1 pinned (page-locked) host, 2 pageable host
  auto kind = [](const void* p) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    cudaGetLastError();
    if (e != cudaSuccess || a.type == cudaMemoryTypeUnregistered) return 2;
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 0 : 1;
  };
  Req tmp;
  tmp.model = model_id;
  tmp.n = n;
  tmp.logpost = s->want_lp ? logpost : nullptr;
  if (n > 0) {
    tmp.in_host = kind(X) != 0;
    const int kl = kind(label), km = kind(margin), kp = tmp.logpost ? kind(logpost) : kl;
    const int lo = std::min(kl, std::min(km, kp)), hi = std::max(kl, std::max(km, kp));
    if (lo == 0 && hi != 0) {
      set_error("nb_classify_stream: outputs must be all device or all host memory");
      return NB_EINVAL;
    }
    tmp.out_kind = hi;
    const size_t need = dev_stage_bytes(s, &tmp);
    const size_t hneed = hi == 2 ? out_bytes(s, &tmp) + 256 : 0;
    if (need > s->budget || hneed > s->hbudget) {
      set_error("nb_classify_stream: the group needs %zu device / %zu host staging bytes, more "
                "than the budgets %zu / %zu", need, hneed, s->budget, s->hbudget);
      return NB_EBUSY;
    }
  }
  Req* r = new (std::nothrow) Req();
  if (!r) {
    set_error("nb_classify_stream: out of host memory");
    return NB_ENOMEM;
  }
  r->model = model_id;
  r->X = X;
  r->n = n;
  r->in_host = tmp.in_host;
  r->out_kind = tmp.out_kind;
  r->label = label;
  r->margin = margin;
  r->logpost = tmp.logpost;
  r->t_arrive = t_arrive;
  *out = r;
  return NB_OK;
}

// queues built requests under the server lock; false when shutting down
static bool enqueue(nb_server* s, Req* const* reqs, int count, uint64_t* tickets) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return false;
    for (int i = 0; i < count; ++i) {
      Req* r = reqs[i];
      r->ticket = s->next_ticket++;
      if (s->first_arrival < 0 || r->t_arrive < s->first_arrival) s->first_arrival = r->t_arrive;
      s->tickets[r->ticket] = r;
      s->queue.push_back(r);
      tickets[i] = r->ticket;
    }
  }
  s->cv_work.notify_one();
  return true;
}

extern "C" nb_status nb_classify_stream(nb_server* s, int model_id, const void* X, int64_t n,
                                        int32_t F, uint8_t* label, float* margin, float* logpost,
                                        uint64_t* ticket) {
  if (!s || !ticket || F != s->F) {
    set_error("nb_classify_stream: NULL server or ticket, or F differs from the models'");
    return NB_EINVAL;
  }
  Req* r = nullptr;
  nb_status st = make_req(s, model_id, X, n, label, margin, logpost, now_us(), &r);
  if (st != NB_OK) return st;
  if (!enqueue(s, &r, 1, ticket)) {
    delete r;
    set_error("nb_classify_stream: server is shutting down");
    return NB_EBUSY;
  }
  return NB_OK;
}

extern "C" nb_status nb_classify_stream_batch(nb_server* s, int count, const int* model_ids,
                                              const void* const* X, const int64_t* n,
                                              uint8_t* const* label, float* const* margin,
                                              float* const* logpost, const double* arrival_us,
                                              uint64_t* tickets, int* submitted) {
  if (submitted) *submitted = 0;
  if (!s || count < 0 || (count > 0 && (!model_ids || !X || !n || !label || !margin ||
                                        !tickets || (s->want_lp && !logpost)))) {
    set_error("nb_classify_stream_batch: NULL server or arrays");
    return NB_EINVAL;
  }
  std::vector<Req*> reqs;
  reqs.reserve((size_t)count);
  const double t = now_us();
  nb_status st = NB_OK;
  for (int i = 0; i < count && st == NB_OK; ++i) {
    Req* r = nullptr;
    st = make_req(s, model_ids[i], X[i], n[i], label[i], margin[i], logpost ? logpost[i] : nullptr,
                  arrival_us ? arrival_us[i] : t, &r);
    if (st == NB_OK) reqs.push_back(r);
  }
  if (!enqueue(s, reqs.data(), (int)reqs.size(), tickets)) {
    for (Req* r : reqs) delete r;
    set_error("nb_classify_stream_batch: server is shutting down");
    return NB_EBUSY;
  }
  if (submitted) *submitted = (int)reqs.size();
  return st;
}

extern "C" double nb_clock_us(void) { return now_us(); }

extern "C" nb_status nb_wait(nb_server* s, uint64_t ticket, int64_t timeout_us) {
  if (!s) {
    set_error("nb_wait: NULL server");
    return NB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) {
    set_error("nb_wait: unknown or already collected ticket %llu", (unsigned long long)ticket);
    return NB_EINVAL;
  }
  Req* r = it->second;
  auto pred = [&]() { return r->done; };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    set_error("nb_wait: ticket %llu not complete after %lld us", (unsigned long long)ticket,
              (long long)timeout_us);
    return NB_ETIMEOUT;
  }
  s->tickets.erase(it);
  delete r;
  if (s->fault != NB_OK) {
    set_error("nb_wait: a batch of this server failed");
    return s->fault;
  }
  return NB_OK;
}

extern "C" nb_status nb_server_stats(nb_server* s, double* p50_us, double* p99_us,
                                     double* files_per_s) {
  if (!s) {
    set_error("nb_server_stats: NULL server");
    return NB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->lat_us;
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)k, v.end());
    return v[k];
  };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (files_per_s) {
    const double span = s->last_done - s->first_arrival;
    *files_per_s = span > 0 ? (double)s->files_done / (span * 1e-6) : 0.0;
  }
  return NB_OK;
}

extern "C" void nb_server_destroy(nb_server* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  for (auto& kv : s->tickets) delete kv.second;
  for (cudaEvent_t e : s->event_cache) cudaEventDestroy(e);
  if (s->batch) nb_batch_destroy(s->batch);
  if (s->copy_st) cudaStreamSynchronize(s->copy_st);
  if (s->comp_st) cudaStreamSynchronize(s->comp_st);
  if (s->copy_st) cudaStreamDestroy(s->copy_st);
  if (s->comp_st) cudaStreamDestroy(s->comp_st);
  if (s->dpool) cudaFree(s->dpool);
  if (s->hpool) cudaFreeHost(s->hpool);
  delete s;
}
