// Continuous-batching request loop for encrypted queries (the serving side of
// CryptoTL's protocol: every client query is one ClassifyHE call, Fig. alg:cryptotl).
//
// A server holds lanes (one parameter set + frozen model each) and clients (one key set
// each, resident in HBM, bound to a lane).  Requests are ciphertexts in coefficient form
// from host memory.  Worker threads take the oldest queued request, group it with the
// other queued requests of the same client (up to max_batch: they share keys, so they
// run as one batch), reserve their device-memory estimate against the budget (admission)
// and run import -> forward -> export on their own stream, so batches of different clients
// overlap on the device and new requests are admitted as earlier ones finish.  A failing
// batch marks its requests failed and the loop keeps serving.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <algorithm>
#include "ctl_internal.h"

using namespace ctl;
using Clock = std::chrono::steady_clock;

extern "C" int ctl_context_clone(const ctl_context* c, ctl_context** out);

namespace {

struct Lane {
  ctl_context* ctx;
  const ctl_model* model;
  uint32_t in_level, out_level;
  double in_scale;
  size_t in_words, out_words;  // per ciphertext
  uint64_t bytes_per_ct;       // admission estimate of device memory per in-flight ciphertext
};
struct Client {
  uint32_t lane;
  const ctl_keys* keys;
};
struct Request {
  uint64_t id;
  uint32_t client;
  std::vector<u64> in, out;
  int status = 1;  // 1 queued, 2 running, 0 done, <0 error code
  Clock::time_point t_submit, t_done;
};
struct Worker {
  std::thread th;
  std::vector<ctl_context*> ctx;  // one clone per lane
  std::vector<u64*> pin_in, pin_out;  // pinned staging per lane
};

}  // namespace

struct ctl_server {
  uint64_t budget = 0, reserved = 0;
  uint32_t max_batch = 1, max_queue = 1, n_workers = 1;
  std::vector<Lane> lanes;
  std::vector<Client> clients;
  std::vector<Worker> workers;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_id = 1;
  bool started = false, stopping = false;
  uint64_t n_submitted = 0, n_completed = 0, n_rejected = 0, n_failed = 0, n_batches = 0, batched_cts = 0;
  uint64_t peak_reserved = 0, n_deferred = 0;  // admission: high-water mark, waits for memory
  std::vector<double> latencies_ms;
};

namespace {

uint64_t estimate_bytes_per_ct(const ctl_context* c, const ctl_model* M, uint32_t in_level) {
  // Admission estimate (not an allocation): the baby steps and inner sums of the widest
  // dense layer (t1 + t2 <= 2 * 2^ceil(log2(t)/2) ciphertexts, t bounded by the largest
  // rotation of the model) plus ping-pong buffers and key-switching temporaries.
  const uint64_t ct = 2ull * in_level * c->N * 8;
  uint32_t nr = 0;
  ctl_model_rotations(M, nullptr, 0, &nr);
  std::vector<int32_t> rots(nr ? nr : 1);
  ctl_model_rotations(M, rots.data(), nr, &nr);
  int32_t mx = 1;
  for (uint32_t i = 0; i < nr; i++) mx = std::max(mx, rots[i] < 0 ? -rots[i] : rots[i]);
  uint32_t t = 1;
  while ((int32_t)t <= mx) t <<= 1;
  uint32_t lg = 0;
  while ((1u << lg) < t) lg++;
  const uint64_t widest = 2ull * (1u << ((lg + 1) / 2)) + 8;
  return ct * widest + ct * (c->K + 4);
}

void finish(ctl_server* s, std::vector<Request*>& grp, int rc) {
  std::lock_guard<std::mutex> lk(s->mu);
  const auto now = Clock::now();
  for (Request* r : grp) {
    r->status = rc;
    r->t_done = now;
    if (rc == 0) {
      s->n_completed++;
      s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
    } else {
      s->n_failed++;
    }
  }
  s->cv.notify_all();
}

void worker_loop(ctl_server* s, uint32_t wi) {
  Worker& W = s->workers[wi];
  cudaSetDevice(s->lanes[0].ctx->device);
  for (;;) {
    std::vector<Request*> grp;
    uint32_t lane = 0;
    uint64_t need = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stopping) return;
        if (!s->queue.empty()) {
          Request* head = s->reqs[s->queue.front()].get();
          const Client& cl = s->clients[head->client];
          const Lane& ln = s->lanes[cl.lane];
          // group the oldest request with queued requests of the same client
          std::vector<uint64_t> ids;
          for (uint64_t id : s->queue) {
            if (s->reqs[id]->client == head->client) ids.push_back(id);
            if (ids.size() >= s->max_batch) break;
          }
          // admission: shrink the group to fit the budget; one request may always run alone
          size_t n = ids.size();
          while (n > 1 && s->reserved + n * ln.bytes_per_ct > s->budget) n--;
          if (s->reserved + n * ln.bytes_per_ct <= s->budget || s->reserved == 0) {
            need = n * ln.bytes_per_ct;
            s->reserved += need;
            s->peak_reserved = std::max(s->peak_reserved, s->reserved);
            lane = cl.lane;
            for (size_t i = 0; i < n; i++) {
              Request* r = s->reqs[ids[i]].get();
              r->status = 2;
              grp.push_back(r);
              s->queue.erase(std::find(s->queue.begin(), s->queue.end(), ids[i]));
            }
            s->n_batches++;
            s->batched_cts += n;
            break;
          }
          s->n_deferred++;  // the oldest request waits until running batches release memory
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    const Lane& ln = s->lanes[lane];
    const Client& cl = s->clients[grp[0]->client];
    ctl_context* c = W.ctx[lane];
    const uint32_t nb = (uint32_t)grp.size();
    u64* pin = W.pin_in[lane];
    u64* pout = W.pin_out[lane];
    for (uint32_t i = 0; i < nb; i++) memcpy(pin + (size_t)i * ln.in_words, grp[i]->in.data(), ln.in_words * 8);
    ctl_ct* in = nullptr;
    ctl_ct* out = nullptr;
    int rc = ctl_ct_import(c, (const uint64_t*)pin, nb, ln.in_level, ln.in_scale, &in);
    if (!rc) rc = ctl_model_forward(c, ln.model, cl.keys, in, &out);
    if (!rc) rc = ctl_ct_export(out, (uint64_t*)pout, (size_t)nb * ln.out_words);
    if (in) ctl_ct_destroy(in);
    if (out) ctl_ct_destroy(out);
    if (rc) cudaStreamSynchronize(c->stream);
    if (!rc)
      for (uint32_t i = 0; i < nb; i++)
        memcpy(grp[i]->out.data(), pout + (size_t)i * ln.out_words, ln.out_words * 8);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->reserved -= need;
    }
    finish(s, grp, rc);
  }
}

}  // namespace

extern "C" int ctl_server_create(ctl_server** out, uint64_t mem_budget_bytes, uint32_t n_workers, uint32_t max_batch,
                                 uint32_t max_queue) {
  if (!out || n_workers == 0 || n_workers > 32 || max_batch == 0 || max_queue == 0) {
    set_error("ctl_server_create: invalid argument");
    return CTL_EINVAL;
  }
  ctl_server* s = new (std::nothrow) ctl_server();
  if (!s) return CTL_ENOMEM;
  s->budget = mem_budget_bytes;
  s->n_workers = n_workers;
  s->max_batch = max_batch;
  s->max_queue = max_queue;
  *out = s;
  return CTL_OK;
}

extern "C" int ctl_server_add_lane(ctl_server* s, ctl_context* ctx, const ctl_model* model, uint32_t* lane) {
  if (!s || !ctx || !model || s->started) {
    set_error("ctl_server_add_lane: invalid argument or server already started");
    return CTL_EINVAL;
  }
  uint32_t out_level = 0;
  double out_scale = 0;
  ctl_model_info(model, &out_level, &out_scale, nullptr);
  Lane ln;
  ln.ctx = ctx;
  ln.model = model;
  ln.in_level = ctx->L;
  ln.out_level = out_level;
  ln.in_scale = ctx->scale;
  ln.in_words = 2ull * ln.in_level * ctx->N;
  ln.out_words = 2ull * out_level * ctx->N;
  ln.bytes_per_ct = estimate_bytes_per_ct(ctx, model, ln.in_level);
  s->lanes.push_back(ln);
  if (lane) *lane = (uint32_t)s->lanes.size() - 1;
  return CTL_OK;
}

extern "C" int ctl_server_add_client(ctl_server* s, uint32_t lane, const ctl_keys* keys, uint32_t* client) {
  if (!s || !keys || lane >= s->lanes.size()) {
    set_error("ctl_server_add_client: invalid argument");
    return CTL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->clients.push_back(Client{lane, keys});
  if (client) *client = (uint32_t)s->clients.size() - 1;
  return CTL_OK;
}

extern "C" int ctl_server_admission(ctl_server* s, uint32_t client, uint64_t* bytes_per_ct,
                                    uint64_t* peak_reserved, uint64_t* deferred) {
  if (!s || client >= s->clients.size()) {
    set_error("ctl_server_admission: unknown client");
    return CTL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes_per_ct) *bytes_per_ct = s->lanes[s->clients[client].lane].bytes_per_ct;
  if (peak_reserved) *peak_reserved = s->peak_reserved;
  if (deferred) *deferred = s->n_deferred;
  return CTL_OK;
}

extern "C" int ctl_server_io_words(const ctl_server* s, uint32_t client, size_t* in_words, size_t* out_words) {
  if (!s || client >= s->clients.size()) {
    set_error("ctl_server_io_words: unknown client");
    return CTL_EINVAL;
  }
  const Lane& ln = s->lanes[s->clients[client].lane];
  if (in_words) *in_words = ln.in_words;
  if (out_words) *out_words = ln.out_words;
  return CTL_OK;
}

extern "C" int ctl_server_start(ctl_server* s) {
  if (!s || s->started || s->lanes.empty()) {
    set_error("ctl_server_start: no lanes or already started");
    return CTL_EINVAL;
  }
  s->workers.resize(s->n_workers);
  for (auto& W : s->workers) {
    for (auto& ln : s->lanes) {
      ctl_context* cc = nullptr;
      if (int rc = ctl_context_clone(ln.ctx, &cc)) return rc;
      W.ctx.push_back(cc);
      u64 *pi = nullptr, *po = nullptr;
      if (cudaMallocHost(&pi, s->max_batch * ln.in_words * 8) != cudaSuccess ||
          cudaMallocHost(&po, s->max_batch * ln.out_words * 8) != cudaSuccess) {
        set_error("ctl_server_start: pinned host allocation failed");
        return CTL_ENOMEM;
      }
      W.pin_in.push_back(pi);
      W.pin_out.push_back(po);
    }
  }
  s->started = true;
  for (uint32_t i = 0; i < s->n_workers; i++) s->workers[i].th = std::thread(worker_loop, s, i);
  return CTL_OK;
}

extern "C" int ctl_server_submit(ctl_server* s, uint32_t client, const uint64_t* ct_coeffs, uint64_t* request) {
  if (!s || !ct_coeffs || !request || client >= s->clients.size()) {
    set_error("ctl_server_submit: invalid argument");
    return CTL_EINVAL;
  }
  const Lane& ln = s->lanes[s->clients[client].lane];
  std::unique_ptr<Request> r(new Request());
  r->client = client;
  r->in.assign(ct_coeffs, ct_coeffs + ln.in_words);
  r->out.assign(ln.out_words, 0);
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->started || s->stopping) {
    set_error("ctl_server_submit: server not running");
    return CTL_EINVAL;
  }
  if (s->queue.size() >= s->max_queue) {
    s->n_rejected++;
    set_error("ctl_server_submit: queue full (%u requests)", s->max_queue);
    return CTL_EBUSY;
  }
  r->id = s->next_id++;
  r->t_submit = Clock::now();
  *request = r->id;
  s->queue.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  s->n_submitted++;
  s->cv.notify_one();
  return CTL_OK;
}

static int take_result(ctl_server* s, uint64_t id, uint64_t* out, size_t cap, double* latency_ms) {
  auto it = s->reqs.find(id);
  Request* r = it->second.get();
  const int st = r->status;
  if (st < 0) {
    set_error("ctl_server: request %llu failed with %d", (unsigned long long)id, st);
    s->reqs.erase(it);
    return st;
  }
  if (out) {
    if (cap < r->out.size()) {
      set_error("ctl_server: capacity %zu < %zu", cap, r->out.size());
      return CTL_EINVAL;
    }
    memcpy(out, r->out.data(), r->out.size() * 8);
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  s->reqs.erase(it);
  return CTL_OK;
}

extern "C" int ctl_server_poll(ctl_server* s, uint64_t request, uint64_t* out, size_t cap, double* latency_ms) {
  if (!s) return CTL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end()) {
    set_error("ctl_server_poll: unknown request %llu", (unsigned long long)request);
    return CTL_EINVAL;
  }
  if (it->second->status > 0) return CTL_EBUSY;
  return take_result(s, request, out, cap, latency_ms);
}

extern "C" int ctl_server_wait(ctl_server* s, uint64_t request, uint32_t timeout_ms, uint64_t* out, size_t cap,
                               double* latency_ms) {
  if (!s) return CTL_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request);
  if (it == s->reqs.end()) {
    set_error("ctl_server_wait: unknown request %llu", (unsigned long long)request);
    return CTL_EINVAL;
  }
  Request* r = it->second.get();
  if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->status <= 0; })) {
    set_error("ctl_server_wait: request %llu not done after %u ms", (unsigned long long)request, timeout_ms);
    return CTL_ETIMEOUT;
  }
  return take_result(s, request, out, cap, latency_ms);
}

extern "C" int ctl_server_stats(ctl_server* s, uint64_t* counts6, double* p50_ms, double* p99_ms) {
  if (!s) return CTL_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (counts6) {
    counts6[0] = s->n_submitted;
    counts6[1] = s->n_completed;
    counts6[2] = s->n_rejected;
    counts6[3] = s->n_failed;
    counts6[4] = s->n_batches;
    counts6[5] = s->batched_cts;
  }
  std::vector<double> v = s->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  return CTL_OK;
}

extern "C" void ctl_server_destroy(ctl_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto& W : s->workers)
    if (W.th.joinable()) W.th.join();
  for (auto& W : s->workers) {
    for (auto* cc : W.ctx) ctl_context_destroy(cc);
    for (auto* p : W.pin_in) cudaFreeHost(p);
    for (auto* p : W.pin_out) cudaFreeHost(p);
  }
  delete s;
}
