// Continuous-batching serving loop for Q-less QR and least-squares requests.
//
// Requests reference device-resident matrices owned by the caller.  A scheduler thread
// admits queued requests (FIFO) while the in-flight request count stays within max_slots
// and the HBM budget covers the request's data plus the server's own device buffers
// (outputs and batch workspace, carved from one arena allocated at creation), and launches
// every admitted group as ONE batched persistent kernel (ql_batch_launch) on an idle one
// of its CUDA streams: each stream runs one group at a time, so requests that arrive while
// groups run coalesce into the next group, and the groups of different streams overlap on
// the device.  Groups complete when their events fire; one device-to-host copy per group
// returns all statuses.  Plans are uploaded through a pinned staging ring, so the
// scheduler never blocks on the device.  Latency is measured from submit to the scheduler
// observing the group's completion event.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

namespace ql {

using Clock = std::chrono::steady_clock;
static double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// First-fit allocator over [0, size) with coalescing frees (offsets aligned to 256 B).
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        size_t rem = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rem) free_[start] = rem;
        used_ += bytes;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
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
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

struct Req {
  ql_request r;
  double t_submit = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 in flight, 2 done
  size_t out_off = 0, out_bytes = 0, data_bytes = 0;
  int32_t* info_host = nullptr;
  ql_status status = QL_OK;
  int32_t index = 0;
};

struct Group {
  std::vector<uint64_t> tickets;
  cudaEvent_t ev = nullptr;
  int stream = 0;
  size_t ws_off = 0, ws_bytes = 0, pin_off = 0, pin_bytes = 0;
  size_t data_bytes = 0;
  double t_launch = 0;
};

// QL_SERVER_TRACE=1 prints one line per completed group (size, launch -> completion time).
static bool trace_on() {
  static const bool on = [] {
    const char* v = std::getenv("QL_SERVER_TRACE");
    return v && v[0] == '1';
  }();
  return on;
}

}  // namespace ql

struct ql_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;  // one group in flight per stream
  unsigned char* dev_base = nullptr;
  ql::Arena dev;
  unsigned char* pin_base = nullptr;
  ql::Arena pin;
  size_t data_in_flight = 0, peak_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, ql::Req> reqs;
  std::vector<ql::Group> inflight;
  int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0, inflight_reqs = 0;
  std::vector<double> latencies;
  double t_first = 0, t_last = 0;
};

namespace ql {

static size_t out_bytes_of(const ql_request& r) {
  int64_t n1 = r.n + 1;
  return (size_t)(n1 * n1 + n1 + 1) * sizeof(double) + 64;  // R (or R_ext), x + residual, info
}
static size_t data_bytes_of(const ql_request& r) {
  return (size_t)r.m * r.n * (r.dtype == QL_F64 ? 8 : 4) + (r.kind == 1 ? (size_t)r.m * (r.dtype == QL_F64 ? 8 : 4) : 0);
}

static void complete_groups(ql_server* s) {
  for (size_t g = 0; g < s->inflight.size();) {
    Group& G = s->inflight[g];
    if (cudaEventQuery(G.ev) != cudaSuccess) {
      ++g;
      continue;
    }
    double t = now_s();
    if (trace_on())
      std::fprintf(stderr, "[ql_server] group of %zu on stream %d: %.3f ms, %.1f MB data\n", G.tickets.size(),
                   G.stream, (t - G.t_launch) * 1e3, G.data_bytes / 1e6);
    for (uint64_t tk : G.tickets) {
      Req& q = s->reqs[tk];
      q.state = 2;
      q.t_done = t;
      q.status = q.info_host[0];
      q.index = q.info_host[1];
      s->latencies.push_back((t - q.t_submit) * 1e3);
      s->completed++;
      s->inflight_reqs--;
      s->t_last = t;
    }
    s->dev.release(G.ws_off, G.ws_bytes);
    s->pin.release(G.pin_off, G.pin_bytes);
    s->data_in_flight -= G.data_bytes;
    s->stream_busy[G.stream] = 0;
    cudaEventDestroy(G.ev);
    s->inflight.erase(s->inflight.begin() + g);
  }
}

// Admit queued requests into one group and launch it; returns whether a group started.
static bool admit_and_launch(ql_server* s) {
  if (s->queue.empty()) return false;
  // a group starts only on an idle stream: requests that arrive meanwhile coalesce into the
  // next, larger group (continuous batching across the streams)
  int sidx = -1;
  for (int i = 0; i < (int)s->streams.size(); ++i)
    if (!s->stream_busy[i]) {
      sidx = i;
      break;
    }
  if (sidx < 0) return false;
  std::vector<uint64_t> group;
  size_t data = 0;
  while (!s->queue.empty() && s->inflight_reqs + (int64_t)group.size() < s->max_slots) {
    uint64_t tk = s->queue.front();
    Req& q = s->reqs[tk];
    size_t off;
    if (s->dev.used() + s->data_in_flight + data + q.data_bytes + q.out_bytes > s->budget) break;
    if (!s->dev.alloc(q.out_bytes, &off)) break;
    q.out_off = off;
    data += q.data_bytes;
    group.push_back(tk);
    s->queue.pop_front();
  }
  if (group.empty()) return false;
  std::vector<ql_problem> probs(group.size());
  for (size_t i = 0; i < group.size(); ++i) {
    Req& q = s->reqs[group[i]];
    int64_t n1 = q.r.n + 1;
    double* base = reinterpret_cast<double*>(s->dev_base + q.out_off);
    ql_problem& p = probs[i];
    p.m = q.r.m;
    p.n = q.r.n;
    p.ld = q.r.ld;
    p.X = q.r.X;
    p.dtype = q.r.dtype;
    p.kind = q.r.kind;
    p.b = q.r.b;
    p.R = base;
    p.x = base + n1 * n1;
    p.info = nullptr;  // set below: one status array per group
    p.method_hint = q.r.method_hint;
    p.kappa_hint = q.r.kappa_hint;
  }
  // The group's workspace (R-trees) must fit next to its data and outputs: drop requests
  // from the tail (back to the front of the queue, in order) until it does.
  Group G;
  size_t wsb = 0, upb = 0, infob = 0;
  for (;;) {
    infob = (probs.size() * 2 * sizeof(int32_t) + 255) / 256 * 256;
    for (auto& p : probs) p.info = reinterpret_cast<int32_t*>(s->dev_base);  // placeholder for sizing
    wsb = ql_batch_workspace_bytes((int32_t)probs.size(), probs.data());
    upb = batch_plan_upload_bytes((int32_t)probs.size(), probs.data());
    bool fits = wsb > 0 && s->dev.used() + s->data_in_flight + data + wsb + infob <= s->budget &&
                s->dev.alloc(wsb + infob, &G.ws_off);
    if (fits && s->pin.alloc(upb + infob + 256, &G.pin_off)) break;
    if (fits) s->dev.release(G.ws_off, wsb + infob);
    Req& q = s->reqs[group.back()];
    s->dev.release(q.out_off, q.out_bytes);
    data -= q.data_bytes;
    s->queue.push_front(group.back());
    group.pop_back();
    probs.pop_back();
    if (group.empty()) return false;
  }
  int32_t* info_dev = reinterpret_cast<int32_t*>(s->dev_base + G.ws_off + wsb);
  for (size_t i = 0; i < probs.size(); ++i) probs[i].info = info_dev + 2 * i;
  G.ws_bytes = wsb + infob;
  G.pin_bytes = upb + infob + 256;
  G.data_bytes = data;
  G.tickets = group;
  G.stream = sidx;
  cudaStream_t st = s->streams[sidx];
  s->stream_busy[sidx] = 1;
  unsigned char* pin = s->pin_base + G.pin_off;
  int32_t* info_host = reinterpret_cast<int32_t*>(pin + (upb + 255) / 256 * 256);
  ql_status st1 = batch_prepare_async((int32_t)probs.size(), probs.data(), s->dev_base + G.ws_off, wsb, st, pin, upb);
  ql_status st2 = st1 == QL_OK ? ql_batch_launch(s->dev_base + G.ws_off, st) : st1;
  if (st2 == QL_OK)
    cudaMemcpyAsync(info_host, info_dev, probs.size() * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  for (size_t i = 0; i < group.size(); ++i) {
    Req& q = s->reqs[group[i]];
    q.state = 1;
    q.info_host = info_host + 2 * i;
    if (st2 != QL_OK) q.info_host[0] = st2, q.info_host[1] = 0;
  }
  G.t_launch = now_s();
  cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming);
  cudaEventRecord(G.ev, st);
  s->inflight_reqs += (int64_t)group.size();
  s->data_in_flight += data;
  s->peak_bytes = std::max(s->peak_bytes, s->dev.used() + s->data_in_flight);
  s->inflight.push_back(G);
  return true;
}

static void worker_main(ql_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    complete_groups(s);
    bool launched = admit_and_launch(s);
    if (!launched) s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 500 : 50));
  }
}

}  // namespace ql

using namespace ql;

extern "C" {

ql_server* ql_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t streams) {
  if (hbm_budget_bytes < (1u << 20) || max_slots < 1 || streams < 1) return nullptr;
  ql_server* s = new ql_server();
  cudaGetDevice(&s->device);
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  // the server's own buffers: at most a quarter of the budget (the rest is request data)
  size_t arena = std::max<size_t>(hbm_budget_bytes / 4, 64u << 20);
  if (cudaMalloc(&s->dev_base, arena) != cudaSuccess) {
    delete s;
    return nullptr;
  }
  s->dev.init(arena);
  size_t pin = 64u << 20;
  if (cudaHostAlloc(&s->pin_base, pin, cudaHostAllocDefault) != cudaSuccess) {
    cudaFree(s->dev_base);
    delete s;
    return nullptr;
  }
  s->pin.init(pin);
  for (int i = 0; i < streams; ++i) {
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->streams.push_back(st);
    s->stream_busy.push_back(0);
  }
  s->worker = std::thread(worker_main, s);
  return s;
}

ql_status ql_server_submit(ql_server* s, const ql_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return QL_ERR_ARG;
  const ql_request& r = *req;
  if (r.m < 0 || r.n < 1 || r.n > (r.kind == 1 ? 63 : 64) || r.ld < (r.m > 1 ? r.m : 1) ||
      (r.dtype != QL_F64 && r.dtype != QL_F32) || (r.m > 0 && !r.X) || (r.kind == 1 && !r.b))
    return QL_ERR_ARG;
  Req q;
  q.r = r;
  q.out_bytes = out_bytes_of(r);
  q.data_bytes = data_bytes_of(r);
  std::lock_guard<std::mutex> lk(s->mu);
  if (q.out_bytes + q.data_bytes + (64u << 20) > s->budget) {
    s->rejected++;
    return QL_ERR_BUDGET;
  }
  q.t_submit = now_s();
  if (s->submitted == 0) s->t_first = q.t_submit;
  uint64_t tk = s->next_ticket++;
  s->reqs.emplace(tk, q);
  s->queue.push_back(tk);
  s->submitted++;
  *ticket = tk;
  s->cv.notify_one();
  return QL_OK;
}

ql_status ql_server_poll(ql_server* s, uint64_t ticket, ql_result* out) {
  if (!s || !out) return QL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return QL_ERR_UNKNOWN;
  Req& q = it->second;
  if (q.state != 2) return QL_ERR_BUSY;
  int64_t n1 = q.r.n + 1;
  double* base = reinterpret_cast<double*>(s->dev_base + q.out_off);
  out->status = q.status;
  out->index = q.index;
  out->latency_ms = (q.t_done - q.t_submit) * 1e3;
  out->R = base;
  out->x = q.r.kind == 1 ? base + n1 * n1 : nullptr;
  return QL_OK;
}

ql_status ql_server_release(ql_server* s, uint64_t ticket) {
  if (!s) return QL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return QL_ERR_UNKNOWN;
  if (it->second.state != 2) return QL_ERR_BUSY;
  s->dev.release(it->second.out_off, it->second.out_bytes);
  s->reqs.erase(it);
  s->cv.notify_one();
  return QL_OK;
}

ql_status ql_server_cancel(ql_server* s, uint64_t ticket) {
  if (!s) return QL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return QL_ERR_UNKNOWN;
  if (it->second.state != 0) return QL_ERR_BUSY;  // launched (or done): it completes normally
  auto qi = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (qi != s->queue.end()) s->queue.erase(qi);
  s->reqs.erase(it);
  s->cancelled++;
  s->cv.notify_one();
  return QL_OK;
}

ql_status ql_server_drain(ql_server* s, double timeout_s) {
  if (!s) return QL_ERR_ARG;
  double t0 = now_s();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->queue.empty() && s->inflight.empty()) return QL_OK;
    }
    if (now_s() - t0 > timeout_s) return QL_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

ql_status ql_server_stats(ql_server* s, ql_stats* out) {
  if (!s || !out) return QL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->in_flight = s->inflight_reqs;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  out->mean_ms = l.empty() ? 0.0 : sum / l.size();
  double span = s->t_last - s->t_first;
  out->solves_per_s = span > 0 ? s->completed / span : 0.0;
  out->hbm_in_use_bytes = (double)(s->dev.used() + s->data_in_flight);
  out->hbm_peak_bytes = (double)s->peak_bytes;
  return QL_OK;
}

void ql_server_destroy(ql_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_one();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& G : s->inflight) {
    cudaEventSynchronize(G.ev);
    cudaEventDestroy(G.ev);
  }
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(s->dev_base);
  cudaFreeHost(s->pin_base);
  delete s;
}

}  // extern "C"
