// Serving loop: continuous batching of encrypted-instruction requests from
// many clients (the paper's cloud service model, §4: clients send cleartext
// instructions over their encrypted registers; the server evaluates them).
//
// Requests enter a queue from any host thread.  A worker thread keeps the
// engine's tick loop running: every tick it first starts queued requests
// (one in flight per client, so each client's requests run in order), then
// runs one level of every in-flight instruction of every client in one
// batched launch, and retires instructions that reached their last level.
// A request that arrives while others are on the GPU joins at the next
// tick; its work overlaps theirs on the device.  A request is complete when
// the CUDA event recorded after its last tick has completed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ce_internal.h"
#include "ctx.h"
#include "launch.h"
#include "netlist.h"

namespace ce {

// Engine hooks (engine.cu).
struct EngineRunHooks;
ce_status engine_serve_tick(ce_ctx *ctx, cudaStream_t st, const std::vector<int> &start_clients,
                            const std::vector<ce_insn> &start_insns, std::vector<int> &retired,
                            int *active_after, int *bootstraps);

}  // namespace ce

using namespace ce;

namespace {

uint64_t now_ns() {
  return uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(
                      std::chrono::steady_clock::now().time_since_epoch())
                      .count());
}

struct Ticket {
  int client = 0;
  ce_insn insn{};
  uint64_t submit_ns = 0, start_ns = 0, done_ns = 0;
  int state = 0;  // 0 queued, 1 running, 2 retired (waiting for its event), 3 done, <0 error
  ce_status status = CE_OK;
};

}  // namespace

struct ce_server {
  ce_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  int max_inflight = 0;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::map<uint64_t, Ticket> tickets;
  std::deque<uint64_t> queue;             // submitted, not started
  std::map<int, uint64_t> running;        // client -> ticket in flight
  std::deque<std::pair<cudaEvent_t, std::vector<uint64_t>>> pending;  // retired, awaiting GPU
  std::deque<cudaEvent_t> ticks_in_flight;  // one event per enqueued tick, oldest first
  std::vector<cudaEvent_t> ev_free;
  uint64_t next_ticket = 1;
  bool stop = false;
  ce_status fatal = CE_OK;
  std::thread worker;
  uint64_t ticks = 0, bootstraps = 0;
};

namespace {

cudaEvent_t take_ev(ce_server *s) {
  if (!s->ev_free.empty()) {
    cudaEvent_t e = s->ev_free.back();
    s->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

// Marks retired tickets done once their GPU work has finished.
void reap(ce_server *s, bool block) {
  while (!s->pending.empty()) {
    auto &front = s->pending.front();
    cudaError_t q = block ? cudaEventSynchronize(front.first) : cudaEventQuery(front.first);
    if (q == cudaErrorNotReady) return;
    const uint64_t t = now_ns();
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (uint64_t id : front.second) {
        Ticket &tk = s->tickets[id];
        tk.done_ns = t;
        tk.state = q == cudaSuccess ? 3 : -1;
        if (q != cudaSuccess) tk.status = CE_ECUDA;
      }
    }
    s->done_cv.notify_all();
    s->ev_free.push_back(front.first);
    s->pending.pop_front();
  }
}

void serve_loop(ce_server *s) {
  cudaSetDevice(s->ctx->device);
  for (;;) {
    std::vector<int> start_clients;
    std::vector<ce_insn> start_insns;
    std::vector<uint64_t> start_ids;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->queue.empty() && s->running.empty()) {
        if (s->stop && s->pending.empty()) return;
        if (s->pending.empty())
          s->cv.wait_for(lock, std::chrono::milliseconds(2),
                         [&] { return s->stop || !s->queue.empty(); });
      }
      // start queued requests of clients with nothing in flight (in order)
      std::map<int, bool> busy;
      for (auto &r : s->running) busy[r.first] = true;
      for (auto it = s->queue.begin(); it != s->queue.end();) {
        if (int(s->running.size()) >= s->max_inflight) break;
        Ticket &tk = s->tickets[*it];
        if (busy.count(tk.client)) {
          ++it;
          continue;
        }
        busy[tk.client] = true;
        s->running[tk.client] = *it;
        tk.state = 1;
        tk.start_ns = now_ns();
        start_clients.push_back(tk.client);
        start_insns.push_back(tk.insn);
        start_ids.push_back(*it);
        it = s->queue.erase(it);
      }
    }
    std::vector<int> retired;
    int active = 0, boots = 0;
    const bool work = !start_clients.empty() || [&] {
      std::lock_guard<std::mutex> lock(s->mu);
      return !s->running.empty();
    }();
    if (work) {
      // At most two ticks in flight on the GPU: wait for older ones here,
      // outside the context lock, so that other calls on the context get
      // their turn between ticks instead of waiting for the whole queue.
      while (s->ticks_in_flight.size() >= 2) {
        cudaEventSynchronize(s->ticks_in_flight.front());
        s->ev_free.push_back(s->ticks_in_flight.front());
        s->ticks_in_flight.pop_front();
      }
      ce_status st = engine_serve_tick(s->ctx, s->stream, start_clients, start_insns, retired,
                                       &active, &boots);
      if (st != CE_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->fatal = st;
        for (auto &r : s->running) {
          s->tickets[r.second].state = -1;
          s->tickets[r.second].status = st;
        }
        s->running.clear();
        s->done_cv.notify_all();
        continue;
      }
      ++s->ticks;
      s->bootstraps += uint64_t(boots);
      cudaEvent_t te = take_ev(s);
      cudaEventRecord(te, s->stream);
      s->ticks_in_flight.push_back(te);
      if (!retired.empty()) {
        std::vector<uint64_t> ids;
        {
          std::lock_guard<std::mutex> lock(s->mu);
          for (int c : retired) {
            auto it = s->running.find(c);
            if (it == s->running.end()) continue;
            s->tickets[it->second].state = 2;
            ids.push_back(it->second);
            s->running.erase(it);
          }
        }
        cudaEvent_t e = take_ev(s);
        cudaEventRecord(e, s->stream);
        s->pending.emplace_back(e, std::move(ids));
      }
    }
    reap(s, false);
  }
}

}  // namespace

namespace ce {

bool server_client_busy(ce_server *s, int client) {
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->running.count(client)) return true;
  for (uint64_t id : s->queue)
    if (s->tickets[id].client == client) return true;
  return false;
}

}  // namespace ce

extern "C" ce_status ce_server_create(ce_ctx *ctx, int max_inflight, ce_server **out) {
  if (!ctx || !out) return set_error(CE_EINVAL, "ce_server_create: bad argument");
  ce_server *s = new ce_server();
  s->ctx = ctx;
  s->max_inflight = max_inflight > 0 ? max_inflight : 1 << 20;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return cuda_error(e, "ce_server_create");
  }
  {
    std::lock_guard<std::recursive_mutex> lock(ctx->mu);
    ctx->servers.push_back(s);
  }
  s->worker = std::thread(serve_loop, s);
  *out = s;
  return CE_OK;
}

extern "C" ce_status ce_server_submit(ce_server *s, int client, const ce_insn *insn,
                                      uint64_t *ticket) {
  if (!s || !insn || !ticket) return set_error(CE_EINVAL, "ce_server_submit: bad argument");
  if (insn->op > CE_I_UMULH || insn->rd > 7 || insn->rn > 7 || insn->rm > 7 || insn->cond > 13)
    return set_error(CE_EINVAL, "ce_server_submit: malformed instruction");
  // the client stays admitted while its ticket is queued: eviction checks
  // the queue under the same lock
  std::lock_guard<std::mutex> cl_lock(s->ctx->clients_mu);
  if (client < 0 || client >= int(s->ctx->clients.size()) || !s->ctx->clients[client].live)
    return set_error(CE_ENOTFOUND, "ce_server_submit: unknown client");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fatal != CE_OK) return set_error(s->fatal, "ce_server_submit: server failed");
    const uint64_t id = s->next_ticket++;
    Ticket tk;
    tk.client = client;
    tk.insn = *insn;
    tk.submit_ns = now_ns();
    s->tickets[id] = tk;
    s->queue.push_back(id);
    *ticket = id;
  }
  s->cv.notify_one();
  return CE_OK;
}

extern "C" ce_status ce_server_poll(ce_server *s, uint64_t ticket, int *done, uint64_t *submit_ns,
                                    uint64_t *start_ns, uint64_t *done_ns) {
  if (!s || !done) return set_error(CE_EINVAL, "ce_server_poll: bad argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return set_error(CE_ENOTFOUND, "ce_server_poll: unknown ticket");
  const Ticket &tk = it->second;
  if (tk.state < 0) return set_error(tk.status, "ce_server_poll: request failed");
  *done = tk.state == 3;
  if (submit_ns) *submit_ns = tk.submit_ns;
  if (start_ns) *start_ns = tk.start_ns;
  if (done_ns) *done_ns = tk.done_ns;
  return CE_OK;
}

extern "C" ce_status ce_server_wait(ce_server *s, uint64_t ticket, uint64_t timeout_ns) {
  if (!s) return set_error(CE_EINVAL, "ce_server_wait: null server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return set_error(CE_ENOTFOUND, "ce_server_wait: unknown ticket");
  auto pred = [&] { return it->second.state == 3 || it->second.state < 0; };
  if (timeout_ns) {
    if (!s->done_cv.wait_for(lock, std::chrono::nanoseconds(timeout_ns), pred))
      return set_error(CE_ETIMEOUT, "ce_server_wait: timeout");
  } else {
    s->done_cv.wait(lock, pred);
  }
  return it->second.state < 0 ? set_error(it->second.status, "ce_server_wait: request failed")
                              : CE_OK;
}

extern "C" ce_status ce_server_stats(ce_server *s, uint64_t *ticks, uint64_t *bootstraps,
                                     uint64_t *queued, uint64_t *running) {
  if (!s) return set_error(CE_EINVAL, "ce_server_stats: null server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (ticks) *ticks = s->ticks;
  if (bootstraps) *bootstraps = s->bootstraps;
  if (queued) *queued = s->queue.size();
  if (running) *running = s->running.size();
  return CE_OK;
}

extern "C" void ce_server_destroy(ce_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  reap(s, true);
  cudaStreamSynchronize(s->stream);
  for (auto e : s->ticks_in_flight) s->ev_free.push_back(e);
  s->ticks_in_flight.clear();
  {
    std::lock_guard<std::recursive_mutex> lock(s->ctx->mu);
    auto &v = s->ctx->servers;
    v.erase(std::remove(v.begin(), v.end(), s), v.end());
  }
  for (auto e : s->ev_free) cudaEventDestroy(e);
  cudaStreamDestroy(s->stream);
  delete s;
}
