// sst_load.cpp -- a native client for the served path (arXiv 2101.11489 section 3:
// events processed concurrently as they come): an open-loop Poisson stream of
// events submitted through sst_submit and collected through sst_poll, so that the
// server's capacity and latencies are measured without a scripting-language client
// in the way.  It uses only the public calls.
//
// Arrival i is due at the i-th point of a Poisson process of the offered rate
// (exponential gaps from a seeded generator; rate 0: all due at once, i.e. as fast
// as the server admits).  Submitter thread k takes the arrivals i = k mod S, waits
// for each one's due time, and submits event i mod n_events, retrying while the
// server answers BUSY or BUDGET; admitted tickets go to a queue in admission order,
// from which poller threads collect the results (waiting without a timeout).
// Latency is measured from the due time (so that queueing in the client counts)
// and, separately, from the admission, to the time the server saw the event's
// batch complete (sst_result_info).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include <sys/prctl.h>

#include "sst_internal.h"

namespace {

double now_us() {
  using namespace std::chrono;
  return duration_cast<duration<double, std::micro>>(steady_clock::now().time_since_epoch()).count();
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" sst_status sst_serve_load(sst_ctx* ctx, const uint8_t* const* raw, const uint64_t* raw_bytes,
                                     const uint32_t* const* fed_len, uint32_t n_events, uint64_t n_requests,
                                     double rate, uint32_t submitters, uint32_t pollers, uint64_t seed,
                                     double* latency_us, sst_load_result* out) {
  if (!ctx || !raw || !raw_bytes || !fed_len || !out || n_events == 0 || n_requests == 0 || !(rate >= 0.0) ||
      submitters == 0 || submitters > 64 || pollers == 0 || pollers > 16)
    return SST_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < n_events; i++)
    if (!raw[i] || !fed_len[i]) return SST_ERR_INVALID_ARG;
  // due times of the arrivals, relative to the start
  std::vector<double> due(n_requests, 0.0);
  if (rate > 0) {
    std::mt19937_64 gen(seed);
    std::exponential_distribution<double> gap(rate / 1e6);  // per microsecond
    double t = 0;
    for (uint64_t i = 0; i < n_requests; i++) {
      t += gap(gen);
      due[i] = t;
    }
  }
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::pair<uint64_t, uint64_t>> admitted;  // (ticket, arrival)
  uint64_t n_admitted = 0;
  std::atomic<uint64_t> retries{0};
  std::atomic<int> failed{0};  // first failing status, 0: none
  std::vector<double> lat_due(n_requests, 0.0), lat_adm(n_requests, 0.0);
  std::atomic<uint64_t> done{0};
  double t_last = 0;
  const double t0 = now_us() + 1000.0;  // every thread is running before the first arrival
  auto fail = [&](sst_status code) {
    int z = 0;
    failed.compare_exchange_strong(z, code);
    cv.notify_all();
  };
  auto submitter = [&](uint32_t k) {
    // sleep precisely (1 us timer slack instead of the default 50 us), so that a
    // submitter wakes just before its next arrival and spins only briefly: at
    // high rates spinning submitters would otherwise take the cores the server's
    // loop thread and the pollers need
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
    for (uint64_t i = k; i < n_requests && !failed.load(); i += submitters) {
      const double when = t0 + due[i];
      for (double now = now_us(); now < when; now = now_us()) {
        if (when - now > 40.0) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)(when - now - 20.0)));
      }
      const uint32_t e = (uint32_t)(i % n_events);
      uint64_t tk = 0;
      const double t_try = now_us();
      for (;;) {
        const sst_status r = sst_submit(ctx, raw[e], raw_bytes[e], fed_len[e], &tk);
        if (r == SST_OK) break;
        if (r != SST_ERR_BUSY && r != SST_ERR_BUDGET) {
          fail(r);
          return;
        }
        if (now_us() - t_try > 60e6) {  // refused for a minute: the server makes no progress
          fail(SST_ERR_TIMEOUT);
          return;
        }
        retries++;
        // the server is full: back off instead of contending for its lock
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
      {
        std::lock_guard<std::mutex> g(mu);
        admitted.emplace_back(tk, i);
        n_admitted++;
      }
      cv.notify_one();
    }
  };
  auto poller = [&]() {
    for (;;) {
      std::pair<uint64_t, uint64_t> a;
      {
        std::unique_lock<std::mutex> g(mu);
        cv.wait(g, [&] { return !admitted.empty() || failed.load() || n_admitted >= n_requests; });
        if (admitted.empty()) return;  // everything admitted was collected (or a failure)
        a = admitted.front();
        admitted.pop_front();
      }
      sst_result_info info{};
      const sst_status r = sst_poll(ctx, a.first, -1, &info, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
      if (r != SST_OK) {
        fail(r);
        return;
      }
      lat_due[a.second] = info.t_done_us - (t0 + due[a.second]);
      lat_adm[a.second] = info.t_done_us - info.t_submit_us;
      {
        std::lock_guard<std::mutex> g(mu);
        if (info.t_done_us > t_last) t_last = info.t_done_us;
      }
      if (++done == n_requests) cv.notify_all();
    }
  };
  std::vector<std::thread> th;
  for (uint32_t k = 0; k < submitters; k++) th.emplace_back(submitter, k);
  std::vector<std::thread> po;
  for (uint32_t k = 0; k < pollers; k++) po.emplace_back(poller);
  for (auto& t : th) t.join();
  cv.notify_all();
  for (auto& t : po) t.join();
  if (failed.load()) return (sst_status)failed.load();
  if (done.load() != n_requests) return SST_ERR_STATE;
  out->offered_rate = rate;
  out->requests = n_requests;
  out->retries = retries.load();
  const double span = t_last - t0;
  out->throughput = span > 0 ? (double)n_requests / (span * 1e-6) : 0.0;
  out->p50_us = percentile(lat_due, 0.50);
  out->p99_us = percentile(lat_due, 0.99);
  out->max_us = *std::max_element(lat_due.begin(), lat_due.end());
  double sum = 0;
  for (double v : lat_due) sum += v;
  out->mean_us = sum / (double)n_requests;
  out->p50_admitted_us = percentile(lat_adm, 0.50);
  out->p99_admitted_us = percentile(lat_adm, 0.99);
  if (latency_us) std::copy(lat_due.begin(), lat_due.end(), latency_us);
  return SST_OK;
}
