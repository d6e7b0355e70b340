// Open-loop load generator for the serving loop (ccm_serve_replay): submits
// requests at their arrival times and drains completions, on one host thread,
// through the public ccm_submit / ccm_poll_completed calls only.
#include <chrono>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ccm_host.h"

using namespace ccm;

ccm_status ccm_serve_replay(ccm_ctx ctx, const ccm_request* reqs, const double* arrival_s,
                            int64_t n, double* lag_s, double* latency_s, double* elapsed_s) {
  if (!ctx || (n > 0 && (!reqs || !arrival_s)) || n < 0)
    return fail(CCM_ERR_INVALID, "NULL context, requests or arrival times");
  for (int64_t k = 1; k < n; ++k)
    if (arrival_s[k] < arrival_s[k - 1]) return fail(CCM_ERR_INVALID, "arrivals must not decrease");
  using clock = std::chrono::steady_clock;
  const clock::time_point t0 = clock::now();
  auto since = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
  std::vector<double> lag(n, 0.0);
  std::unordered_map<ccm_ticket, int64_t> index;
  index.reserve((size_t)n);
  const int64_t cap = 4096;
  std::vector<ccm_ticket> done_t(cap);
  std::vector<double> done_l(cap);
  int64_t k = 0, n_done = 0;
  ccm_status err = CCM_OK;
  while (n_done < k || (k < n && err == CCM_OK)) {
    bool progress = false;
    const double now = since();
    while (err == CCM_OK && k < n && arrival_s[k] <= now) {
      ccm_ticket tk = 0;
      const ccm_status s = ccm_submit(ctx, &reqs[k], &tk);
      if (s == CCM_ERR_BUSY) break;   // queue full: drain first
      if (s != CCM_OK) {
        err = s;
        break;
      }
      lag[k] = since() - arrival_s[k];
      index.emplace(tk, k);
      ++k;
      progress = true;
    }
    int64_t m = 0;
    const ccm_status s = ccm_poll_completed(ctx, done_t.data(), done_l.data(), cap, &m);
    if (s != CCM_OK) return s;
    for (int64_t j = 0; j < m; ++j) {
      auto it = index.find(done_t[j]);
      if (it == index.end()) continue;   // retired elsewhere
      if (latency_s) latency_s[it->second] = lag[it->second] + done_l[j];
      index.erase(it);
      ++n_done;
      progress = true;
    }
    if (!progress) std::this_thread::yield();
  }
  if (lag_s)
    for (int64_t q = 0; q < n; ++q) lag_s[q] = lag[q];
  if (elapsed_s) *elapsed_s = since();
  return err;
}
