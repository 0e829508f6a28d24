// Serving loop of libmbt: instability-scan requests tracked with continuous
// batching (host code; the device work is the batched push/post kernels).
//
// A server thread owns all device work.  Requests wait in a FIFO queue and
// are admitted, in order, while the number of active requests and the device
// memory they hold stay within the configured limits.  All active requests
// advance together, turns_per_step turns at a time (fewer when a request is
// about to finish), through one batched push and one batched post launch per
// turn; the batch is rebuilt only when its membership changes.  After every
// step the server reads each request's per-turn moments, keeps their summary
// (rms over bunches of the bunch centroids, per turn) and retires requests
// that reached their turn count, which frees their memory for the queue.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mbt.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  mbt_request spec{};
  std::vector<double> Rs, fr, Q;
  std::vector<int32_t> range, bucket;
  std::vector<double> current;
  std::vector<int64_t> nmp;
  int state = MBT_REQ_QUEUED;
  mbt_ctx *ctx = nullptr;
  int64_t done_turns = 0;
  int64_t bytes = 0;
  double t_submit = 0, t_start = 0, t_finish = 0;
  std::vector<double> history;   // [turns][2]
  std::vector<double> final_moments;   // [nb][6]
  std::string error;
};

}  // namespace

struct mbt_server {
  mbt_server_config cfg{};
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  bool stop = false;
  int64_t used_bytes = 0;
  mbt_server_stats stats{};
  std::thread worker;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device bytes a request will hold once admitted, for admission: the
// context's buffers (particles, histograms, wake, phasor and scan state,
// record ring of turns_per_step turns, tables) plus a margin for its own
// launch plan.  The accounting afterwards uses the context's own figure.
int64_t estimate_bytes(const mbt_request &r, int turns_per_step) {
  const bool mixed = r.precision == MBT_PREC_MIXED;
  int64_t n_alloc = 4;
  for (int m = 0; m < r.nb; ++m) n_alloc += (r.n_mp[m] + 3) / 4 * 4;
  int nlong = 0;
  for (int i = 0; i < r.nres; ++i) nlong += (r.range[i] & MBT_RANGE_LONG) ? 1 : 0;
  const int64_t nl = std::max(1, nlong), nb = r.nb, nbins = r.nbins, ntb = (nb + 31) / 32;
  int64_t toep = nbins * 8;
  if (mixed) {
    toep = 0;
    for (int64_t mt = 0; mt < nbins / 128; ++mt) toep += 512 * std::min<int64_t>(nbins, 128 * (mt + 1));
  }
  const int64_t bytes = n_alloc * (mixed ? 12 : 16) + 2 * nb * nbins * 4 + nb * nbins * (mixed ? 4 : 8) +
                        nl * nb * 32 + nl * ntb * 48 + nl * 16 + (int64_t)turns_per_step * nb * 48 + 16 + nb * 28 +
                        nbins * 4 + nl * nb * 16 + nl * nbins * 24 + toep;
  const int64_t tiles = n_alloc / 64 + 2 * nb + 16;
  return bytes + tiles * 96 + (64 << 10);
}

mbt_status make_ctx(Request &q, int record_turns) {
  const mbt_request &r = q.spec;
  mbt_ctx *c = nullptr;
  mbt_status st = mbt_create(&r.ring, r.precision, r.flags, r.seed, &c);
  if (st != MBT_OK) return st;
  for (int i = 0; i < r.nres && st == MBT_OK; ++i) st = mbt_add_resonator(c, q.Rs[i], q.fr[i], q.Q[i], q.range[i]);
  if (st == MBT_OK) st = mbt_set_grid(c, r.nbins, r.half_width_sigmas);
  if (st == MBT_OK) st = mbt_set_record(c, record_turns);
  if (st == MBT_OK) st = mbt_set_fill(c, r.nb, q.bucket.data(), q.current.data(), q.nmp.data());
  if (st == MBT_OK) st = mbt_init_particles(c, nullptr);
  if (st != MBT_OK) {
    q.error = mbt_last_error(c);
    mbt_destroy(c);
    return st;
  }
  mbt_info info;
  mbt_get_info(c, &info);
  q.bytes = info.device_bytes;
  q.ctx = c;
  return MBT_OK;
}

void serve_loop(mbt_server *S) {
  cudaSetDevice(S->device);
  // The batch is keyed by request ids, which are never reused (a context's
  // host address can be, once an earlier one has been destroyed), and it is
  // destroyed before any of its member contexts is.
  mbt_batch *batch = nullptr;
  std::vector<int64_t> batch_ids;
  std::vector<double> rec;
  auto drop_batch = [&] {
    if (batch) mbt_batch_destroy(batch);
    batch = nullptr;
    batch_ids.clear();
  };
  for (;;) {
    // admission (FIFO, no overtaking)
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (!S->stop && S->queue.empty() && S->active.empty()) S->cv.wait(lk);
      if (S->stop) break;
      while (!S->queue.empty() && (int)S->active.size() < S->cfg.max_active) {
        std::shared_ptr<Request> q = S->queue.front();
        const int64_t need = estimate_bytes(q->spec, S->cfg.turns_per_step);
        if (!S->active.empty() && S->used_bytes + need > (int64_t)S->cfg.hbm_budget_bytes) break;
        S->queue.pop_front();
        lk.unlock();
        const mbt_status st = make_ctx(*q, S->cfg.turns_per_step);
        lk.lock();
        if (st != MBT_OK) {
          q->state = MBT_REQ_FAILED;
          if (q->error.empty()) q->error = mbt_status_string(st);
          q->t_finish = S->now();
          S->stats.failed += 1;
          S->done_cv.notify_all();
          continue;
        }
        q->state = MBT_REQ_RUNNING;
        q->t_start = S->now();
        S->used_bytes += q->bytes;
        S->active.push_back(q);
      }
      S->stats.max_active_seen = std::max<int64_t>(S->stats.max_active_seen, (int64_t)S->active.size());
      S->stats.max_bytes_seen = std::max<int64_t>(S->stats.max_bytes_seen, S->used_bytes);
    }
    if (S->active.empty()) continue;

    // (re)build the batch when its membership changed
    std::vector<int64_t> ids;
    for (auto &q : S->active) ids.push_back(q->id);
    if (!batch || ids != batch_ids) {
      drop_batch();
      std::vector<mbt_ctx *> members;
      for (auto &q : S->active) members.push_back(q->ctx);
      mbt_status bst = mbt_batch_create(members.data(), (int)members.size(), &batch);
      if (bst == MBT_OK && S->cfg.lanes > 1 && members.size() > 1) {
        bst = mbt_batch_set_lanes(batch, std::min<int>(S->cfg.lanes, (int)members.size()));
        if (bst != MBT_OK) mbt_batch_destroy(batch);
      }
      if (bst != MBT_OK) {
        batch = nullptr;
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &q : S->active) {
          q->state = MBT_REQ_FAILED;
          q->error = "batch creation failed";
          q->t_finish = S->now();
          mbt_destroy(q->ctx);
          q->ctx = nullptr;
          S->used_bytes -= q->bytes;
        }
        S->stats.failed += (int64_t)S->active.size();
        S->active.clear();
        S->done_cv.notify_all();
        continue;
      }
      batch_ids = ids;
    }
    int64_t step = S->cfg.turns_per_step;
    for (auto &q : S->active) step = std::min(step, q->spec.turns - q->done_turns);
    const auto tb = Clock::now();
    mbt_status st = mbt_batch_track(batch, step, nullptr);
    if (st == MBT_OK) st = mbt_batch_sync(batch);
    const double busy = std::chrono::duration<double>(Clock::now() - tb).count();

    // per-turn summaries
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.busy_seconds += busy;
    S->stats.steps += 1;
    bool retire = false;
    for (auto &q : S->active) {
      const int nb = q->spec.nb;
      if (st == MBT_OK) {
        rec.resize((size_t)step * nb * 6);
        st = mbt_read_moments(q->ctx, q->done_turns, step, rec.data());
      }
      if (st != MBT_OK) {
        q->state = MBT_REQ_FAILED;
        q->error = mbt_last_error(q->ctx);
      } else {
        for (int64_t t = 0; t < step; ++t) {
          double s2t = 0.0, s2d = 0.0;
          for (int m = 0; m < nb; ++m) {
            const double *r = rec.data() + ((size_t)t * nb + m) * 6;
            s2t += r[0] * r[0];
            s2d += r[2] * r[2];
          }
          q->history.push_back(std::sqrt(s2t / nb));
          q->history.push_back(std::sqrt(s2d / nb));
        }
        q->done_turns += step;
        int64_t np = 0;
        for (int m = 0; m < nb; ++m) np += q->nmp[m];
        S->stats.mp_turns += (double)np * (double)step;
        if (q->done_turns >= q->spec.turns) {
          q->final_moments.assign(rec.end() - (size_t)nb * 6, rec.end());
          q->state = MBT_REQ_DONE;
        }
      }
      retire = retire || q->state != MBT_REQ_RUNNING;
    }
    if (!retire) continue;

    // retirement: the batch goes first, then the finished contexts
    drop_batch();
    std::vector<std::shared_ptr<Request>> still;
    for (auto &q : S->active) {
      if (q->state == MBT_REQ_RUNNING) {
        still.push_back(q);
        continue;
      }
      q->t_finish = S->now();
      mbt_destroy(q->ctx);
      q->ctx = nullptr;
      S->used_bytes -= q->bytes;
      if (q->state == MBT_REQ_DONE) S->stats.completed += 1;
      else S->stats.failed += 1;
    }
    S->active.swap(still);
    S->done_cv.notify_all();
  }
  drop_batch();
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto &q : S->active)
    if (q->ctx) mbt_destroy(q->ctx);
}

}  // namespace

extern "C" {

mbt_status mbt_server_create(const mbt_server_config *cfg, mbt_server **out) {
  if (!cfg || !out || cfg->max_active < 1 || cfg->turns_per_step < 1 || cfg->hbm_budget_bytes == 0 ||
      cfg->lanes < 0 || cfg->lanes > 8)
    return MBT_ERR_ARG;
  mbt_server *S = new (std::nothrow) mbt_server();
  if (!S) return MBT_ERR_NOMEM;
  S->cfg = *cfg;
  S->t0 = Clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return MBT_ERR_CUDA;
  }
  S->worker = std::thread(serve_loop, S);
  *out = S;
  return MBT_OK;
}

mbt_status mbt_server_submit(mbt_server *S, const mbt_request *r, int64_t *id) {
  if (!S || !r || !id || r->nb < 1 || !r->bucket || !r->current_A || !r->n_mp || r->turns < 1 || r->nres < 0 ||
      r->nres > 8 || (r->nres > 0 && (!r->Rs_ohm || !r->fr_Hz || !r->Q || !r->range)))
    return MBT_ERR_ARG;
  auto q = std::make_shared<Request>();
  q->spec = *r;
  q->Rs.assign(r->Rs_ohm, r->Rs_ohm + r->nres);
  q->fr.assign(r->fr_Hz, r->fr_Hz + r->nres);
  q->Q.assign(r->Q, r->Q + r->nres);
  q->range.assign(r->range, r->range + r->nres);
  q->bucket.assign(r->bucket, r->bucket + r->nb);
  q->current.assign(r->current_A, r->current_A + r->nb);
  q->nmp.assign(r->n_mp, r->n_mp + r->nb);
  // the request's arrays now point at its own copies
  q->spec.Rs_ohm = q->Rs.data();
  q->spec.fr_Hz = q->fr.data();
  q->spec.Q = q->Q.data();
  q->spec.range = q->range.data();
  q->spec.bucket = q->bucket.data();
  q->spec.current_A = q->current.data();
  q->spec.n_mp = q->nmp.data();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (estimate_bytes(*r, S->cfg.turns_per_step) > (int64_t)S->cfg.hbm_budget_bytes) return MBT_ERR_BUDGET;
    q->id = S->next_id++;
    q->t_submit = S->now();
    S->queue.push_back(q);
    S->all[q->id] = q;
    S->stats.submitted += 1;
    *id = q->id;
  }
  S->cv.notify_all();
  return MBT_OK;
}

mbt_status mbt_server_poll(mbt_server *S, int64_t id, mbt_request_status *status, double *final_moments,
                           double *history) {
  if (!S || !status) return MBT_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return MBT_ERR_ARG;
  const Request &q = *it->second;
  status->state = q.state;
  status->turns_done = q.done_turns;
  status->t_submit = q.t_submit;
  status->t_start = q.t_start;
  status->t_finish = q.t_finish;
  status->device_bytes = q.bytes;
  std::snprintf(status->error, sizeof status->error, "%s", q.error.c_str());
  if (q.state == MBT_REQ_DONE) {
    if (final_moments) std::memcpy(final_moments, q.final_moments.data(), q.final_moments.size() * sizeof(double));
    if (history) std::memcpy(history, q.history.data(), q.history.size() * sizeof(double));
  }
  return MBT_OK;
}

mbt_status mbt_server_wait(mbt_server *S, int64_t id, double timeout_s) {
  if (!S) return MBT_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return MBT_ERR_ARG;
  auto q = it->second;
  const bool ok = S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return q->state == MBT_REQ_DONE || q->state == MBT_REQ_FAILED;
  });
  if (!ok) return MBT_ERR_TIMEOUT;
  return q->state == MBT_REQ_DONE ? MBT_OK : MBT_ERR_CUDA;
}

mbt_status mbt_server_get_stats(mbt_server *S, mbt_server_stats *out) {
  if (!S || !out) return MBT_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->queued = (int64_t)S->queue.size();
  out->active = (int64_t)S->active.size();
  out->used_bytes = S->used_bytes;
  out->now = S->now();
  return MBT_OK;
}

void mbt_server_destroy(mbt_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  delete S;
}

}  // extern "C"
