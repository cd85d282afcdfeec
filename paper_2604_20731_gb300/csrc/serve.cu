// Continuous-batching server for many independent hybrid-step scenarios on
// one GPU (host runtime; every computation is the context kernels).
//
// A worker thread owns the device work.  Requests wait in an arrival queue;
// between rounds the worker admits the oldest requests while the estimated
// device memory of the resident scenarios stays within the budget (and the
// resident count within its cap), creating each scenario's context on one of
// several CUDA streams and enqueuing its pretraining.  Every round enqueues
// one hybrid step of every resident scenario (streams round-robin, so the
// scenarios' kernels overlap on the device), then polls the steps' completion
// events and records each step's latency (enqueue to completion, host clock).
// A scenario that has run its steps copies its saturation and pressure to the
// request's result buffers and releases its memory, which lets the next
// arrivals in.  Results depend only on the scenario's own inputs (the kernels
// use fixed-order reductions), so a scenario gives the same result alone and
// in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/adsgb.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  ads_request_spec spec{};
  std::vector<double> K, phi, S0, theta0;
  bool has_phi = false, has_S0 = false, has_theta = false;
  size_t est = 0;
  // state
  ads_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int steps_done = 0;
  Clock::time_point t_submit, t_admit, t_done;
  std::vector<double> lat_ms;  // per step
  std::vector<double> S_out, P_out;
  hybrid_stats last{};
  ads_status status = ADS_OK;
  bool done = false;
  cudaEvent_t ev = nullptr;
  Clock::time_point t_enq;
};

}  // namespace

struct ads_server {
  ads_server_config cfg{};
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  size_t used = 0, peak_used = 0;
  int peak_active = 0;
  bool stop = false;
  std::thread worker;
  std::vector<double> lat_all;
  int64_t steps_total = 0, completed = 0, rejected = 0;
  int device = 0;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t count_nodes(const ads_params& p, int plus) {
  size_t v = 1;
  for (int i = 0; i < p.dim; ++i) v *= (size_t)(p.n + plus);
  return v;
}

void finish(ads_server* s, const std::shared_ptr<Request>& r, ads_status st) {
  if (r->ctx) {
    if (st == ADS_OK) {
      size_t nc = count_nodes(r->spec.params, 2);
      r->S_out.resize(nc);
      r->P_out.resize(nc);
      st = ads_get(r->ctx, ADS_FIELD_S, r->S_out.data(), nc);
      if (st == ADS_OK) st = ads_get(r->ctx, ADS_FIELD_P, r->P_out.data(), nc);
    }
    ads_destroy(r->ctx);
    r->ctx = nullptr;
  }
  if (r->ev) {
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= r->est;
  r->status = st;
  r->done = true;
  r->t_done = Clock::now();
  if (st == ADS_OK) {
    s->completed++;
    s->lat_all.insert(s->lat_all.end(), r->lat_ms.begin(), r->lat_ms.end());
  }
  s->cv_done.notify_all();
}

ads_status admit(ads_server* s, const std::shared_ptr<Request>& r) {
  r->stream = s->streams[s->next_stream];
  s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
  ads_status st = ads_init(&r->spec.params, &r->spec.crv, r->K.data(),
                           r->has_phi ? r->phi.data() : nullptr,
                           r->has_S0 ? r->S0.data() : nullptr, (void*)r->stream, &r->ctx);
  if (st != ADS_OK) return st;
  {
    // resident scenarios overlap on the streams: launch for total throughput
    const int conc = s->cfg.n_streams < s->cfg.max_active ? s->cfg.n_streams : s->cfg.max_active;
    st = ads_set_concurrency(r->ctx, conc);
    if (st != ADS_OK) return st;
  }
  if (r->has_theta) {
    st = crvpinn_set_theta(r->ctx, r->theta0.data());
    if (st != ADS_OK) return st;
  }
  if (r->spec.pretrain_iters > 0) {
    st = crvpinn_pretrain(r->ctx, r->spec.pretrain_iters, r->spec.pretrain_lr, nullptr);
    if (st != ADS_OK) return st;
  }
  if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) return ADS_ERR_CUDA;
  r->t_admit = Clock::now();
  return ADS_OK;
}

void worker_loop(ads_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<std::shared_ptr<Request>> to_admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty() && s->pending.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                            [&] { return s->stop || !s->pending.empty(); });
      if (s->stop) {
        // shutting down: release the resident scenarios, leave the queue
        std::vector<std::shared_ptr<Request>> act = s->active;
        s->active.clear();
        lk.unlock();
        for (auto& r : act) finish(s, r, ADS_ERR_STATE);
        return;
      }
      // admission: oldest first, within the memory budget and the resident cap
      size_t planned = s->used;
      int resident = (int)s->active.size();
      while (!s->pending.empty() && resident < s->cfg.max_active) {
        auto& r = s->pending.front();
        if (planned + r->est > s->cfg.hbm_budget && resident > 0) break;
        planned += r->est;
        resident++;
        to_admit.push_back(r);
        s->pending.pop_front();
      }
      s->used = planned;
      s->peak_used = std::max(s->peak_used, s->used);
    }
    for (auto& r : to_admit) {
      ads_status st = admit(s, r);
      if (st != ADS_OK) {
        finish(s, r, st);
        continue;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->active.push_back(r);
      s->peak_active = std::max(s->peak_active, (int)s->active.size());
    }
    std::vector<std::shared_ptr<Request>> act;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      act = s->active;
    }
    if (act.empty()) continue;
    // one round: a hybrid step of every resident scenario
    for (auto& r : act) {
      r->t_enq = Clock::now();
      ads_status st = hybrid_step(r->ctx, &r->spec.hp, nullptr);
      if (st == ADS_OK && cudaEventRecord(r->ev, r->stream) != cudaSuccess) st = ADS_ERR_CUDA;
      if (st != ADS_OK) r->status = st;
    }
    // completion polling with a deadline per round
    std::vector<bool> seen(act.size(), false);
    size_t left = act.size();
    const auto t0 = Clock::now();
    while (left > 0) {
      for (size_t i = 0; i < act.size(); ++i) {
        if (seen[i]) continue;
        auto& r = act[i];
        if (r->status != ADS_OK) {
          seen[i] = true;
          --left;
          continue;
        }
        cudaError_t e = cudaEventQuery(r->ev);
        if (e == cudaSuccess) {
          r->lat_ms.push_back(ms_between(r->t_enq, Clock::now()));
          r->steps_done++;
          seen[i] = true;
          --left;
        } else if (e != cudaErrorNotReady) {
          r->status = ADS_ERR_CUDA;
          seen[i] = true;
          --left;
        }
      }
      if (left == 0) break;
      if (ms_between(t0, Clock::now()) > 600e3) {
        for (size_t i = 0; i < act.size(); ++i)
          if (!seen[i]) act[i]->status = ADS_ERR_TIMEOUT;
        break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // retire finished or failed scenarios
    std::vector<std::shared_ptr<Request>> keep;
    for (auto& r : act) {
      if (r->status != ADS_OK) {
        finish(s, r, r->status);
      } else if (r->steps_done >= r->spec.n_steps) {
        hybrid_stats hs{};
        ads_status st = ads_sync(r->ctx, 600.0);
        if (st == ADS_OK) {
          double dt = 0, loss = 0;
          ads_get(r->ctx, ADS_FIELD_DT, &dt, 1);
          ads_get(r->ctx, ADS_FIELD_LOSS, &loss, 1);
          hs.dt_used = dt;
          hs.loss_last = loss;
          double m[3];
          ads_get(r->ctx, ADS_FIELD_MASS, m, 3);
          hs.mass_total = m[0];
          hs.mass_err = m[1];
          r->last = hs;
        }
        {
          std::lock_guard<std::mutex> lk(s->mu);
          s->steps_total += r->steps_done;
        }
        finish(s, r, st);
      } else {
        keep.push_back(r);
      }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->active = keep;
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t k = (size_t)std::min<double>((double)v.size() - 1, std::ceil(q * v.size()) - 1);
  return v[k];
}

}  // namespace

extern "C" {

ads_status ads_server_create(const ads_server_config* cfg, ads_server** out) {
  if (!cfg || !out) return ADS_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->hbm_budget == 0 || cfg->max_active < 1 || cfg->n_streams < 1 || cfg->n_streams > 64)
    return ADS_ERR_INVALID_ARG;
  ads_server* s = new ads_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  for (int i = 0; i < cfg->n_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return ADS_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return ADS_OK;
}

ads_status ads_server_submit(ads_server* s, const ads_request_spec* spec, const double* K_nodal,
                             const double* phi_nodal, const double* S0, const double* theta0,
                             int64_t* id_out) {
  if (!s || !spec || !K_nodal || !id_out) return ADS_ERR_INVALID_ARG;
  if (spec->n_steps < 0) return ADS_ERR_INVALID_ARG;
  size_t est = ads_hbm_estimate(&spec->params, &spec->crv);
  if (est == 0) return ADS_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->spec = *spec;
  r->est = est;
  size_t nn = count_nodes(spec->params, 1), nc = count_nodes(spec->params, 2);
  r->K.assign(K_nodal, K_nodal + nn);
  if (phi_nodal) {
    r->phi.assign(phi_nodal, phi_nodal + nn);
    r->has_phi = true;
  }
  if (S0) {
    r->S0.assign(S0, S0 + nc);
    r->has_S0 = true;
  }
  if (theta0) {
    int np = spec->crv.width * spec->params.dim + spec->crv.width +
             (spec->crv.hidden_layers - 1) * (spec->crv.width * spec->crv.width + spec->crv.width) +
             spec->crv.width + 1;
    r->theta0.assign(theta0, theta0 + np);
    r->has_theta = true;
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (est > s->cfg.hbm_budget) {
    s->rejected++;
    return ADS_ERR_OOM;  // can never be admitted under this budget
  }
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->pending.push_back(r);
  *id_out = r->id;
  s->cv_work.notify_one();
  return ADS_OK;
}

ads_status ads_server_wait(ads_server* s, int64_t id, double timeout_s, double* S_out,
                           double* P_out, ads_request_result* res) {
  if (!s) return ADS_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return ADS_ERR_INVALID_ARG;
  r = it->second;
  if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 600.0),
                           [&] { return r->done; }))
    return ADS_ERR_TIMEOUT;
  if (r->status == ADS_OK) {
    if (S_out) std::memcpy(S_out, r->S_out.data(), r->S_out.size() * sizeof(double));
    if (P_out) std::memcpy(P_out, r->P_out.data(), r->P_out.size() * sizeof(double));
  }
  if (res) {
    res->status = r->status;
    res->steps = r->steps_done;
    res->queue_ms = r->t_admit.time_since_epoch().count() ? ms_between(r->t_submit, r->t_admit) : 0.0;
    res->total_ms = ms_between(r->t_submit, r->t_done);
    res->p50_step_ms = percentile(r->lat_ms, 0.5);
    res->p99_step_ms = percentile(r->lat_ms, 0.99);
    res->last = r->last;
  }
  s->all.erase(id);
  return r->status;
}

ads_status ads_server_stats(ads_server* s, ads_server_stats_t* out) {
  if (!s || !out) return ADS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->steps = s->steps_total;
  out->pending = (int64_t)s->pending.size();
  out->active = (int64_t)s->active.size();
  out->peak_active = s->peak_active;
  out->bytes_in_use = s->used;
  out->peak_bytes = s->peak_used;
  out->p50_step_ms = percentile(s->lat_all, 0.5);
  out->p99_step_ms = percentile(s->lat_all, 0.99);
  return ADS_OK;
}

void ads_server_destroy(ads_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->all)
    if (kv.second->ctx) ads_destroy(kv.second->ctx);
  for (auto x : s->streams) cudaStreamDestroy(x);
  delete s;
}

}  // extern "C"
