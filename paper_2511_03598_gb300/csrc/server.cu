// Request server: admits rounding requests in arrival order while their estimated device footprint
// fits a memory budget, and runs them on worker threads, one CUDA stream each.  Host code only;
// every kernel it causes is launched by tt_round_adaptive_sum.
//
// Admission is strict first-come first-served: the oldest waiting request is admitted as soon as
// its footprint fits next to the running ones, and no later request overtakes it (no starvation
// of large requests).  A request whose footprint exceeds the whole budget is refused at submit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ttr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int32_t s = 0, d = 0;
  const int64_t* n = nullptr;
  std::vector<const int64_t*> r;
  std::vector<const double* const*> cores;
  double tol = 0.0;
  int64_t block = 0;
  uint64_t seed = 0;
  ttr_options opts{};
  uint64_t footprint = 0, bytes_in = 0;
  Clock::time_point t_submit, t_admit;
  bool done = false;
  ttr_server_result res{};
};

}  // namespace

struct ttr_server {
  ttr_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> waiting;
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  std::vector<std::thread> workers;
  int64_t next_id = 1;
  uint64_t in_use = 0, peak = 0;
  int64_t admitted = 0;
  int64_t submitted = 0, completed = 0, failed = 0, running = 0;
  bool stop = false;
};

namespace {

// Device bytes a rounding of the sum may hold at once: the input copies, the output arena and the
// work buffers of tt_round_adaptive_sum, all sized by the formal ranks R_k = sum_i r_k^(i) (an
// upper estimate; the library's memory pool may keep freed blocks for reuse on top of it).
uint64_t footprint_of(int32_t s, int32_t d, const int64_t* n, const int64_t* const* r, uint64_t* bytes_in) {
  std::vector<double> R(d + 1, 0.0);
  double in = 0.0, rpart = 1.0;
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < d; ++k) {
      in += (double)r[i][k] * n[k] * r[i][k + 1];
      if (k > 0) rpart = std::max(rpart, (double)r[i][k]);
    }
  for (int k = 1; k < d; ++k)
    for (int i = 0; i < s; ++i) R[k] += (double)r[i][k];
  R[0] = R[d] = 1.0;
  double formal = 0.0, cmax = 1.0, rowsmax = 1.0, rmax = 1.0, nmax = 1.0, Wrows = 0.0;
  for (int k = 0; k < d; ++k) {
    const double c = R[k] * n[k] * R[k + 1];
    formal += c;
    cmax = std::max(cmax, c);
    rowsmax = std::max(rowsmax, R[k] * n[k]);
    rmax = std::max(rmax, R[k + 1]);
    nmax = std::max(nmax, (double)n[k]);
    if (k >= 1) Wrows += R[k];
  }
  const double wcap = 2.0 * rmax + 64.0;                  // sketch columns (rank + one block, geometric growth)
  double dbl = in + formal + 2.0 * cmax;                  // inputs, output arena, two projected cores
  dbl += rowsmax * (rmax + 3.0 * std::max(rmax, wcap) + 2.0 * wcap);   // Q, QR scratch, S, all sketches, T
  dbl += Wrows * wcap * 3.0;                              // W_2..W_d and their kept digit planes
  dbl += (double)d * nmax * wcap * 1.5;                   // Omega and its integer copy
  dbl += 4.0 * rmax * rmax + rmax * nmax * rpart + 2.0 * nmax * rmax;
  dbl += 2.0 * rowsmax * rmax;                            // digit planes of the largest tensor-core B operand
  dbl += rowsmax * (rmax + wcap + 64.0);                  // the block loop's rows when they live in global memory
  *bytes_in = (uint64_t)(8.0 * in);
  return (uint64_t)(8.0 * dbl) + (64ull << 20);
}

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Run one admitted request on `stream`; fills q.res (status and, on success, the host result).
void run_request(Request& q, cudaStream_t stream) {
  ttr_server_result& out = q.res;
  out.status = TTR_OK;
  // device copies of every summand's cores, in one allocation
  std::vector<int64_t> off;
  int64_t total = 0;
  for (int i = 0; i < q.s; ++i)
    for (int k = 0; k < q.d; ++k) {
      off.push_back(total);
      total += q.r[i][k] * q.n[k] * q.r[i][k + 1];
    }
  double* dev = nullptr;
  const size_t bytes = sizeof(double) * std::max<int64_t>(total, 1);
  cudaMemPool_t pool = ttr::library_pool(stream);   // keeps the freed input copy for the next request
  cudaError_t e = pool ? cudaMallocFromPoolAsync((void**)&dev, bytes, pool, stream)
                       : cudaMallocAsync((void**)&dev, bytes, stream);
  if (e != cudaSuccess) {
    out.status = TTR_ERR_OOM;
    return;
  }
  std::vector<const double*> ptrs((size_t)q.s * q.d);
  std::vector<const double* const*> per(q.s);
  for (int i = 0; i < q.s && e == cudaSuccess; ++i) {
    for (int k = 0; k < q.d && e == cudaSuccess; ++k) {
      const size_t j = (size_t)i * q.d + k;
      ptrs[j] = dev + off[j];
      e = cudaMemcpyAsync(dev + off[j], q.cores[i][k], sizeof(double) * q.r[i][k] * q.n[k] * q.r[i][k + 1],
                          cudaMemcpyHostToDevice, stream);
    }
    per[i] = ptrs.data() + (size_t)i * q.d;
  }
  ttr_result res{};
  int st = e == cudaSuccess ? TTR_OK : TTR_ERR_CUDA;
  if (st == TTR_OK)
    st = tt_round_adaptive_sum(q.s, q.d, q.n, q.r.data(), per.data(), q.tol, q.block, q.seed, &q.opts, stream, &res);
  if (st == TTR_OK) {
    out.d = res.d;
    out.ranks = (int64_t*)malloc(sizeof(int64_t) * (res.d + 1));
    int64_t cnt = 0;
    for (int k = 0; k < res.d; ++k) cnt += res.ranks[k] * q.n[k] * res.ranks[k + 1];
    out.data = (double*)malloc(sizeof(double) * std::max<int64_t>(cnt, 1));
    out.cores = (double**)malloc(sizeof(double*) * res.d);
    if (!out.ranks || !out.data || !out.cores) {
      st = TTR_ERR_OOM;
    } else {
      memcpy(out.ranks, res.ranks, sizeof(int64_t) * (res.d + 1));
      int64_t o = 0;
      for (int k = 0; k < res.d && st == TTR_OK; ++k) {
        const int64_t c = res.ranks[k] * q.n[k] * res.ranks[k + 1];
        out.cores[k] = out.data + o;
        if (cudaMemcpyAsync(out.data + o, res.cores[k], sizeof(double) * c, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess)
          st = TTR_ERR_CUDA;
        o += c;
      }
      if (st == TTR_OK && cudaStreamSynchronize(stream) != cudaSuccess) st = TTR_ERR_CUDA;
    }
    ttr_free(&res, stream);
  }
  cudaFreeAsync(dev, stream);
  cudaStreamSynchronize(stream);
  if (st != TTR_OK) {
    snprintf(out.message, sizeof(out.message), "%s", ttr_last_error());
    free(out.ranks);
    free(out.data);
    free(out.cores);
    out.ranks = nullptr;
    out.data = nullptr;
    out.cores = nullptr;
    out.d = 0;
  }
  out.status = st;
}

void worker_main(ttr_server* S) {
  cudaStream_t stream = nullptr;
  bool ready = false;
  for (;;) {
    Request* q = nullptr;
    bool quit = false;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] {
        return S->stop ? S->waiting.empty() || S->in_use + S->waiting.front()->footprint <= S->cfg.device_budget
                       : !S->waiting.empty() && S->in_use + S->waiting.front()->footprint <= S->cfg.device_budget;
      });
      if (S->waiting.empty()) {
        quit = true;   // stopping and nothing left
      } else {
        q = S->waiting.front();
        S->waiting.pop_front();
        S->in_use += q->footprint;
        S->peak = std::max(S->peak, S->in_use);
        S->running++;
        q->res.admit_order = S->admitted++;
        q->t_admit = Clock::now();
      }
    }
    if (quit) break;
    S->cv_work.notify_all();   // the next request in line may fit too
    if (!ready) {
      if (cudaSetDevice(S->cfg.device) == cudaSuccess &&
          cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess)
        ready = true;
    }
    if (ready) {
      run_request(*q, stream);
    } else {
      q->res.status = TTR_ERR_CUDA;
      snprintf(q->res.message, sizeof(q->res.message), "could not select the device or create a stream");
    }
    const auto t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      q->res.ms_queue = ms_since(q->t_submit, q->t_admit);
      q->res.ms_run = ms_since(q->t_admit, t_done);
      q->res.footprint = q->footprint;
      q->res.bytes_in = q->bytes_in;
      q->done = true;
      S->in_use -= q->footprint;
      S->running--;
      if (q->res.status == TTR_OK) S->completed++;
      else S->failed++;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int ttr_server_create(const ttr_server_config* cfg, ttr_server** out) {
  if (!cfg || !out) return ttr::set_error("cfg and out must be non-null"), TTR_ERR_ARG;
  *out = nullptr;
  if (cfg->workers < 1 || cfg->workers > 256) return ttr::set_error("workers must be in [1, 256]"), TTR_ERR_ARG;
  if (cfg->device_budget == 0) return ttr::set_error("device_budget must be positive"), TTR_ERR_ARG;
  if (cfg->device < 0 || cfg->max_sms < 0) return ttr::set_error("device and max_sms must be >= 0"), TTR_ERR_ARG;
  ttr_server* S = new (std::nothrow) ttr_server;
  if (!S) return ttr::set_error("host allocation"), TTR_ERR_OOM;
  S->cfg = *cfg;
  try {
    for (int i = 0; i < cfg->workers; ++i) S->workers.emplace_back(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return ttr::set_error("could not start the worker threads"), TTR_ERR_OOM;
  }
  *out = S;
  return TTR_OK;
}

int ttr_server_submit(ttr_server* S, int32_t s, int32_t d, const int64_t* n, const int64_t* const* r,
                      const double* const* const* host_cores, double tol, int64_t block, uint64_t seed,
                      const ttr_options* opts, int64_t* id) {
  if (!S || !id) return ttr::set_error("server and id must be non-null"), TTR_ERR_ARG;
  if (s < 1 || s > TTR_MAX_SUMMANDS) return ttr::set_error("number of summands must be in [1, TTR_MAX_SUMMANDS]"), TTR_ERR_ARG;
  if (d < 2 || d > TTR_MAX_D || !n || !r || !host_cores) return ttr::set_error("bad TT arguments"), TTR_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol)) return ttr::set_error("tol must be positive and finite"), TTR_ERR_ARG;
  for (int i = 0; i < s; ++i) {
    if (!r[i] || !host_cores[i]) return ttr::set_error("null rank or core array of a summand"), TTR_ERR_ARG;
    if (r[i][0] != 1 || r[i][d] != 1) return ttr::set_error("r[0] and r[d] must be 1"), TTR_ERR_ARG;
    for (int k = 0; k < d; ++k) {
      if (n[k] < 1 || r[i][k + 1] < 1) return ttr::set_error("mode sizes and ranks must be >= 1"), TTR_ERR_ARG;
      if (!host_cores[i][k]) return ttr::set_error("null core pointer"), TTR_ERR_ARG;
    }
  }
  auto q = std::make_unique<Request>();
  q->s = s;
  q->d = d;
  q->n = n;
  q->r.assign(r, r + s);
  q->cores.assign(host_cores, host_cores + s);
  q->tol = tol;
  q->block = block;
  q->seed = seed;
  if (opts) q->opts = *opts;
  else ttr_default_options(&q->opts);
  if (S->cfg.max_sms > 0) {
    q->opts.max_sms = S->cfg.max_sms;
  } else {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->cfg.device) != cudaSuccess) nsm = 0;
    q->opts.max_sms = nsm > 0 ? std::max(1, nsm / S->cfg.workers) : 0;
  }
  q->footprint = footprint_of(s, d, n, r, &q->bytes_in);
  if (q->footprint > S->cfg.device_budget)
    return ttr::set_error("request needs about " + std::to_string((unsigned long long)q->footprint) +
                          " bytes of device memory, more than the whole budget"),
           TTR_ERR_UNSUPPORTED;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return ttr::set_error("server is stopping"), TTR_ERR_ARG;
    q->id = S->next_id++;
    *id = q->id;
    S->waiting.push_back(q.get());
    S->all.emplace(q->id, std::move(q));
    S->submitted++;
  }
  S->cv_work.notify_all();
  return TTR_OK;
}

int ttr_server_wait(ttr_server* S, int64_t id, ttr_server_result* out) {
  if (!S || !out) return ttr::set_error("server and out must be non-null"), TTR_ERR_ARG;
  memset(out, 0, sizeof(*out));
  std::unique_ptr<Request> q;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return ttr::set_error("unknown or already collected request id"), TTR_ERR_ARG;
    Request* p = it->second.get();
    // p stays valid while the entry is in the map; another thread waiting for the same id may
    // collect it first, so look the entry up again after waking
    S->cv_done.wait(lock, [&] {
      auto jt = S->all.find(id);
      return jt == S->all.end() || jt->second.get() != p || p->done;
    });
    auto jt = S->all.find(id);
    if (jt == S->all.end() || jt->second.get() != p) return ttr::set_error("request collected by another wait"), TTR_ERR_ARG;
    q = std::move(jt->second);
    S->all.erase(jt);
  }
  *out = q->res;
  return q->res.status;
}

void ttr_server_result_free(ttr_server_result* res) {
  if (!res) return;
  free(res->ranks);
  free(res->data);
  free(res->cores);
  memset(res, 0, sizeof(*res));
}

int ttr_server_get_stats(ttr_server* S, ttr_server_stats* out) {
  if (!S || !out) return ttr::set_error("server and out must be non-null"), TTR_ERR_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->waiting = (int64_t)S->waiting.size();
  out->running = S->running;
  out->in_use = S->in_use;
  out->peak_in_use = S->peak;
  return TTR_OK;
}

void ttr_server_destroy(ttr_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->all) ttr_server_result_free(&kv.second->res);
  delete S;
}

}  // extern "C"
