// Batched inversion (many SPD matrices of uneven order) and the
// continuous-batching request server.
//
// Both run on a pool of worker threads; each worker owns one CUDA stream and
// a cache of plans keyed by (padded order, K, h), and runs the single-matrix
// pipeline of ibmi_invert on its stream, so the kernels of different matrices
// overlap on the GPU.  Orders are padded up to size buckets by embedding A in
// [[A, 0], [0, I]], whose inverse is [[A^{-1}, 0], [0, I]]: one plan then
// serves every matrix of a bucket.  The partition (K, h) of each bucket is
// chosen by measuring candidate partitions on the first matrix of the bucket.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "batch_dev.cuh"
#include "batch_plan.h"
#include "mixed.cuh"
#include "plan.cuh"

namespace ibmi {

// Copies A (p x p, lda) into the top-left of Ab (pb x pb) and fills the rest
// with the identity; H is copied back by the caller from the top-left block.
__global__ void k_pad_embed(const double* A, int64_t lda, int64_t p, double* Ab, int64_t pb) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pb * pb) return;
  int64_t i = idx / pb, j = idx - i * pb;
  Ab[idx] = (i < p && j < p) ? A[i * lda + j] : (i == j ? 1.0 : 0.0);
}

__global__ void k_unpad(const double* Hb, int64_t pb, int64_t p, double* H, int64_t ldh) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * p) return;
  int64_t i = idx / p, j = idx - i * p;
  H[i * ldh + j] = Hb[i * pb + j];
}

static ibmi_plan_desc desc_for(const Shape& s, const ibmi_batch_opts& o) {
  ibmi_plan_desc d;
  ibmi_plan_desc_init(&d);
  d.p = s.p;
  d.K = s.K;
  d.h = s.h;
  d.precision = o.precision;
  d.tol = o.tol;
  d.max_sweeps = o.max_sweeps;
  d.check_every = 1;
  // an unfinished tail returns to the sweeps
  d.ns_theta = handover_theta(s.p, o.precision == IBMI_MIXED, o.ns_theta);
  d.ns_max = o.ns_max;
  return d;
}

// One worker: a stream and a small plan cache.  Every plan runs on its own
// staging buffers (P->dA, P->dH of the bucket order), so the CUDA graphs the
// mixed pipeline captures stay valid from one matrix to the next.
struct Worker {
  int device = 0;
  cudaStream_t stream = nullptr;
  struct Cached {
    ibmi_plan_t plan;
    size_t bytes;
    uint64_t last_use;
  };
  std::map<std::pair<Shape, int>, Cached> plans;   // by (partition, precision)
  size_t plan_bytes = 0;
  uint64_t clock = 0;
  // device-batched groups this worker ran, by (partition, group size): their
  // buffers are kept for the next call of the same composition
  struct CachedGroup {
    std::unique_ptr<DevGroup> g;
    uint64_t last_use = 0;
  };
  std::map<std::pair<Shape, int>, CachedGroup> groups;
  size_t group_bytes = 0;
  // The cached group for (s, n), created if missing; with a nonzero cap, least
  // recently used groups and plans go first until it fits (nullptr if it
  // cannot be created).
  DevGroup* group(const Shape& s, int n, size_t cap) {
    auto it = groups.find({s, n});
    if (it != groups.end()) {
      it->second.last_use = ++clock;
      return it->second.g.get();
    }
    const size_t need = DevGroup::bytes_per_matrix(s.p, s.K, s.h) * (size_t)n;
    if (cap) {
      while (!groups.empty() && group_bytes + plan_bytes + need > cap) {
        auto lru = groups.begin();
        for (auto jt = groups.begin(); jt != groups.end(); ++jt)
          if (jt->second.last_use < lru->second.last_use) lru = jt;
        group_bytes -= lru->second.g->bytes();
        groups.erase(lru);
      }
      evict_for(group_bytes + need, cap);
    }
    std::unique_ptr<DevGroup> g(new DevGroup());
    if (g->create(s.p, s.K, s.h, n) != IBMI_OK) return nullptr;
    group_bytes += g->bytes();
    DevGroup* r = g.get();
    groups[{s, n}] = CachedGroup{std::move(g), ++clock};
    return r;
  }

  ibmi_status init(int dev) {
    device = dev;
    cudaSetDevice(dev);
    IBMI_CUDA_TRY(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    return IBMI_OK;
  }
  void release_plans() {
    for (auto& kv : plans) ibmi_plan_destroy(kv.second.plan);
    plans.clear();
    plan_bytes = 0;
  }
  // Frees least recently used plans until `need` more bytes fit in `cap`.
  void evict_for(size_t need, size_t cap) {
    while (!plans.empty() && plan_bytes + need > cap) {
      auto lru = plans.begin();
      for (auto it = plans.begin(); it != plans.end(); ++it)
        if (it->second.last_use < lru->second.last_use) lru = it;
      ibmi_plan_destroy(lru->second.plan);
      plan_bytes -= lru->second.bytes;
      plans.erase(lru);
    }
  }
  void destroy() {
    cudaSetDevice(device);
    release_plans();
    groups.clear();
    group_bytes = 0;
    if (stream) cudaStreamDestroy(stream);
  }
  ibmi_status plan(const Shape& s, const ibmi_batch_opts& o, size_t max_plan_bytes, ibmi_plan_t* out) {
    auto it = plans.find({s, o.precision});
    if (it != plans.end()) {
      // stopping parameters may differ from call to call
      it->second.last_use = ++clock;
      ibmi_plan_t P = it->second.plan;
      const ibmi_plan_desc d = desc_for(s, o);
      P->d.tol = d.tol;
      P->d.max_sweeps = d.max_sweeps;
      P->d.ns_theta = d.ns_theta;
      P->d.ns_max = d.ns_max;
      if (o.precision == IBMI_MIXED) mixed_enable_graphs(P, o.graphs != 0);
      *out = P;
      return IBMI_OK;
    }
    ibmi_plan_desc d = desc_for(s, o);
    const size_t need = ibmi_plan_bytes(&d) + 16 * (size_t)s.p * s.p;
    if (max_plan_bytes) evict_for(need, max_plan_bytes);
    ibmi_plan_t P = nullptr;
    IBMI_TRY(ibmi_plan(&d, &P));
    if (cudaMalloc(&P->dA, sizeof(double) * s.p * s.p) != cudaSuccess ||
        cudaMalloc(&P->dH, sizeof(double) * s.p * s.p) != cudaSuccess) {
      cudaGetLastError();
      ibmi_plan_destroy(P);
      return IBMI_ERR_OOM;
    }
    if (o.precision == IBMI_MIXED) mixed_enable_graphs(P, o.graphs != 0);
    plans[{s, o.precision}] = Cached{P, need, ++clock};
    plan_bytes += need;
    *out = P;
    return IBMI_OK;
  }
  // Inverts one matrix (device A, H of order p) with the plan for `s`: A is
  // embedded in the plan's staging buffer (identity padding up to s.p), the
  // result copied back from its leading block.
  ibmi_status run(const Shape& s, const ibmi_batch_opts& o, size_t max_plan_bytes, const double* A, int64_t lda,
                  int64_t p, double* H, int64_t ldh, ibmi_result* res) {
    ibmi_plan_t P;
    IBMI_TRY(plan(s, o, max_plan_bytes, &P));
    const int64_t pb = s.p;
    note_launch();
    k_pad_embed<<<(unsigned)((pb * pb + 255) / 256), 256, 0, stream>>>(A, lda, p, P->dA, pb);
    IBMI_CUDA_TRY(cudaGetLastError());
    ibmi_status st = ibmi_invert(P, P->dA, pb, P->dH, pb, stream, res);
    if (st == IBMI_OK || st == IBMI_NOT_CONVERGED) {
      note_launch();
      k_unpad<<<(unsigned)((p * p + 255) / 256), 256, 0, stream>>>(P->dH, pb, p, H, ldh);
      IBMI_CUDA_TRY(cudaGetLastError());
      IBMI_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    return st;
  }
};

// Process-wide cache of tuned partitions per (bucket, precision).
static std::mutex g_tune_mu;
static std::map<std::pair<int64_t, int>, Shape> g_tuned;

// Times the candidate partitions of bucket pb (tune_candidates) on one matrix
// and keeps the fastest that converges.
static Shape tune_bucket(Worker& w, int64_t pb, const ibmi_batch_opts& o, const double* A, int64_t lda, int64_t p,
                         double* H, int64_t ldh) {
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned.find({pb, o.precision});
    if (it != g_tuned.end()) return it->second;
  }
  Shape best = default_shape(pb);
  double best_t = INFINITY;
  for (const Shape& s : tune_candidates(pb)) {
    ibmi_result r;
    double t = INFINITY;
    for (int rep = 0; rep < 2; ++rep) {   // first run includes plan creation
      auto t0 = std::chrono::steady_clock::now();
      ibmi_status st = w.run(s, o, 0, A, lda, p, H, ldh, &r);
      double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (st != IBMI_OK) { t = INFINITY; break; }
      t = dt;
    }
    if (t < best_t) { best_t = t; best = s; }
  }
  w.release_plans();
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned[{pb, o.precision}] = best;
  return best;
}

// Process-wide pool of batch workers per device: their streams, plans and the
// CUDA graphs captured in those plans persist from one batched call to the
// next.  One batched call runs at a time.
static std::mutex g_pool_mu;
static std::map<int, std::vector<std::unique_ptr<Worker>>> g_pool;
static constexpr size_t kWorkerPlanCap = (size_t)6 << 30;   // plan bytes a pooled worker may keep
static constexpr int64_t kDevMaxOrder = 2048;                // largest bucket run as device groups
static std::mutex g_stats_mu;
static ibmi_batch_stats g_stats{};                           // of the last batched call
static constexpr size_t kDevGroupMax = 64;                   // matrices per device group
static constexpr size_t kDevGroupBytes = (size_t)4 << 30;    // device bytes per group

static Shape shape_for(int64_t p, const ibmi_batch_opts& o) {
  const int64_t pb = bucket_of(p);
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned.find({pb, o.precision});
  if (it != g_tuned.end()) return it->second;
  return default_shape(pb);
}

// Inverts one matrix with its bucket's tuned partition; a matrix that does not
// converge with it is run once more with the robust partition (the counts in
// *res then cover both runs).
static ibmi_status run_tuned(Worker& w, const ibmi_batch_opts& o, size_t max_plan_bytes, const double* A, int64_t lda,
                             int64_t p, double* H, int64_t ldh, ibmi_result* res) {
  memset(res, 0, sizeof(ibmi_result));
  const Shape s = shape_for(p, o);
  ibmi_status st = w.run(s, o, max_plan_bytes, A, lda, p, H, ldh, res);
  const Shape rs = robust_shape(bucket_of(p));
  if (st == IBMI_NOT_CONVERGED && (s.K != rs.K || s.h != rs.h)) {
    ibmi_result again;
    memset(&again, 0, sizeof(again));
    st = w.run(rs, o, max_plan_bytes, A, lda, p, H, ldh, &again);
    again.sweeps += res->sweeps;
    again.ns_steps += res->ns_steps;
    again.flops += res->flops;
    again.seconds += res->seconds;
    *res = again;
  }
  res->status = st;
  return st;
}

// ----------------------------------------------------------------- server --

struct Request {
  uint64_t id = 0;
  int64_t p = 0;
  double tol = 0.0;
  std::vector<double> A;     // host copy of the input
  std::vector<double> H;     // host result
  ibmi_result res{};
  int state = 0;             // 0 queued, 1 admitted, 2 done, 3 cancelled
  int home = 0;              // worker that holds the plans of its size bucket
  size_t bytes = 0;          // device bytes charged while admitted
  std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
};

}  // namespace ibmi

struct ibmi_server_impl {
  ibmi_batch_opts opts{};
  size_t budget = 0;       // total device bytes the server may hold
  size_t req_budget = 0;   // part of it for admitted requests (a quarter; the rest caps the plan caches)
  size_t in_use = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::shared_ptr<ibmi::Request>> reqs;
  std::vector<double> latencies;     // seconds, completed requests
  std::chrono::steady_clock::time_point t_first_done, t_last_done;
  int64_t completed = 0;
  std::vector<std::thread> threads;
  std::vector<ibmi::Worker> workers;
  std::vector<char> busy;            // per worker: running a batch (guarded by mu)
};

namespace ibmi {

static size_t request_bytes(int64_t p) {
  // device copies of A and H plus the padded staging of the plan that runs it
  const int64_t pb = bucket_of(p);
  return sizeof(double) * (size_t)(2 * p * p + 2 * pb * pb);
}

static constexpr int kServeGroupMax = 8;   // requests one device group of the server takes

// Home worker of a request: the plans and device groups a worker caches are
// those of the size buckets it ran, so a request goes to the worker of its
// bucket while that worker is free; a busy home lets any free worker take it.
static int home_worker(int64_t p, int workers) {
  return (int)(((uint64_t)bucket_of(p) * 0x9E3779B97F4A7C15ull >> 32) % (uint64_t)workers);
}

static bool same_shape(const Shape& a, const Shape& b) { return !(a < b) && !(b < a); }

// One server worker: admits the oldest queued request that fits the budget,
// together with the queued requests of the same size bucket, partition and
// tolerance that fit too (at most kServeGroupMax, orders up to kDevMaxOrder,
// mixed precision), and inverts them as one device group; a request the
// group leaves unfinished, and every other request, runs on the
// single-matrix pipeline of this worker.  Requests that arrive meanwhile are
// taken by the next free worker.
static void server_loop(ibmi_server_impl* S, int wi) {
  Worker& w = S->workers[wi];
  cudaSetDevice(S->device);
  std::vector<double*> dA, dH;   // staging per request slot
  std::vector<int64_t> dcap;
  const size_t cache_cap = (S->budget - S->req_budget) / S->workers.size();
  auto fits = [&](const std::shared_ptr<Request>& q) {
    return q->state == 0 && (q->home == wi || S->busy[q->home]) &&
           (S->in_use + q->bytes <= S->req_budget || S->in_use == 0);
  };
  while (true) {
    std::vector<std::shared_ptr<Request>> batch;
    Shape sh{};
    bool grouped = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop) return true;
        for (uint64_t id : S->queue)
          if (fits(S->reqs[id])) return true;
        return false;
      });
      if (S->stop) break;
      std::shared_ptr<Request> r;
      for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        auto& q = S->reqs[*it];
        if (fits(q)) {
          r = q;
          S->queue.erase(it);
          break;
        }
      }
      if (!r) continue;
      auto admit = [&](const std::shared_ptr<Request>& q) {
        q->state = 1;
        q->t_admit = std::chrono::steady_clock::now();
        S->in_use += q->bytes;
        batch.push_back(q);
      };
      admit(r);
      S->busy[wi] = 1;
      grouped = S->opts.precision == IBMI_MIXED && S->opts.device_batch && bucket_of(r->p) <= kDevMaxOrder;
      if (grouped) {
        sh = shape_for(r->p, S->opts);
        for (auto it = S->queue.begin(); it != S->queue.end() && (int)batch.size() < kServeGroupMax;) {
          auto& q = S->reqs[*it];
          if (q->state == 0 && q->tol == r->tol && bucket_of(q->p) == sh.p && same_shape(shape_for(q->p, S->opts), sh) &&
              S->in_use + q->bytes <= S->req_budget) {
            admit(q);
            it = S->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
    }
    const int nb = (int)batch.size();
    std::vector<ibmi_status> st(nb, IBMI_OK);
    if ((int)dA.size() < nb) {
      dA.resize(nb, nullptr);
      dH.resize(nb, nullptr);
      dcap.resize(nb, 0);
    }
    for (int b = 0; b < nb; ++b) {
      const int64_t p = batch[b]->p;
      if (p * p > dcap[b]) {
        cudaFree(dA[b]);
        cudaFree(dH[b]);
        dA[b] = dH[b] = nullptr;
        dcap[b] = 0;
        if (cudaMalloc(&dA[b], sizeof(double) * p * p) != cudaSuccess ||
            cudaMalloc(&dH[b], sizeof(double) * p * p) != cudaSuccess) {
          cudaGetLastError();
          st[b] = IBMI_ERR_OOM;
          continue;
        }
        dcap[b] = p * p;
      }
      if (cudaMemcpyAsync(dA[b], batch[b]->A.data(), sizeof(double) * p * p, cudaMemcpyHostToDevice, w.stream) !=
          cudaSuccess)
        st[b] = IBMI_ERR_CUDA;
    }
    ibmi_batch_opts o = S->opts;
    o.tol = batch[0]->tol;
    std::vector<int> single(nb, 1);   // requests for the single-matrix pipeline
    std::vector<ibmi_result> first(nb);
    std::vector<char> tried(nb, 0);
    if (grouped) {
      std::vector<int> ok;
      for (int b = 0; b < nb; ++b)
        if (st[b] == IBMI_OK) ok.push_back(b);
      int cap = 1;
      while (cap < (int)ok.size()) cap *= 2;
      DevGroup* g = ok.empty() ? nullptr : w.group(sh, cap, cache_cap);
      if (g) {
        std::vector<BatchMat> mats;
        for (int b : ok) mats.push_back(BatchMat{dA[b], batch[b]->p, dH[b], batch[b]->p, batch[b]->p});
        std::vector<ibmi_result> r(ok.size());
        std::vector<int> fb(ok.size(), 1);
        const ibmi_status gs =
            g->run(mats.data(), (int)ok.size(), o, handover_theta(sh.p, true, o.ns_theta), w.stream, r.data(), fb.data());
        if (gs == IBMI_OK) {
          for (size_t j = 0; j < ok.size(); ++j) {
            const int b = ok[j];
            if (!fb[j]) {
              batch[b]->res = r[j];
              st[b] = (ibmi_status)r[j].status;
              single[b] = 0;
            } else {
              first[b] = r[j];
              tried[b] = 1;
            }
          }
        }
      }
    }
    for (int b = 0; b < nb; ++b) {
      if (!single[b] || st[b] != IBMI_OK) continue;
      const int64_t p = batch[b]->p;
      st[b] = run_tuned(w, o, cache_cap, dA[b], p, p, dH[b], p, &batch[b]->res);
      if (tried[b]) {
        batch[b]->res.sweeps += first[b].sweeps;
        batch[b]->res.ns_steps += first[b].ns_steps;
        batch[b]->res.flops += first[b].flops;
      }
    }
    for (int b = 0; b < nb; ++b) {
      Request& r = *batch[b];
      const int64_t p = r.p;
      if (st[b] == IBMI_OK || st[b] == IBMI_NOT_CONVERGED) {
        r.H.resize((size_t)p * p);
        if (cudaMemcpyAsync(r.H.data(), dH[b], sizeof(double) * p * p, cudaMemcpyDeviceToHost, w.stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(w.stream) != cudaSuccess)
          st[b] = IBMI_ERR_CUDA;
      }
      r.res.status = st[b];
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& rp : batch) {
        Request& r = *rp;
        r.t_done = std::chrono::steady_clock::now();
        S->in_use -= r.bytes;
        if (r.state != 3) r.state = 2;
        std::vector<double>().swap(r.A);
        S->latencies.push_back(std::chrono::duration<double>(r.t_done - r.t_submit).count());
        if (S->completed == 0) S->t_first_done = r.t_done;
        S->t_last_done = r.t_done;
        ++S->completed;
      }
      S->busy[wi] = 0;
    }
    S->cv.notify_all();
  }
  for (size_t b = 0; b < dA.size(); ++b) {
    cudaFree(dA[b]);
    cudaFree(dH[b]);
  }
}

}  // namespace ibmi

using namespace ibmi;

extern "C" {

void ibmi_batch_opts_init(ibmi_batch_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = IBMI_MIXED;
  o->tol = 1e-10;
  o->max_sweeps = 500;
  o->ns_theta = 0.0;   // by order
  o->ns_max = 8;
  o->workers = 8;
  o->autotune = 1;
  o->graphs = 1;
  o->device_batch = 1;
}

size_t ibmi_plan_bytes(const ibmi_plan_desc* d) {
  if (!d || d->p < 2 || d->K < 1) return 0;
  const double p = (double)d->p, K = (double)d->K;
  const double m = std::min(p, p / K + 2.0 * (double)d->h);
  double b = 8.0 * (K * m * m + m * m + p * p / 4096.0 + 64.0);              // A_I^{-1}, S, partials
  b += 8.0 * p * p;                                                          // A from its lower triangle
  const double ncols = d->precision == IBMI_MIXED ? m : p;
  b += 8.0 * K * (m * m + m * ncols + 32.0 * m);                             // batched factorisation
  if (d->precision == IBMI_MIXED) {
    const double ldp = ceil(p / 64.0) * 64.0;
    b += 4.0 * p * ldp + 4.0 * p * ldp + 4.0 * K * m * ldp + 4.0 * 64.0 * m * m;   // H master + slices, W, split-K
    b += 2.0 * p * ldp * 25.0 + 4.0 * p * ldp * 10.0 + 16.0 * p * p;          // refinement planes
  } else {
    b += 8.0 * K * m * p;                                                     // W
    b += (d->ns_theta > 0.0 ? 16.0 * p * p : 0.0);
  }
  return (size_t)b;
}

ibmi_status ibmi_invert_batched(int32_t n, const int64_t* p, const double* const* A, const int64_t* lda,
                                double* const* H, const int64_t* ldh, const ibmi_batch_opts* opts,
                                ibmi_result* out) {
  if (n < 0 || (n > 0 && (!p || !A || !H || !lda || !ldh || !out))) return IBMI_ERR_INVALID_ARG;
  ibmi_batch_opts o;
  if (opts) o = *opts; else ibmi_batch_opts_init(&o);
  if (o.workers < 1 || o.workers > 64 || (o.precision != IBMI_FP64 && o.precision != IBMI_MIXED))
    return IBMI_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (p[i] < 2 || lda[i] < p[i] || ldh[i] < p[i] || !A[i] || !H[i]) return IBMI_ERR_INVALID_ARG;
  if (n == 0) return IBMI_OK;
  int dev = 0;
  IBMI_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> pool_lock(g_pool_mu);
  auto& pool = g_pool[dev];
  const int W = std::min<int>(o.workers, n);
  while ((int)pool.size() < W) {
    auto w = std::make_unique<Worker>();
    IBMI_TRY(w->init(dev));
    pool.push_back(std::move(w));
  }
  // largest matrices first: better balance across workers
  std::vector<int32_t> order(n);
  for (int32_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return p[a] > p[b]; });
  // autotune: first matrix of each untuned bucket, in parallel across workers
  if (o.autotune) {
    std::vector<int32_t> firsts;
    std::map<int64_t, bool> seen;
    for (int32_t i : order) {
      const int64_t pb = bucket_of(p[i]);
      if (seen.count(pb)) continue;
      seen[pb] = true;
      std::lock_guard<std::mutex> g(g_tune_mu);
      if (!g_tuned.count({pb, o.precision})) firsts.push_back(i);
    }
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int wi = 0; wi < W; ++wi)
      th.emplace_back([&, wi] {
        cudaSetDevice(dev);
        for (int j; (j = next.fetch_add(1)) < (int)firsts.size();) {
          const int32_t i = firsts[j];
          tune_bucket(*pool[wi], bucket_of(p[i]), o, A[i], lda[i], p[i], H[i], ldh[i]);
        }
      });
    for (auto& t : th) t.join();
  }
  std::vector<ibmi_status> st(n, IBMI_OK);
  ibmi_batch_stats stats{};
  auto t_groups = std::chrono::steady_clock::now();
  // device-side groups: matrices of one bucket and partition, in lockstep
  std::vector<int32_t> rest;               // matrices for the single-matrix pipeline
  std::vector<ibmi_result> first_try(n);   // a fallback's device attempt (its counts are added)
  std::vector<char> tried(n, 0);
  if (o.precision == IBMI_MIXED && o.device_batch) {
    std::map<Shape, std::vector<int32_t>> by_shape;
    for (int32_t i : order) {
      if (bucket_of(p[i]) > kDevMaxOrder) rest.push_back(i);
      else by_shape[shape_for(p[i], o)].push_back(i);
    }
    struct Task {
      Shape s;
      std::vector<int32_t> idx;
    };
    std::vector<Task> tasks;
    for (auto& kv : by_shape) {
      const size_t per = DevGroup::bytes_per_matrix(kv.first.p, kv.first.K, kv.first.h);
      const size_t cap = std::max<size_t>(1, std::min<size_t>(kDevGroupMax, kDevGroupBytes / per));
      const size_t nb = (kv.second.size() + cap - 1) / cap;   // balanced chunks
      for (size_t c = 0; c < nb; ++c) {
        Task t{kv.first, {}};
        for (size_t j = c; j < kv.second.size(); j += nb) t.idx.push_back(kv.second[j]);
        tasks.push_back(std::move(t));
      }
    }
    // most work first; task t always runs on worker t % W, so a repeated call
    // with the same batch finds its groups' buffers where it left them
    std::stable_sort(tasks.begin(), tasks.end(), [](const Task& a, const Task& b) {
      return (double)a.idx.size() * a.s.p * a.s.p * a.s.p > (double)b.idx.size() * b.s.p * b.s.p * b.s.p;
    });
    std::mutex mu;
    std::vector<std::thread> tg;
    for (int wi = 0; wi < W; ++wi)
      tg.emplace_back([&, wi] {
        cudaSetDevice(dev);
        Worker& w = *pool[wi];
        for (size_t t = wi; t < tasks.size(); t += W) {
          const Task& task = tasks[t];
          const int ng = (int)task.idx.size();
          DevGroup* slot = w.group(task.s, ng, 0);
          ibmi_status s = slot ? IBMI_OK : IBMI_ERR_OOM;
          std::vector<BatchMat> mats(ng);
          std::vector<ibmi_result> r(ng);
          std::vector<int> fb(ng, 1);
          for (int b = 0; b < ng; ++b) {
            const int32_t i = task.idx[b];
            mats[b] = BatchMat{A[i], lda[i], H[i], ldh[i], p[i]};
          }
          if (s == IBMI_OK) s = slot->run(mats.data(), ng, o, handover_theta(task.s.p, true, o.ns_theta), w.stream,
                                          r.data(), fb.data());
          std::lock_guard<std::mutex> g(mu);
          if (s == IBMI_OK) {
            stats.groups += 1;
            stats.device_matrices += ng;
            stats.rounds_max = std::max<int64_t>(stats.rounds_max, slot->rounds());
            stats.rounds_total += slot->rounds();
          }
          for (int b = 0; b < ng; ++b) {
            const int32_t i = task.idx[b];
            if (s == IBMI_OK && fb[b]) stats.fallbacks += 1;
            if (s == IBMI_OK && !fb[b]) {
              out[i] = r[b];
              st[i] = (ibmi_status)r[b].status;
            } else {
              if (s == IBMI_OK) {
                first_try[i] = r[b];
                tried[i] = 1;
              }
              rest.push_back(i);
            }
          }
        }
      });
    for (auto& t : tg) t.join();
    std::stable_sort(rest.begin(), rest.end(), [&](int32_t a, int32_t b) { return p[a] > p[b]; });
  } else {
    rest = order;
  }
  auto t_single = std::chrono::steady_clock::now();
  stats.seconds_groups = std::chrono::duration<double>(t_single - t_groups).count();
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  const int nrest = (int)rest.size();
  for (int wi = 0; wi < W; ++wi)
    th.emplace_back([&, wi] {
      cudaSetDevice(dev);
      Worker& w = *pool[wi];
      for (int j; (j = next.fetch_add(1)) < nrest;) {
        const int32_t i = rest[j];
        st[i] = run_tuned(w, o, kWorkerPlanCap, A[i], lda[i], p[i], H[i], ldh[i], &out[i]);
        out[i].status = st[i];
        if (tried[i]) {   // the device attempt's work counts too
          out[i].sweeps += first_try[i].sweeps;
          out[i].ns_steps += first_try[i].ns_steps;
          out[i].flops += first_try[i].flops;
        }
      }
    });
  for (auto& t : th) t.join();
  stats.seconds_single = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_single).count();
  {
    std::lock_guard<std::mutex> g(g_stats_mu);
    g_stats = stats;
  }
  ibmi_status worst = IBMI_OK;
  for (int32_t i = 0; i < n; ++i)
    if (st[i] != IBMI_OK && (worst == IBMI_OK || worst == IBMI_NOT_CONVERGED)) worst = st[i];
  return worst;
}

ibmi_status ibmi_batch_last_stats(ibmi_batch_stats* out) {
  if (!out) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_stats_mu);
  *out = g_stats;
  return IBMI_OK;
}

ibmi_status ibmi_batch_release(void) {
  std::lock_guard<std::mutex> pool_lock(g_pool_mu);
  for (auto& kv : g_pool)
    for (auto& w : kv.second) w->destroy();
  g_pool.clear();
  return IBMI_OK;
}

ibmi_status ibmi_serve_create(size_t hbm_budget, const ibmi_batch_opts* opts, ibmi_server_t* out) {
  if (!out || hbm_budget == 0) return IBMI_ERR_INVALID_ARG;
  auto* S = new ibmi_server_impl();
  if (opts) S->opts = *opts; else ibmi_batch_opts_init(&S->opts);
  if (S->opts.workers < 1 || S->opts.workers > 64) { delete S; return IBMI_ERR_INVALID_ARG; }
  S->budget = hbm_budget;
  S->req_budget = hbm_budget / 4;
  cudaGetDevice(&S->device);
  S->workers.resize(S->opts.workers);
  S->busy.assign(S->opts.workers, 0);
  for (auto& w : S->workers) {
    if (w.init(S->device) != IBMI_OK) {
      for (auto& x : S->workers) x.destroy();
      delete S;
      return IBMI_ERR_CUDA;
    }
  }
  for (int i = 0; i < S->opts.workers; ++i) S->threads.emplace_back(server_loop, S, i);
  *out = (ibmi_server_t)S;
  return IBMI_OK;
}

ibmi_status ibmi_serve_submit(ibmi_server_t h, const double* A_host, int64_t p, int64_t lda, double tol,
                              uint64_t* req) {
  auto* S = (ibmi_server_impl*)h;
  if (!S || !A_host || !req || p < 2 || lda < p || !(tol >= 0.0)) return IBMI_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->p = p;
  r->tol = tol;
  r->bytes = request_bytes(p);
  r->home = home_worker(p, (int)S->workers.size());
  if (r->bytes > S->req_budget) return IBMI_ERR_BUDGET;
  r->A.resize((size_t)p * p);
  for (int64_t i = 0; i < p; ++i) memcpy(&r->A[(size_t)i * p], A_host + i * lda, sizeof(double) * p);
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r->id);
    *req = r->id;
  }
  S->cv.notify_all();
  return IBMI_OK;
}

ibmi_status ibmi_serve_poll(ibmi_server_t h, uint64_t req, double* H_host, int64_t ldh, ibmi_result* res) {
  auto* S = (ibmi_server_impl*)h;
  if (!S) return IBMI_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req);
    if (it == S->reqs.end()) return IBMI_ERR_INVALID_ARG;
    r = it->second;
    if (r->state == 3) { S->reqs.erase(it); return IBMI_ERR_CANCELLED; }
    if (r->state != 2) return IBMI_NOT_READY;
    S->reqs.erase(it);
  }
  if (res) *res = r->res;
  if (H_host && !r->H.empty()) {
    if (ldh < r->p) return IBMI_ERR_INVALID_ARG;
    for (int64_t i = 0; i < r->p; ++i) memcpy(H_host + i * ldh, &r->H[(size_t)i * r->p], sizeof(double) * r->p);
  }
  return (ibmi_status)r->res.status;
}

ibmi_status ibmi_serve_cancel(ibmi_server_t h, uint64_t req) {
  auto* S = (ibmi_server_impl*)h;
  if (!S) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req);
  if (it == S->reqs.end()) return IBMI_ERR_INVALID_ARG;
  auto& r = it->second;
  if (r->state == 0) {
    S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), req), S->queue.end());
    r->state = 3;
    return IBMI_OK;
  }
  return r->state == 3 ? IBMI_OK : IBMI_NOT_READY;   // admitted or finished: runs to completion
}

ibmi_status ibmi_serve_stats_reset(ibmi_server_t h) {
  auto* S = (ibmi_server_impl*)h;
  if (!S) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->latencies.clear();
  S->completed = 0;
  return IBMI_OK;
}

ibmi_status ibmi_serve_stats(ibmi_server_t h, double* p50, double* p99, double* inv_per_s, int64_t* completed,
                             uint64_t* bytes_in_use) {
  auto* S = (ibmi_server_impl*)h;
  if (!S) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return (double)NAN;
    size_t i = (size_t)std::min<double>((double)l.size() - 1, floor(q * (double)(l.size() - 1) + 0.5));
    return l[i];
  };
  if (p50) *p50 = pct(0.50);
  if (p99) *p99 = pct(0.99);
  if (inv_per_s) {
    const double span = std::chrono::duration<double>(S->t_last_done - S->t_first_done).count();
    *inv_per_s = (S->completed > 1 && span > 0) ? (double)(S->completed - 1) / span : NAN;
  }
  if (completed) *completed = S->completed;
  if (bytes_in_use) *bytes_in_use = S->in_use;
  return IBMI_OK;
}

ibmi_status ibmi_serve_destroy(ibmi_server_t h) {
  auto* S = (ibmi_server_impl*)h;
  if (!S) return IBMI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->threads) t.join();
  for (auto& w : S->workers) w.destroy();
  delete S;
  return IBMI_OK;
}

}  // extern "C"
