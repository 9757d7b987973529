// Registration server: continuous batching of Algorithm 2 on one GPU.
//
// Three kinds of work overlap:
//   * callers submit requests (host threads, never blocked by the GPU);
//   * the admission thread takes requests in FIFO order as soon as the
//     request's device-memory bound fits the budget and a slot is free, and
//     prepares each one on its own stream (copy-in, checks, normalisation,
//     masses, tree or packed reference, state), leaving it resident;
//   * the runner thread advances all resident pairs together on the run
//     stream, `iters_per_tick` iterations per tick with the batch kernels
//     (one force launch and one epilogue launch per iteration for all pairs).
//     Between ticks it adds newly prepared pairs and retires finished ones.
//
// The runner keeps one tick in flight ahead of the one it inspects: tick k+1
// is launched before the done flags of tick k are read, so the host work of a
// tick boundary is hidden behind GPU work. A pair that finishes inside a tick
// (iteration limit or stop test, both decided on the device) skips its work
// in the remaining launches, so it stops after exactly the same iterations as
// it would alone. Its state is read on a third stream (no kernel writes a
// finished pair's state) and its memory is released on the run stream,
// ordered after every launch that still lists it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fga_batch.cuh"

namespace fga {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  fga_pair q{};
  fga_params prm{};  // this request's parameters (its own or the server's)
  int64_t charge = 0;
  double work = 0;  // estimated force terms per iteration
  double submit_ms = 0;
};

// One admitted pair: its resident device memory and descriptor.
struct Slot {
  Request req;
  std::unique_ptr<Scratch> keep;
  fga_tree* tree = nullptr;
  DevState* ds = nullptr;
  PairDev P{};
  double info[8] = {0, 0, 0, 0, 0, 0, 0, 1};
  double admit_ms = 0, start_ms = -1;
  bool retiring = false;
};

void copy_message(char* dst, size_t cap, const char* msg) {
  std::strncpy(dst, msg ? msg : "", cap - 1);
  dst[cap - 1] = '\0';
}

}  // namespace
}  // namespace fga

using namespace fga;

struct fga_server {
  fga_params p{};
  fga_server_config cfg{};
  int device = 0;
  int64_t budget = 0;
  std::vector<cudaStream_t> prep_s;  // one per preparation thread
  cudaStream_t run_s = nullptr, read_s = nullptr;
  Clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_admit, cv_run, cv_done;
  std::deque<Request> pending;
  std::deque<std::unique_ptr<Slot>> ready;
  std::deque<fga_served> completed;
  int preparing = 0, resident = 0;
  int64_t charged = 0, next_ticket = 1;
  double work = 0, max_work = 0;
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_taken = 0;
  int64_t ticks = 0, pair_iters = 0;
  double busy_ms = 0;
  bool stop = false;
  std::vector<std::thread> admit_thr;
  std::thread run_thr;

  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

  // Completes a request that never became resident (caller holds mu).
  void fail_locked(const Request& r, int code, const char* msg, double admit_ms) {
    fga_served out;
    std::memset(&out, 0, sizeof(out));
    out.ticket = r.ticket;
    out.result.status = code;
    out.submit_ms = r.submit_ms;
    out.admit_ms = admit_ms;
    out.start_ms = -1;
    out.done_ms = now_ms();
    copy_message(out.error, sizeof(out.error), msg);
    completed.push_back(out);
    ++n_completed;
    ++n_failed;
    cv_done.notify_all();
  }
};

namespace {

// Prepares one request on a preparation stream; on success the slot holds the
// resident pair and its state is initialised.
int prepare_slot(fga_server* S, Slot& sl, cudaStream_t s) {
  const fga_pair& q = sl.req.q;
  int64_t h2d = 0;
  Prepared pr;
  Scratch tmp(s);  // staged inputs and normalised copies, freed after setup
  sl.keep.reset(new Scratch(s));
  int rc = prepare_inputs(tmp, q.X, q.N, q.Y, q.M, q.mX, q.mY, &sl.req.prm, pr, h2d, s);
  if (rc) return rc;
  int flags[8];
  FGA_CUDA_TRY(cudaMemcpyAsync(flags, pr.flags, sizeof(flags), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  if ((rc = check_pair_flags(flags, "fga_server", sl.req.ticket))) return rc;
  if (sl.keep->alloc(&sl.ds, 1)) return FGA_ENOMEM;
  if ((rc = build_pair(q, pr, &sl.req.prm, *sl.keep, &sl.tree, sl.ds, sl.P, s))) return rc;
  FGA_CUDA_TRY(cudaMemcpyAsync(sl.info, pr.info, sizeof(sl.info), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  return FGA_OK;
}

// Frees a slot's device memory on stream s (after the work queued there).
void release_slot(Slot& sl, cudaStream_t s) {
  if (sl.tree) {
    sl.tree->stream = s;
    fga_tree_destroy(sl.tree);
    sl.tree = nullptr;
  }
  if (sl.keep) {
    sl.keep->s = s;
    sl.keep.reset();
  }
}

void admit_loop(fga_server* S, int w) {
  cudaSetDevice(S->device);
  cudaStream_t ps = S->prep_s[w];
  for (;;) {
    std::unique_ptr<Slot> sl(new Slot);
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_admit.wait(lk, [&] {
        if (S->stop) return true;
        if (S->pending.empty()) return false;
        const int held = S->preparing + (int)S->ready.size() + S->resident;
        const Request& h = S->pending.front();
        const bool work_ok = S->max_work <= 0 || held == 0 || S->work + h.work <= S->max_work;
        return held < S->cfg.max_pairs && S->charged + h.charge <= S->budget && work_ok;
      });
      if (S->stop) return;
      sl->req = S->pending.front();
      S->pending.pop_front();
      S->charged += sl->req.charge;
      S->work += sl->req.work;
      ++S->preparing;
      sl->admit_ms = S->now_ms();
    }
    clear_error();
    const int rc = prepare_slot(S, *sl, ps);
    std::string msg = rc ? std::string(fga_last_error()) : std::string();
    if (rc) {
      release_slot(*sl, ps);
      cudaStreamSynchronize(ps);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    --S->preparing;
    if (rc) {
      S->charged -= sl->req.charge;
      S->work -= sl->req.work;
      S->fail_locked(sl->req, rc, msg.c_str(), sl->admit_ms);
      S->cv_admit.notify_all();
    } else {
      S->ready.push_back(std::move(sl));
      S->cv_run.notify_all();
    }
  }
}

}  // namespace

namespace {

// Pinned host staging of one tick: the pair listing uploaded for it, the done
// flags read back after it, and the slots it lists.
struct TickStage {
  PairDev* pairs = nullptr;
  unsigned* tstart = nullptr;
  unsigned* bstart = nullptr;
  int* flags = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  std::vector<std::shared_ptr<Slot>> listed;
  bool in_flight = false;
};

int stage_reserve(TickStage& t, size_t n) {
  if (n <= t.cap) return FGA_OK;
  size_t cap = std::max<size_t>(64, t.cap);
  while (cap < n) cap *= 2;
  cudaFreeHost(t.pairs);
  cudaFreeHost(t.tstart);
  cudaFreeHost(t.bstart);
  cudaFreeHost(t.flags);
  t.pairs = nullptr;
  t.tstart = t.bstart = nullptr;
  t.flags = nullptr;
  t.cap = 0;
  FGA_CUDA_TRY(cudaMallocHost((void**)&t.pairs, sizeof(PairDev) * cap));
  FGA_CUDA_TRY(cudaMallocHost((void**)&t.tstart, sizeof(unsigned) * (cap + 1)));
  FGA_CUDA_TRY(cudaMallocHost((void**)&t.bstart, sizeof(unsigned) * (cap + 1)));
  FGA_CUDA_TRY(cudaMallocHost((void**)&t.flags, sizeof(int) * cap));
  t.cap = cap;
  return FGA_OK;
}

void stage_free(TickStage& t) {
  cudaFreeHost(t.pairs);
  cudaFreeHost(t.tstart);
  cudaFreeHost(t.bstart);
  cudaFreeHost(t.flags);
  if (t.ev) cudaEventDestroy(t.ev);
  t = TickStage();
}

// Device copies of the current listing (shared by consecutive ticks; an
// upload is ordered after the ticks already queued on the run stream).
struct Listing {
  PairDev* pairs = nullptr;
  unsigned* tstart = nullptr;
  unsigned* bstart = nullptr;
  int* flags = nullptr;
  unsigned* ctr = nullptr;
  size_t cap = 0;
  int n = 0;
  unsigned ntasks = 0, nblocks = 0;
  int fgrid = 1;
  unsigned* cost = nullptr;   // per-task cost of the last force launch
  unsigned* order = nullptr;  // heavy-first order derived from it
  size_t task_cap = 0;
  int launches = 0;           // force launches since the listing changed
  bool have_order = false;
};

int listing_reserve(Listing& L, size_t n, cudaStream_t s) {
  if (n <= L.cap) return FGA_OK;
  size_t cap = std::max<size_t>(64, L.cap);
  while (cap < n) cap *= 2;
  dev_free(L.pairs, s);
  dev_free(L.tstart, s);
  dev_free(L.bstart, s);
  dev_free(L.flags, s);
  L.pairs = nullptr;
  L.tstart = L.bstart = nullptr;
  L.flags = nullptr;
  L.cap = 0;
  if (dev_alloc_n(&L.pairs, cap, s) || dev_alloc_n(&L.tstart, cap + 1, s) ||
      dev_alloc_n(&L.bstart, cap + 1, s) || dev_alloc_n(&L.flags, cap, s))
    return FGA_ENOMEM;
  L.cap = cap;
  return FGA_OK;
}

class Runner {
 public:
  explicit Runner(fga_server* S) : S_(S), s_(S->run_s) {}

  void loop() {
    cudaSetDevice(S_->device);
    if (setup()) {
      fail_all(FGA_ECUDA, fga_last_error());
      wait_for_stop();
      return;
    }
    auto last = Clock::now();
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(S_->mu);
        if (active_.empty() && !any_in_flight())
          S_->cv_run.wait(lk, [&] { return S_->stop || !S_->ready.empty(); });
        if (S_->stop) break;
        while (!S_->ready.empty()) {
          active_.push_back(std::shared_ptr<Slot>(S_->ready.front().release()));
          S_->ready.pop_front();
          ++S_->resident;
          dirty_ = true;
        }
      }
      const auto now = Clock::now();
      const bool busy = !active_.empty();
      clear_error();
      int rc = FGA_OK;
      bool launched = false;
      if (has_live()) {
        rc = launch_tick(stage_[cur_]);
        launched = rc == FGA_OK;
      }
      if (rc == FGA_OK && stage_[cur_ ^ 1].in_flight) rc = inspect(stage_[cur_ ^ 1]);
      if (rc != FGA_OK) {
        // a failed launch or copy: finish every resident pair with the error
        const std::string msg = fga_last_error();
        cudaStreamSynchronize(s_);
        for (auto& t : stage_) {
          t.in_flight = false;
          t.listed.clear();
        }
        fail_all(rc, msg.c_str());
        launched = false;
      }
      if (launched) {
        stage_[cur_].in_flight = true;
        cur_ ^= 1;
      }
      {
        std::lock_guard<std::mutex> lk(S_->mu);
        if (busy) S_->busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - now).count();
      }
      last = now;
    }
    (void)last;
    cudaStreamSynchronize(s_);
    for (auto& t : stage_) t.listed.clear();
    for (auto& sl : active_) release_slot(*sl, s_);
    active_.clear();
    cudaStreamSynchronize(s_);
    teardown();
  }

 private:
  fga_server* S_;
  cudaStream_t s_;
  std::vector<std::shared_ptr<Slot>> active_;  // admitted, not yet retired
  std::vector<std::shared_ptr<Slot>> listing_slots_;
  TickStage stage_[2];
  Listing L_;
  int cur_ = 0;
  bool dirty_ = true;
  DevState* h_states_ = nullptr;  // pinned: states of the pairs being retired
  size_t h_states_cap_ = 0;
  cudaEvent_t ev_read_ = nullptr;

  bool any_in_flight() const { return stage_[0].in_flight || stage_[1].in_flight; }

  bool has_live() const {
    for (const auto& sl : active_)
      if (!sl->retiring) return true;
    return false;
  }

  int setup() {
    for (auto& t : stage_) FGA_CUDA_TRY(cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming));
    FGA_CUDA_TRY(cudaEventCreateWithFlags(&ev_read_, cudaEventDisableTiming));
    if (dev_alloc_n(&L_.ctr, 2, s_)) return FGA_ENOMEM;
    FGA_CUDA_TRY(cudaMemsetAsync(L_.ctr, 0, 2 * sizeof(unsigned), s_));
    return FGA_OK;
  }

  void teardown() {
    for (auto& t : stage_) stage_free(t);
    if (ev_read_) cudaEventDestroy(ev_read_);
    cudaFreeHost(h_states_);
    dev_free(L_.pairs, s_);
    dev_free(L_.tstart, s_);
    dev_free(L_.bstart, s_);
    dev_free(L_.flags, s_);
    dev_free(L_.ctr, s_);
    dev_free(L_.cost, s_);
    dev_free(L_.order, s_);
    cudaStreamSynchronize(s_);
  }

  void wait_for_stop() {
    std::unique_lock<std::mutex> lk(S_->mu);
    S_->cv_run.wait(lk, [&] { return S_->stop; });
  }

  // Queues one tick on the run stream: the listing upload if the resident set
  // changed, iters_per_tick iterations, the done flags and their read-back.
  int launch_tick(TickStage& T) {
    int rc = FGA_OK;
    if (dirty_) {
      listing_slots_.clear();
      for (int pass = 0; pass < 2; ++pass)  // Barnes-Hut pairs first
        for (const auto& sl : active_)
          if (!sl->retiring && (sl->P.method == FGA_BH) == (pass == 0)) listing_slots_.push_back(sl);
      const size_t n = listing_slots_.size();
      if ((rc = stage_reserve(T, n)) || (rc = listing_reserve(L_, n, s_))) return rc;
      std::vector<PairDev> v(n);
      for (size_t k = 0; k < n; ++k) v[k] = listing_slots_[k]->P;
      std::vector<unsigned> ts, bs;
      if (!batch_layout(v, ts, bs)) {
        set_error("fga_server: too many tasks resident at once (2^31)");
        return FGA_EINVAL;
      }
      std::memcpy(T.pairs, v.data(), sizeof(PairDev) * n);
      std::memcpy(T.tstart, ts.data(), sizeof(unsigned) * (n + 1));
      std::memcpy(T.bstart, bs.data(), sizeof(unsigned) * (n + 1));
      FGA_CUDA_TRY(cudaMemcpyAsync(L_.pairs, T.pairs, sizeof(PairDev) * n, cudaMemcpyHostToDevice, s_));
      FGA_CUDA_TRY(cudaMemcpyAsync(L_.tstart, T.tstart, sizeof(unsigned) * (n + 1), cudaMemcpyHostToDevice, s_));
      FGA_CUDA_TRY(cudaMemcpyAsync(L_.bstart, T.bstart, sizeof(unsigned) * (n + 1), cudaMemcpyHostToDevice, s_));
      L_.n = (int)n;
      L_.ntasks = ts[n];
      L_.nblocks = bs[n];
      L_.fgrid = batch_force_grid(L_.ntasks);
      if (L_.ntasks > L_.task_cap) {
        dev_free(L_.cost, s_);
        dev_free(L_.order, s_);
        L_.cost = L_.order = nullptr;
        L_.task_cap = 0;
        const size_t cap = std::max<size_t>(4096, 2 * (size_t)L_.ntasks);
        if (dev_alloc_n(&L_.cost, cap, s_) || dev_alloc_n(&L_.order, cap + TASK_ORDER_SCRATCH, s_))
          return FGA_ENOMEM;
        L_.task_cap = cap;
      }
      // task indices changed: the next launch runs in index order and records costs
      L_.launches = 0;
      L_.have_order = false;
      dirty_ = false;
    } else if ((rc = stage_reserve(T, (size_t)L_.n))) {
      return rc;
    }
    for (int it = 0; it < S_->cfg.iters_per_tick; ++it) {
      if ((rc = launch_batch_iteration(L_.pairs, L_.n, L_.tstart, L_.ntasks, L_.bstart, 0, L_.ctr, L_.fgrid,
                                       s_, L_.have_order ? L_.order : nullptr, L_.cost)))
        return rc;
      if (bh_reorder_due(++L_.launches, FGA_BATCH_REORDER_EVERY)) {
        if ((rc = launch_task_order(L_.cost, L_.ntasks, L_.order, s_))) return rc;
        L_.have_order = true;
        count_launch(1);
      }
      if ((rc = launch_batch_iteration(L_.pairs, L_.n, L_.tstart, 0, L_.bstart, L_.nblocks, L_.ctr, L_.fgrid,
                                       s_)))
        return rc;
      count_launch(2);
    }
    if ((rc = launch_done_flags(L_.pairs, L_.n, L_.flags, s_))) return rc;
    count_launch(1);
    FGA_CUDA_TRY(cudaMemcpyAsync(T.flags, L_.flags, sizeof(int) * L_.n, cudaMemcpyDeviceToHost, s_));
    FGA_CUDA_TRY(cudaEventRecord(T.ev, s_));
    T.listed = listing_slots_;
    const double now = S_->now_ms();
    for (auto& sl : T.listed)
      if (sl->start_ms < 0) sl->start_ms = now;
    std::lock_guard<std::mutex> lk(S_->mu);
    ++S_->ticks;
    S_->pair_iters += (int64_t)L_.n * S_->cfg.iters_per_tick;
    return FGA_OK;
  }

  // Waits for a tick, retires the pairs it reported done and publishes their
  // results.
  int inspect(TickStage& T) {
    FGA_CUDA_TRY(cudaEventSynchronize(T.ev));
    T.in_flight = false;
    std::vector<std::shared_ptr<Slot>> fin;
    for (size_t k = 0; k < T.listed.size(); ++k)
      if (T.flags[k] && !T.listed[k]->retiring) {
        T.listed[k]->retiring = true;
        fin.push_back(T.listed[k]);
      }
    T.listed.clear();
    if (fin.empty()) return FGA_OK;
    if (fin.size() > h_states_cap_) {
      cudaFreeHost(h_states_);
      h_states_ = nullptr;
      h_states_cap_ = 0;
      const size_t cap = std::max<size_t>(64, 2 * fin.size());
      FGA_CUDA_TRY(cudaMallocHost((void**)&h_states_, sizeof(DevState) * cap));
      h_states_cap_ = cap;
    }
    // finished pairs are read on the side stream while the next tick runs
    for (size_t j = 0; j < fin.size(); ++j)
      FGA_CUDA_TRY(cudaMemcpyAsync(&h_states_[j], fin[j]->ds, sizeof(DevState), cudaMemcpyDeviceToHost,
                                   S_->read_s));
    FGA_CUDA_TRY(cudaEventRecord(ev_read_, S_->read_s));
    FGA_CUDA_TRY(cudaEventSynchronize(ev_read_));
    FGA_CUDA_TRY(cudaStreamWaitEvent(s_, ev_read_, 0));
    std::vector<fga_served> outs(fin.size());
    const double now = S_->now_ms();
    for (size_t j = 0; j < fin.size(); ++j) {
      Slot& sl = *fin[j];
      fga_served& o = outs[j];
      std::memset(&o, 0, sizeof(o));
      o.ticket = sl.req.ticket;
      fill_pair_result(h_states_[j], sl.info, sl.P.method, &sl.req.prm, o.result);
      o.submit_ms = sl.req.submit_ms;
      o.admit_ms = sl.admit_ms;
      o.start_ms = sl.start_ms;
      o.done_ms = now;
      if (o.result.status == FGA_EINTERNAL)
        copy_message(o.error, sizeof(o.error), "a device check failed: non-finite transform");
      release_slot(sl, s_);
    }
    active_.erase(std::remove_if(active_.begin(), active_.end(),
                                 [](const std::shared_ptr<Slot>& sl) { return sl->retiring; }),
                  active_.end());
    dirty_ = true;
    std::lock_guard<std::mutex> lk(S_->mu);
    for (size_t j = 0; j < fin.size(); ++j) {
      S_->completed.push_back(outs[j]);
      ++S_->n_completed;
      if (outs[j].result.status == FGA_EINTERNAL) ++S_->n_failed;
      S_->charged -= fin[j]->req.charge;
      S_->work -= fin[j]->req.work;
      --S_->resident;
    }
    S_->cv_done.notify_all();
    S_->cv_admit.notify_all();
    return FGA_OK;
  }

  void fail_all(int code, const char* msg) {
    for (auto& sl : active_) release_slot(*sl, s_);
    cudaStreamSynchronize(s_);
    std::lock_guard<std::mutex> lk(S_->mu);
    for (auto& sl : active_) {
      S_->fail_locked(sl->req, code, msg, sl->admit_ms);
      S_->charged -= sl->req.charge;
      S_->work -= sl->req.work;
      --S_->resident;
    }
    active_.clear();
    listing_slots_.clear();
    dirty_ = true;
    S_->cv_admit.notify_all();
  }
};

void run_loop(fga_server* S) {
  Runner r(S);
  r.loop();
}

}  // namespace

extern "C" int fga_server_create(const fga_params* p, const fga_server_config* cfg, fga_server** out) {
  clear_error();
  if (!out) {
    set_error("fga_server_create: null output");
    return FGA_EINVAL;
  }
  *out = nullptr;
  int rc = check_register_params(p);
  if (rc) return rc;
  if (p->max_depth < 1 || p->max_depth > 20) {
    set_error("fga_server_create: max_depth must be in 1..20");
    return FGA_EINVAL;
  }
  if (p->max_iter < 1) {
    set_error("fga_server_create: max_iter must be >= 1");
    return FGA_EINVAL;
  }
  std::unique_ptr<fga_server> S(new fga_server);
  S->p = *p;
  S->p.profile = 0;
  if (cfg) S->cfg = *cfg;
  if (S->cfg.max_pairs <= 0) S->cfg.max_pairs = 4096;
  if (S->cfg.iters_per_tick <= 0) S->cfg.iters_per_tick = 4;
  if (S->cfg.prep_threads <= 0) S->cfg.prep_threads = 4;
  S->cfg.prep_threads = std::min(S->cfg.prep_threads, 64);
  S->max_work = S->cfg.max_work == 0 ? 4e9 : S->cfg.max_work;
  if (S->cfg.device >= 0) {
    FGA_CUDA_TRY(cudaSetDevice(S->cfg.device));
    S->device = S->cfg.device;
  } else {
    FGA_CUDA_TRY(cudaGetDevice(&S->device));
  }
  S->budget = S->cfg.mem_budget;
  if (S->budget <= 0) {
    size_t free_b = 0, total_b = 0;
    FGA_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    S->budget = (int64_t)(free_b / 4 * 3);
  }
  S->prep_s.assign(S->cfg.prep_threads, nullptr);
  for (auto& ps : S->prep_s) FGA_CUDA_TRY(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
  FGA_CUDA_TRY(cudaStreamCreateWithFlags(&S->run_s, cudaStreamNonBlocking));
  FGA_CUDA_TRY(cudaStreamCreateWithFlags(&S->read_s, cudaStreamNonBlocking));
  S->t0 = Clock::now();
  fga_server* raw = S.release();
  for (int w = 0; w < raw->cfg.prep_threads; ++w) raw->admit_thr.emplace_back(admit_loop, raw, w);
  raw->run_thr = std::thread(run_loop, raw);
  *out = raw;
  return FGA_OK;
}

extern "C" int fga_server_submit(fga_server* S, const fga_pair* req, int64_t* ticket) {
  clear_error();
  if (!S || !req || !ticket) {
    set_error("fga_server_submit: null argument");
    return FGA_EINVAL;
  }
  if (!req->X || !req->Y || req->N <= 0 || req->M <= 0 || req->N > ((int64_t)1 << 26) ||
      req->M > ((int64_t)1 << 26)) {
    set_error("fga_server_submit: bad sizes or null points");
    return FGA_EINVAL;
  }
  Request r;
  r.q = *req;
  r.prm = req->params ? *req->params : S->p;
  r.prm.profile = 0;
  r.q.params = nullptr;
  if (req->params) {
    int rc = check_register_params(&r.prm);
    if (rc) return rc;
    if (r.prm.max_iter < 1) {
      set_error("fga_server_submit: max_iter must be >= 1");
      return FGA_EINVAL;
    }
  }
  const int method = resolve_method(&r.prm, req->N);
  r.charge = pair_bytes_bound(req->N, req->M, method, &r.prm);
  r.work = method == FGA_BH ? 64.0 * (double)req->M * std::log2((double)req->N + 1.0)
                            : (double)req->N * (double)req->M;
  std::lock_guard<std::mutex> lk(S->mu);
  if (r.charge > S->budget) {
    set_error("fga_server_submit: the pair needs up to " + std::to_string(r.charge) +
              " device bytes, more than the whole budget of " + std::to_string(S->budget));
    return FGA_EINVAL;
  }
  if (S->stop) {
    set_error("fga_server_submit: the server is stopping");
    return FGA_EINVAL;
  }
  r.ticket = S->next_ticket++;
  r.submit_ms = S->now_ms();
  S->pending.push_back(r);
  ++S->n_submitted;
  *ticket = r.ticket;
  S->cv_admit.notify_all();
  return FGA_OK;
}

extern "C" int fga_server_poll(fga_server* S, fga_served* out, int max, int* n, int wait_ms) {
  clear_error();
  if (!S || !n || (max > 0 && !out)) {
    set_error("fga_server_poll: null argument");
    return FGA_EINVAL;
  }
  *n = 0;
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&] { return !S->completed.empty() || S->n_taken + (int64_t)S->completed.size() >= S->n_submitted; };
  if (S->completed.empty() && wait_ms != 0) {
    if (wait_ms < 0)
      S->cv_done.wait(lk, ready);
    else
      S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
  }
  int k = 0;
  while (k < max && !S->completed.empty()) {
    out[k++] = S->completed.front();
    S->completed.pop_front();
  }
  S->n_taken += k;
  *n = k;
  return FGA_OK;
}

extern "C" int fga_server_stats_get(fga_server* S, fga_server_stats* out) {
  clear_error();
  if (!S || !out) {
    set_error("fga_server_stats_get: null argument");
    return FGA_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->n_submitted;
  out->completed = S->n_completed;
  out->failed = S->n_failed;
  out->pending = (int)S->pending.size();
  out->preparing = S->preparing + (int)S->ready.size();
  out->resident = S->resident;
  out->bytes_charged = S->charged;
  out->work_admitted = S->work;
  out->mem_budget = S->budget;
  out->ticks = S->ticks;
  out->pair_iterations = S->pair_iters;
  out->busy_ms = S->busy_ms;
  return FGA_OK;
}

extern "C" int fga_server_destroy(fga_server* S) {
  clear_error();
  if (!S) return FGA_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->pending.clear();
  }
  S->cv_admit.notify_all();
  S->cv_run.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->admit_thr)
    if (t.joinable()) t.join();
  if (S->run_thr.joinable()) S->run_thr.join();
  cudaSetDevice(S->device);
  for (auto& sl : S->ready) release_slot(*sl, S->run_s);
  S->ready.clear();
  cudaStreamSynchronize(S->run_s);
  for (cudaStream_t ps : S->prep_s) {
    cudaStreamSynchronize(ps);
    cudaStreamDestroy(ps);
  }
  cudaStreamDestroy(S->run_s);
  cudaStreamDestroy(S->read_s);
  delete S;
  return FGA_OK;
}
