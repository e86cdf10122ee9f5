// Continuous-batching server (ssm_server_* in include/ssm.h).
//
// Requests wait in a first-come first-served queue. A free worker (a host thread with
// its own non-blocking CUDA stream) admits the first queued request whose device
// footprint fits in the HBM budget; a later request may pass the head of the queue
// when the head does not fit yet, at most `max_bypass` times per head. Admitted
// solves run concurrently on their streams, so kernels of different solves overlap on
// the GPU. Plans stay resident after their solve (when plan caching is on) and are
// reused by a later request with the same dictionary, grid and plan parameters; idle
// plans are evicted least recently used first when a request needs their memory.
//
// Latency classes: the iteration is HBM-bound, so a request's footprint stands for its
// cost per iteration. A request whose footprint is at most `small_bytes` is class 0;
// each factor of 4 above that is one class more, up to the number of stream priorities
// the device offers. Every worker has one stream per priority and runs a class-c
// request on the c-th highest. Requests above class 0 have their persistent kernels
// launched as `large_waves` waves of CTAs: short-lived CTAs let the block scheduler
// hand SMs to higher-priority streams every few hundred microseconds, so a small solve
// arriving during a large one is not held up for the large one's kernels (which would
// otherwise keep every SM for milliseconds).
//
// Reserved workers: the first `reserved_small` workers admit class-0 requests only, so a
// small request never waits for a worker behind large ones that hold all the others
// (stream priorities and launch waves help only a request that is already running).
// The other workers take any request, first come first served.
//
// Groups (group_small > 1): a worker that admits a class-0 low-rank FP32 request with
// device buffers also admits up to group_small - 1 such requests queued behind it (those
// that fit the budget without evicting), and solves them together with ssm_group_*: one
// launch per iteration for the whole group instead of one per request. Such a request
// always runs in a group (of one when nothing else waits), and a problem's bits do not
// depend on the rest of its group, so its result does not depend on the traffic.
//
// Memory accounting: every plan (running or idle) has a reservation, its peak
// footprint while planning and its persistent footprint afterwards. `held` sums the
// reservations of live plans, `dying` those of evicted plans not yet freed. A worker
// that evicts plans to admit a request frees them before it plans, so the device
// memory the plans hold never exceeds the budget, and held never exceeds it either.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <thread>
#include <unordered_map>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// parameters that determine a plan (everything but the stopping rule), normalised so
// that equivalent settings compare equal
bool same_plan(const ssm_params& a, const ssm_params& b) {
  if (a.ndim != b.ndim || a.P != b.P || a.Q != b.Q) return false;
  for (int d = 0; d < a.ndim; ++d)
    if (a.dims[d] != b.dims[d]) return false;
  const double xa = a.xi_p > 0 ? a.xi_p : 0.0, xb = b.xi_p > 0 ? b.xi_p : 0.0;
  const double ta = a.rank_tol > 0 ? a.rank_tol : 5e-5, tb = b.rank_tol > 0 ? b.rank_tol : 5e-5;
  // the low-rank form runs FP32 unless TF32X3 is asked for (BF16X3 there is FP32)
  auto norm_prec = [](const ssm_params& x) {
    if (x.form != SSM_FORM_LOWRANK) return x.precision;
    return x.precision == SSM_TF32X3 ? (int)SSM_TF32X3 : 0;
  };
  const int pa = norm_prec(a), pb = norm_prec(b);
  const int ra = a.form == SSM_FORM_LOWRANK ? a.rank : 0;
  const int rb = b.form == SSM_FORM_LOWRANK ? b.rank : 0;
  return a.lambda == b.lambda && a.beta == b.beta && xa == xb && a.form == b.form && ra == rb &&
         (a.form != SSM_FORM_LOWRANK || a.rank > 0 || ta == tb) && pa == pb &&
         a.stencil_pairs == b.stencil_pairs;
}

// FNV-1a style hash over the dictionary, one double at a time (a filter only: a match
// is confirmed byte by byte)
uint64_t hash_doubles(const double* data, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    uint64_t w;
    std::memcpy(&w, data + i, sizeof(w));
    h ^= w;
    h *= 1099511628211ull;
    h ^= h >> 29;
  }
  return h;
}

struct Resident {
  ssm_plan_t plan = nullptr;
  ssm_params p{};
  int waves = 1;
  std::vector<double> K;     // the dictionary the plan was made from
  uint64_t khash = 0;
  int64_t bytes = 0;         // reservation
  bool busy = false;
  uint64_t last_used = 0;
};

struct Request {
  int64_t ticket = 0;
  ssm_params p{};
  bool device_io = false;    // M and F are device buffers
  int level = 0;             // latency class: stream priority (0 = highest)
  int waves = 1;
  const double* K = nullptr;
  const float* M = nullptr;
  int64_t ldm = 0;
  float* F = nullptr;
  int64_t ldf = 0;
  uint64_t khash = 0;
  int64_t footprint = 0;     // peak estimate (reserved at admission)
  int bypassed = 0;
  int group_size = 0;        // > 0: solved in a group of this many requests
  bool done = false;
  Clock::time_point t_submit, t_admit, t_done;
  ssm_request_info info{};
  std::string error;
};

}  // namespace
}  // namespace ssm

using namespace ssm;

struct ssm_server_s {
  ssm_server_config cfg{};
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // queue changed, memory freed, or stop
  std::condition_variable cv_done;   // a request finished
  std::deque<Request*> pending;
  std::unordered_map<int64_t, std::unique_ptr<Request>> requests;
  std::list<std::unique_ptr<Resident>> residents;
  int64_t held = 0, dying = 0, peak = 0;
  int64_t next_ticket = 1, next_order = 0;
  uint64_t tick = 0;
  int active = 0;
  bool stop = false;
  ssm_server_stats st{};
  std::vector<std::thread> workers;
  // streams[level][worker]: one stream per priority level and worker (level 0 = highest)
  std::vector<std::vector<cudaStream_t>> streams;

  // choose a request to run (caller holds mu); fills the plan to use and the idle
  // plans to free first
  bool try_admit(int slot, Request** out, Resident** res_out,
                 std::vector<std::unique_ptr<Resident>>* evict) {
    const bool small_only = slot < cfg.reserved_small;
    for (size_t i = 0; i < pending.size(); ++i) {
      Request* q = pending[i];
      if (small_only && q->level != 0) continue;   // a reserved worker: class 0 only
      Resident* match = nullptr;
      if (cfg.cache_plans)
        for (auto& r : residents)
          if (!r->busy && r->khash == q->khash && r->waves == q->waves && same_plan(r->p, q->p) &&
              r->K.size() == (size_t)q->p.P * q->p.Q &&
              std::memcmp(r->K.data(), q->K, sizeof(double) * r->K.size()) == 0) {
            match = r.get();
            break;
          }
      const int64_t need = match ? 0 : q->footprint;
      int64_t avail = budget - held - dying;
      std::vector<Resident*> picks;
      if (need > avail) {
        std::vector<Resident*> idle;
        for (auto& r : residents)
          if (!r->busy && r.get() != match) idle.push_back(r.get());
        std::sort(idle.begin(), idle.end(),
                  [](const Resident* a, const Resident* b) { return a->last_used < b->last_used; });
        for (Resident* r : idle) {
          if (need <= avail) break;
          picks.push_back(r);
          avail += r->bytes;
        }
      }
      if (need <= avail) {
        for (Resident* r : picks) {
          for (auto it = residents.begin(); it != residents.end(); ++it)
            if (it->get() == r) {
              held -= r->bytes;
              dying += r->bytes;
              evict->push_back(std::move(*it));
              residents.erase(it);
              break;
            }
          ++st.plans_evicted;
        }
        if (match) {
          match->busy = true;
          *res_out = match;
          q->info.plan_reused = 1;
          ++st.plans_reused;
        } else {
          auto r = std::make_unique<Resident>();
          r->p = q->p;
          r->waves = q->waves;
          r->khash = q->khash;
          r->bytes = need;
          r->busy = true;
          held += need;
          *res_out = r.get();
          residents.push_back(std::move(r));
        }
        peak = std::max(peak, held);
        pending.erase(pending.begin() + (std::ptrdiff_t)i);
        // passing the head counts against it only when this worker could have taken it
        if (i > 0 && (!small_only || pending.front()->level == 0)) ++pending.front()->bypassed;
        *out = q;
        return true;
      }
      if (i == 0 && q->bypassed >= cfg.max_bypass) return false;   // the head waits for memory
    }
    return false;
  }

  // a request the group path takes: class 0, low-rank FP32, device buffers (any
  // buffers in the scheduler test mode, which moves no data)
  bool groupable(const Request* q) const {
    return cfg.group_small > 1 && q->level == 0 && (q->device_io || cfg.simulate_us > 0) &&
           q->p.form == SSM_FORM_LOWRANK && q->p.precision != SSM_TF32X3;
  }

  // a resident plan for q that is idle and matches (caller holds mu)
  Resident* find_match(const Request* q) {
    if (!cfg.cache_plans) return nullptr;
    for (auto& r : residents)
      if (!r->busy && r->khash == q->khash && r->waves == q->waves && same_plan(r->p, q->p) &&
          r->K.size() == (size_t)q->p.P * q->p.Q &&
          std::memcmp(r->K.data(), q->K, sizeof(double) * r->K.size()) == 0)
        return r.get();
    return nullptr;
  }

  // after `first` was admitted: admit up to group_small - 1 more groupable requests
  // waiting behind it that fit the budget without evicting (caller holds mu)
  void admit_group(std::vector<std::pair<Request*, Resident*>>* members) {
    for (size_t i = 0; i < pending.size() && (int)members->size() < cfg.group_small;) {
      Request* q = pending[i];
      if (!groupable(q)) {
        ++i;
        continue;
      }
      Resident* match = find_match(q);
      const int64_t need = match ? 0 : q->footprint;
      if (need > budget - held - dying) {
        ++i;
        continue;
      }
      if (match) {
        match->busy = true;
        q->info.plan_reused = 1;
        ++st.plans_reused;
      } else {
        auto r = std::make_unique<Resident>();
        r->p = q->p;
        r->waves = q->waves;
        r->khash = q->khash;
        r->bytes = need;
        r->busy = true;
        held += need;
        match = r.get();
        residents.push_back(std::move(r));
      }
      peak = std::max(peak, held);
      pending.erase(pending.begin() + (std::ptrdiff_t)i);
      members->push_back({q, match});
    }
  }

  // make q's plan if it has none (on `stream`); records plan_ms and trims the reservation
  ssm_status ensure_plan(Request* q, Resident* res, cudaStream_t stream) {
    if (res->plan) return SSM_OK;
    const Clock::time_point t0 = Clock::now();
    res->K.assign(q->K, q->K + (size_t)q->p.P * q->p.Q);
    SSM_TRY(plan_create(&res->plan, &q->p, q->K, cfg.device, stream, q->waves));
    q->info.plan_ms = ms_between(t0, Clock::now());
    if (cfg.use_graphs) ssm_plan_set_graphs(res->plan, 1);
    // planning's temporaries are gone: keep only the persistent reservation
    ssm_params pr = q->p;
    if (pr.form == SSM_FORM_LOWRANK) pr.rank = res->plan->r;
    int64_t persistent = 0, peak_b = 0;
    if (plan_footprint(pr, true, q->waves, &persistent, &peak_b) == SSM_OK &&
        persistent < res->bytes) {
      std::lock_guard<std::mutex> lk(mu);
      held -= res->bytes - persistent;
      res->bytes = persistent;
    }
    return SSM_OK;
  }

  // solve admitted groupable requests as one group; statuses per member in `out`
  void run_group(std::vector<std::pair<Request*, Resident*>>& members, int slot,
                 std::vector<ssm_status>* out) {
    const bool sim = cfg.simulate_us > 0;
    const size_t n = members.size();
    out->assign(n, SSM_OK);
    if (sim) {
      int longest = 0;
      for (auto& m : members) {
        if (m.second->K.empty()) m.second->K.assign(m.first->K, m.first->K + (size_t)m.first->p.P * m.first->p.Q);
        longest = std::max(longest, m.first->p.max_iter);
        m.first->info.iterations = 0;
        m.first->info.res_primal = m.first->info.res_change = -1;
        m.first->group_size = (int)n;
      }
      std::this_thread::sleep_for(std::chrono::microseconds((int64_t)longest * cfg.simulate_us));
      return;
    }
    cudaStream_t stream = streams[0][slot];
    std::vector<size_t> idx;          // members that go into the group
    std::vector<ssm_plan_t> plans;
    for (size_t i = 0; i < n; ++i) {
      Request* q = members[i].first;
      Resident* res = members[i].second;
      const ssm_status ps = ensure_plan(q, res, stream);
      if (ps != SSM_OK) {
        (*out)[i] = ps;
        continue;
      }
      ssm_plan_s* pl = res->plan;
      pl->p.max_iter = q->p.max_iter;
      pl->p.check_every = q->p.check_every;
      pl->p.tol_primal = q->p.tol_primal;
      pl->p.tol_change = q->p.tol_change;
      if (pl->r > 32 || pl->mask) {       // not a group problem: solved on its own
        (*out)[i] = run(q, res, slot);
        continue;
      }
      idx.push_back(i);
      plans.push_back(pl);
    }
    if (idx.empty()) return;
    ssm_group_t grp = nullptr;
    ssm_status gs = ssm_group_create(&grp, (int)plans.size(), plans.data(), stream);
    std::vector<const float*> Ms;
    std::vector<float*> Fs;
    std::vector<int64_t> lms, lfs;
    std::vector<ssm_info> infos(idx.size());
    for (size_t i : idx) {
      Ms.push_back(members[i].first->M);
      Fs.push_back(members[i].first->F);
      lms.push_back(members[i].first->ldm);
      lfs.push_back(members[i].first->ldf);
    }
    if (gs == SSM_OK)
      gs = ssm_group_solve(grp, Ms.data(), lms.data(), Fs.data(), lfs.data(), infos.data(),
                           stream);
    ssm_group_destroy(grp);
    for (size_t j = 0; j < idx.size(); ++j) {
      Request* q = members[idx[j]].first;
      q->group_size = (int)idx.size();
      if (gs != SSM_OK && gs != SSM_ENOTCONVERGED && infos[j].iterations == 0 &&
          infos[j].status == SSM_OK) {
        (*out)[idx[j]] = gs;              // the group itself failed
        continue;
      }
      (*out)[idx[j]] = (ssm_status)infos[j].status;
      q->info.iterations = infos[j].iterations;
      q->info.res_primal = infos[j].res_primal;
      q->info.res_change = infos[j].res_change;
    }
  }

  // run one admitted request on `slot`'s stream; returns the solve's status
  ssm_status run(Request* q, Resident* res, int slot) {
    const bool sim = cfg.simulate_us > 0;
    cudaStream_t stream = sim ? nullptr : streams[q->level][slot];
    if (!sim) {
      SSM_TRY(ensure_plan(q, res, stream));
    } else if (res->K.empty()) {
      res->K.assign(q->K, q->K + (size_t)q->p.P * q->p.Q);
    }
    if (sim) {
      std::this_thread::sleep_for(
          std::chrono::microseconds((int64_t)q->p.max_iter * cfg.simulate_us));
      q->info.iterations = 0;
      q->info.res_primal = q->info.res_change = -1;
      return SSM_OK;
    }
    // the stopping rule is per request
    res->plan->p.max_iter = q->p.max_iter;
    res->plan->p.check_every = q->p.check_every;
    res->plan->p.tol_primal = q->p.tol_primal;
    res->plan->p.tol_change = q->p.tol_change;
    ssm_info inf{};
    const ssm_status s =
        q->device_io ? ssm_solve(res->plan, q->M, q->ldm, q->F, q->ldf, &inf, stream)
                     : ssm_solve_host(res->plan, q->M, q->ldm, q->F, q->ldf, &inf, stream);
    q->info.iterations = inf.iterations;
    q->info.res_primal = inf.res_primal;
    q->info.res_change = inf.res_change;
    return s;
  }

  // bookkeeping of a finished request (caller holds mu); returns a plan to free
  std::unique_ptr<Resident> finish(Request* q, Resident* res, ssm_status s,
                                   const std::string& err) {
    const bool sim = cfg.simulate_us > 0;
    std::unique_ptr<Resident> drop;
    q->t_done = Clock::now();
    q->info.status = s;
    q->info.group_size = q->group_size;
    q->info.queue_ms = ms_between(q->t_submit, q->t_admit);
    q->info.solve_ms = ms_between(q->t_admit, q->t_done);
    q->info.latency_ms = ms_between(q->t_submit, q->t_done);
    q->error = err;
    q->done = true;
    res->busy = false;
    res->last_used = ++tick;
    const bool bad = s != SSM_OK && s != SSM_ENOTCONVERGED;
    if (!q->info.plan_reused && (res->plan || sim) && !bad) ++st.plans_created;
    if (bad) ++st.failed;
    else ++st.completed;
    // a plan that failed to build, or any plan when caching is off, is freed now
    if (!cfg.cache_plans || (!res->plan && !sim) || bad) {
      for (auto it = residents.begin(); it != residents.end(); ++it)
        if (it->get() == res) {
          held -= res->bytes;
          dying += res->bytes;
          drop = std::move(*it);
          residents.erase(it);
          break;
        }
    }
    --active;
    return drop;
  }

  void worker(int slot) {
    const bool sim = cfg.simulate_us > 0;
    if (!sim) cudaSetDevice(cfg.device);
    for (;;) {
      Request* q = nullptr;
      Resident* res = nullptr;
      std::vector<std::unique_ptr<Resident>> evict;
      std::vector<std::pair<Request*, Resident*>> members;
      bool group = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] {
          return stop || (!pending.empty() && try_admit(slot, &q, &res, &evict));
        });
        if (!q) return;   // stop
        members.push_back({q, res});
        group = groupable(q);
        if (group) admit_group(&members);
        for (auto& m : members) {
          ++active;
          m.first->t_admit = Clock::now();
          m.first->info.order = next_order++;
          m.first->info.slot = slot;
        }
      }
      if (!evict.empty()) {
        int64_t freed = 0;
        for (auto& r : evict) {
          if (r->plan) ssm_destroy(r->plan);
          freed += r->bytes;
        }
        std::lock_guard<std::mutex> lk(mu);
        dying -= freed;
      }
      std::vector<ssm_status> sts;
      std::vector<std::string> errs;
      if (group) {
        run_group(members, slot, &sts);
      } else {
        sts.push_back(run(q, res, slot));
      }
      for (ssm_status s : sts)
        errs.push_back(s == SSM_OK || s == SSM_ENOTCONVERGED ? "" : ssm_last_error());
      std::vector<std::unique_ptr<Resident>> drops;
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < members.size(); ++i) {
          auto d = finish(members[i].first, members[i].second, sts[i], errs[i]);
          if (d) drops.push_back(std::move(d));
        }
      }
      for (auto& d : drops) {
        if (d->plan) ssm_destroy(d->plan);
        std::lock_guard<std::mutex> lk(mu);
        dying -= d->bytes;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

namespace {

ssm_status collect(ssm_server_s* s, std::unique_lock<std::mutex>& lk, int64_t ticket,
                   ssm_request_info* info) {
  auto it = s->requests.find(ticket);
  (void)lk;
  if (it == s->requests.end()) {
    set_error("unknown ticket");
    return SSM_EINVAL;
  }
  if (!it->second->done) return SSM_EPENDING;
  if (info) *info = it->second->info;
  if (!it->second->error.empty()) set_error(it->second->error);
  s->requests.erase(it);
  return SSM_OK;
}

}  // namespace

namespace {

ssm_status submit(ssm_server_t s, const ssm_params* p, const double* K_host, const float* M,
                  int64_t ldm, float* F, int64_t ldf, bool device_io, int64_t* ticket) {
  if (!s || !ticket || !K_host || !M || !F) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  SSM_TRY(validate_params(p));
  int64_t N = 1;
  for (int d = 0; d < p->ndim; ++d) N *= p->dims[d];
  if (ldm < N || ldf < N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  auto q = std::make_unique<Request>();
  q->p = *p;
  q->device_io = device_io;
  q->K = K_host;
  q->M = M;
  q->ldm = ldm;
  q->F = F;
  q->ldf = ldf;
  q->khash = hash_doubles(K_host, (size_t)p->P * p->Q);
  // the reservation always covers the host staging buffers, so that a resident plan can
  // serve host and device requests alike
  int64_t persistent = 0;
  const bool sim = s->cfg.simulate_us > 0;
  int prev = 0;
  if (!sim) {
    SSM_CUDA(cudaGetDevice(&prev));
    SSM_CUDA(cudaSetDevice(s->cfg.device));
  }
  ssm_status fs = plan_footprint(*p, true, 1, &persistent, &q->footprint);
  // the scheduler test mode has no streams: it ranks requests as a device with six
  // priority levels would (GB300's count)
  const int nlev = sim ? 6 : (int)s->streams.size();
  for (int64_t b = std::max<int64_t>(1, s->cfg.small_bytes); q->footprint > b && q->level < nlev - 1;
       b *= 4)
    ++q->level;
  if (fs == SSM_OK && q->footprint > s->cfg.small_bytes && s->cfg.large_waves > 1) {
    q->waves = s->cfg.large_waves;
    fs = plan_footprint(*p, true, q->waves, &persistent, &q->footprint);
  }
  if (sim)
    cudaGetLastError();   // device queries made without a device leave a sticky error
  else
    cudaSetDevice(prev);
  SSM_TRY(fs);
  q->info.footprint = q->footprint;
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->st.submitted;
  if (q->footprint > s->budget) {
    ++s->st.rejected;
    set_error("request footprint (" + std::to_string(q->footprint) +
              " bytes) exceeds the server's HBM budget (" + std::to_string(s->budget) + ")");
    return SSM_ENOMEM;
  }
  q->ticket = s->next_ticket++;
  q->t_submit = Clock::now();
  *ticket = q->ticket;
  s->pending.push_back(q.get());
  s->requests[q->ticket] = std::move(q);
  s->cv_work.notify_all();
  return SSM_OK;
}

}  // namespace

extern "C" {

ssm_status ssm_server_default_config(ssm_server_config* c) {
  if (!c) return SSM_EINVAL;
  std::memset(c, 0, sizeof(*c));
  c->device = 0;
  c->max_active = 4;
  c->hbm_budget = 0;
  c->use_graphs = 1;
  c->cache_plans = 1;
  c->max_bypass = -1;
  c->simulate_us = 0;
  c->small_bytes = (int64_t)1 << 26;
  c->large_waves = 8;
  c->reserved_small = -1;
  c->group_small = 0;
  return SSM_OK;
}

ssm_status ssm_server_create(ssm_server_t* out, const ssm_server_config* c) {
  if (!out || !c) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  *out = nullptr;
  if (c->max_active < 1 || c->max_active > 256) {
    set_error("max_active must be in [1, 256]");
    return SSM_EINVAL;
  }
  if (c->large_waves < 1 || c->large_waves > 64) {
    set_error("large_waves must be in [1, 64]");
    return SSM_EINVAL;
  }
  auto s = std::make_unique<ssm_server_s>();
  s->cfg = *c;
  if (s->cfg.max_bypass < 0) s->cfg.max_bypass = 2 * c->max_active;
  // one worker for class-0 requests when there are at least two; never all of them
  if (s->cfg.reserved_small < 0) s->cfg.reserved_small = c->max_active >= 2 ? 1 : 0;
  s->cfg.reserved_small = std::min(s->cfg.reserved_small, c->max_active - 1);
  const bool sim = c->simulate_us > 0;
  if (sim) {
    if (c->hbm_budget <= 0) {
      set_error("scheduler test mode needs an explicit hbm_budget");
      return SSM_EINVAL;
    }
    s->budget = c->hbm_budget;
  } else {
    int prev = 0;
    SSM_CUDA(cudaGetDevice(&prev));
    SSM_CUDA(cudaSetDevice(c->device));
    size_t free_b = 0, total_b = 0;
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) {
      s->budget = c->hbm_budget > 0 ? std::min<int64_t>(c->hbm_budget, (int64_t)free_b)
                                    : (int64_t)(0.9 * (double)free_b);
      int least = 0, greatest = 0;
      cudaDeviceGetStreamPriorityRange(&least, &greatest);
      const int nlev = std::max(1, least - greatest + 1);   // greatest is the numerically lowest
      s->streams.assign(nlev, std::vector<cudaStream_t>(c->max_active, nullptr));
      for (int l = 0; l < nlev; ++l)
        for (int i = 0; i < c->max_active; ++i)
          if (cudaStreamCreateWithPriority(&s->streams[l][i], cudaStreamNonBlocking,
                                           greatest + l) != cudaSuccess) {
            set_error("cudaStreamCreateWithPriority failed");
            for (auto& v : s->streams)
              for (auto& x : v)
                if (x) cudaStreamDestroy(x);
            cudaSetDevice(prev);
            return SSM_ECUDA;
          }
    }
    cudaSetDevice(prev);
    SSM_CUDA(e);
  }
  s->st.budget = s->budget;
  ssm_server_s* raw = s.get();
  for (int i = 0; i < c->max_active; ++i) raw->workers.emplace_back([raw, i] { raw->worker(i); });
  *out = s.release();
  return SSM_OK;
}

ssm_status ssm_server_submit(ssm_server_t s, const ssm_params* p, const double* K_host,
                             const float* M_host, int64_t ldm, float* F_host, int64_t ldf,
                             int64_t* ticket) {
  return submit(s, p, K_host, M_host, ldm, F_host, ldf, false, ticket);
}

ssm_status ssm_server_submit_device(ssm_server_t s, const ssm_params* p, const double* K_host,
                                    const float* M_dev, int64_t ldm, float* F_dev, int64_t ldf,
                                    int64_t* ticket) {
  return submit(s, p, K_host, M_dev, ldm, F_dev, ldf, true, ticket);
}

ssm_status ssm_server_poll(ssm_server_t s, int64_t ticket, ssm_request_info* info) {
  if (!s) {
    set_error("NULL server");
    return SSM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  return collect(s, lk, ticket, info);
}

ssm_status ssm_server_wait(ssm_server_t s, int64_t ticket, double timeout_ms,
                           ssm_request_info* info) {
  if (!s) {
    set_error("NULL server");
    return SSM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] {
    auto it = s->requests.find(ticket);
    return it == s->requests.end() || it->second->done;
  };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, ready);
  else
    s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
  return collect(s, lk, ticket, info);
}

ssm_status ssm_server_stats_read(ssm_server_t s, ssm_server_stats* out) {
  if (!s || !out) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_held = s->held;
  out->peak_bytes_held = s->peak;
  out->budget = s->budget;
  out->active = s->active;
  out->pending = (int)s->pending.size();
  return SSM_OK;
}

ssm_status ssm_server_destroy(ssm_server_t s) {
  if (!s) return SSM_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->active == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  const bool sim = s->cfg.simulate_us > 0;
  if (!sim) cudaSetDevice(s->cfg.device);
  for (auto& r : s->residents)
    if (r->plan) ssm_destroy(r->plan);
  for (auto& v : s->streams)
    for (auto& st : v)
      if (st) cudaStreamDestroy(st);
  delete s;
  return SSM_OK;
}

}  // extern "C"
