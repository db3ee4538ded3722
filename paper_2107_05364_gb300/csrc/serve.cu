// Request serving: relax and field-sweep jobs on many geometries,
// continuously batched.
//
// A worker thread owns all device work of a server.  Each geometry that has
// work becomes "resident": its tensor is assembled once and kept on the
// device, with an integrator of B simulation slots on its own stream (an
// engine).  Jobs queue per geometry in arrival order and enter free slots
// between graph replays: a slot whose simulation finished (torque below
// tolerance, time cap, or failure) is retired and refilled while the other
// slots keep integrating, so requests that arrive while others run join the
// batch as slots free up.  Engines of different geometries run on different
// streams and overlap on the device.  Residency is limited by an HBM budget
// (tensor + batch state); idle engines are evicted least-recently-used when a
// waiting geometry needs room.
//
// A relax job integrates its simulation until the torque criterion of
// Brown's equation (Eq. 2) holds or its time cap is spent.  A sweep job is
// the field loop of Sec. 4.1 as one request: its slot is relaxed at each
// applied field of its schedule in turn, the state carried over; between
// values the slot is re-admitted in place (new field, fresh relax goal, k1
// re-evaluated) while the other slots keep running, and <m> and the torque
// at the end of every value are kept for the caller.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <list>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mt_internal.cuh"

namespace mt {
// slot-level integrator control (llg.cu)
size_t integ_ctl_bytes(const mt_integrator *I);
void *integ_stream(const mt_integrator *I);
mt_status integ_admit(mt_integrator *I, int b, const float *m0_host, double alpha, const double *Ha, double tol,
                      double t_max);
mt_status integ_readmit(mt_integrator *I, int b, const double *Ha, double tol, double t_max);
void integ_slot_mavg(const void *ctl_host, int b, double m[3]);
mt_status integ_init_fresh(mt_integrator *I);
mt_status integ_replay(mt_integrator *I, int k);
mt_status integ_poll(mt_integrator *I, void *ctl_host, cudaEvent_t ev);
bool integ_slot_done(const void *ctl_host, int b, mt_stats *st);
mt_status integ_fetch_slot(mt_integrator *I, int b, float *m_host);
mt_status integ_create_idle(mt_tensor *T, const mt_llg_params *p, const mt_ode_opts *o, int B, mt_integrator **out);
size_t tensor_bytes_for(int64_t n, int prec, int layout);
}  // namespace mt

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  int geometry = 0;
  int kind = MT_JOB_RELAX;
  double alpha = 0, tol = 0, t_max = 0;
  double Ha[3] = {0, 0, 0};
  std::vector<double> fields;  // sweep: [n_fields][3]
  std::vector<double> sweep;   // sweep: [n_fields][4] = <m>, torque at the end of each value
  int64_t value = 0;           // sweep: the value in progress
  mt_stats acc{};              // sweep: counters of the values already done
  int64_t converged = 0;       // sweep: values that met the torque tolerance
  std::vector<float> m;        // m0 in, final state out
  mt_job_result res{};
  bool done = false;
};

struct Engine {
  mt_tensor *T = nullptr;
  mt_integrator *I = nullptr;
  int B = 0;
  int64_t n = 0;
  size_t bytes = 0;
  std::vector<std::shared_ptr<Job>> slot;
  float *m_in = nullptr;   // pinned, B * 3n
  float *m_out = nullptr;  // pinned, B * 3n
  void *ctl = nullptr;     // pinned control copies
  cudaEvent_t ev = nullptr;
  bool inflight = false;
  bool need_fresh = false;  // slots admitted or re-admitted since the last k1
  int occupied = 0;
};

struct Geometry {
  int id = 0;
  int64_t n = 0;
  std::vector<double> centre, edge, Ms, Aex, Ku, axis;
  std::vector<int32_t> nbr;
  mt_tiles *tiles = nullptr;
  std::unique_ptr<Engine> eng;
  std::deque<std::shared_ptr<Job>> waiting;
  double last_used = 0;
};

}  // namespace

struct mt_server {
  mt_ctx *ctx = nullptr;
  mt_server_opts o{};
  size_t budget = 0;
  size_t in_use = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> inbox;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::unique_ptr<Geometry>> geoms;
  uint64_t next_id = 1;
  bool stop = false;
  mt_server_stats stats{};
  std::string fatal;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

size_t engine_state_bytes(int64_t n, int B) {
  // state, two stage inputs, H_d, seven stage derivatives (FP32, B x 3n each),
  // operand copies and reductions: a conservative estimate
  return (size_t)B * 3 * n * sizeof(float) * 14 + ((size_t)4 << 20);
}

void destroy_engine(mt_server *S, Geometry &g) {
  Engine *e = g.eng.get();
  if (!e) return;
  if (e->I) mt_integrator_destroy(e->I);
  if (e->T) mt_tensor_destroy(e->T);
  if (e->m_in) cudaFreeHost(e->m_in);
  if (e->m_out) cudaFreeHost(e->m_out);
  if (e->ctl) cudaFreeHost(e->ctl);
  if (e->ev) cudaEventDestroy(e->ev);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use -= e->bytes;
  }
  g.eng.reset();
}

void fail_job(mt_server *S, const std::shared_ptr<Job> &j, mt_status st) {
  std::lock_guard<std::mutex> lk(S->mu);
  j->res.status = st;
  j->res.t_done = S->now();
  j->done = true;
  S->stats.failed++;
  S->cv_done.notify_all();
}

// make g resident: evict idle engines (least recently used) until the tensor
// and batch state fit the budget.  Returns false if it cannot be done now.
bool make_resident(mt_server *S, Geometry &g, const std::vector<Geometry *> &all) {
  const size_t need = mt::tensor_bytes_for(g.n, S->o.prec, S->o.layout) + engine_state_bytes(g.n, S->o.max_batch);
  if (need > S->budget) {
    // can never fit: fail the geometry's waiting jobs
    while (!g.waiting.empty()) {
      fail_job(S, g.waiting.front(), MT_ENOMEM);
      g.waiting.pop_front();
    }
    return false;
  }
  while (S->in_use + need > S->budget) {
    Geometry *victim = nullptr;
    for (Geometry *h : all)
      if (h != &g && h->eng && h->eng->occupied == 0 && !h->eng->inflight && h->waiting.empty() &&
          (!victim || h->last_used < victim->last_used))
        victim = h;
    if (!victim) return false;  // everything resident is busy: wait
    destroy_engine(S, *victim);
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.evictions++;
  }
  if (!g.tiles) {
    mt_status st = mt_tiles_create(S->ctx, g.n, g.centre.data(), g.edge.data(), g.Ms.data(), g.Aex.data(),
                                   g.Ku.data(), g.axis.data(), g.nbr.empty() ? nullptr : g.nbr.data(), &g.tiles);
    if (st != MT_OK) {
      // an invalid geometry never becomes resident: its jobs fail with the
      // creation status instead of waiting for room forever
      g.tiles = nullptr;
      while (!g.waiting.empty()) {
        fail_job(S, g.waiting.front(), st);
        g.waiting.pop_front();
      }
      return false;
    }
  }
  std::unique_ptr<Engine> e(new Engine());
  e->B = S->o.max_batch;
  e->n = g.n;
  e->slot.resize(e->B);
  // the half storage (tiles of one shape) pays for one or two simulations
  // per pass; an engine of 3 or more slots streams every block
  const int layout =
      (S->o.layout == MT_LAYOUT_STREAM && e->B >= 3) ? (int)MT_LAYOUT_STREAM_FULL : (int)S->o.layout;
  mt_status st = mt_demag_assemble_ex(g.tiles, (mt_prec)S->o.prec, layout, &e->T);
  if (st == MT_OK) {
    std::vector<double> alpha(e->B, 0.5), Ha(3 * e->B, 0.0);
    mt_llg_params p{S->o.gamma, alpha.data(), Ha.data(), S->o.form, 1, nullptr};
    st = mt::integ_create_idle(e->T, &p, &S->o.ode, e->B, &e->I);
  }
  const size_t vec = sizeof(float) * 3 * (size_t)g.n * e->B;
  if (st == MT_OK && (cudaMallocHost(&e->m_in, vec) != cudaSuccess || cudaMallocHost(&e->m_out, vec) != cudaSuccess ||
                      cudaMallocHost(&e->ctl, mt::integ_ctl_bytes(e->I)) != cudaSuccess ||
                      cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming) != cudaSuccess))
    st = MT_ENOMEM;
  e->bytes = need;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->in_use += need;
  }
  g.eng = std::move(e);
  if (st != MT_OK) {
    destroy_engine(S, g);
    while (!g.waiting.empty()) {
      fail_job(S, g.waiting.front(), st);
      g.waiting.pop_front();
    }
    return false;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->stats.assemblies++;
  return true;
}

// Retire slot b: the job's final state (already copied to e.m_out) and its
// outcome `st` (counters summed over a sweep's values).
void complete(mt_server *S, Geometry &g, int b, const mt_stats &st, int64_t values_done, int64_t values_converged) {
  Engine &e = *g.eng;
  std::shared_ptr<Job> j = e.slot[b];
  e.slot[b].reset();
  e.occupied--;
  const size_t n3 = 3 * (size_t)g.n;
  std::memcpy(j->m.data(), e.m_out + b * n3, sizeof(float) * n3);
  std::lock_guard<std::mutex> lk(S->mu);
  j->res.status = st.status;
  j->res.n_accept = st.n_accept;
  j->res.n_reject = st.n_reject;
  j->res.n_rhs = st.n_rhs;
  j->res.t_sim = st.t;
  j->res.tau = st.tau;
  j->res.t_done = S->now();
  j->res.values_done = values_done;
  j->res.values_converged = values_converged;
  j->done = true;
  if (st.status == MT_OK) S->stats.completed++;
  else S->stats.failed++;
  S->cv_done.notify_all();
}

// A slot reported done.  Relax job: finished.  Sweep job: record the value's
// <m> and torque; a failure (non-finite state, step cap) ends the job, the
// time cap does not (as a held field value, the torque tells); with values
// left the slot is re-admitted at the next field and true is returned.
bool sweep_advance(Engine &e, int b, const mt_stats &st, mt_stats *final_st, int64_t *converged) {
  Job &j = *e.slot[b];
  if (j.kind != MT_JOB_SWEEP) {
    *final_st = st;
    *converged = (st.status == MT_OK) ? 1 : 0;
    return false;
  }
  const int64_t nf = (int64_t)j.fields.size() / 3;
  double mv[3];
  mt::integ_slot_mavg(e.ctl, b, mv);
  double *row = &j.sweep[4 * (size_t)j.value];
  for (int q = 0; q < 3; ++q) row[q] = mv[q];
  row[3] = st.tau;
  j.acc.n_accept += st.n_accept;
  j.acc.n_reject += st.n_reject;
  j.acc.n_rhs += st.n_rhs;
  j.acc.t += st.t;
  j.acc.tau = st.tau;
  if (st.status == MT_OK) j.converged++;
  const bool ok = st.status == MT_OK || (st.status == MT_ENOCONV && st.t >= j.t_max * (1.0 - 1e-12));
  j.value++;
  if (ok && j.value < nf && mt::integ_readmit(e.I, b, &j.fields[3 * (size_t)j.value], j.tol, j.t_max) == MT_OK)
    return true;
  *final_st = j.acc;
  final_st->status = ok ? MT_OK : st.status;
  final_st->pad = 0;
  *converged = j.converged;
  return false;
}

void worker_loop(mt_server *S) {
  cudaSetDevice(S->ctx->device);
  const int K = S->o.replays_per_poll > 0 ? S->o.replays_per_poll : 16;
  for (;;) {
    // 1. intake (geometries may be added concurrently: work on a snapshot)
    std::vector<Geometry *> all;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      bool busy = false;
      for (auto &g : S->geoms)
        if (!g->waiting.empty() || (g->eng && (g->eng->occupied > 0 || g->eng->inflight))) busy = true;
      if (!busy && S->inbox.empty() && !S->stop)
        S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      if (S->stop) break;
      while (!S->inbox.empty()) {
        auto j = S->inbox.front();
        S->inbox.pop_front();
        S->geoms[j->geometry]->waiting.push_back(j);
      }
      for (auto &g : S->geoms) all.push_back(g.get());
    }
    // 2. completions of engines whose poll has landed
    for (Geometry *gp : all) {
      Geometry &g = *gp;
      Engine *e = g.eng.get();
      if (!e || !e->inflight) continue;
      if (cudaEventQuery(e->ev) != cudaSuccess) continue;
      e->inflight = false;
      struct Fin {
        int b;
        mt_stats st;
        int64_t values, converged;
      };
      std::vector<Fin> fin;
      for (int b = 0; b < e->B; ++b) {
        mt_stats st{};
        if (!e->slot[b] || !mt::integ_slot_done(e->ctl, b, &st)) continue;
        Fin f{b, {}, 0, 0};
        if (sweep_advance(*e, b, st, &f.st, &f.converged)) {
          e->need_fresh = true;  // next value of a sweep: k1 at the new field
          continue;
        }
        f.values = e->slot[b]->kind == MT_JOB_SWEEP ? e->slot[b]->value : 1;
        fin.push_back(f);
      }
      if (!fin.empty()) {
        for (auto &f : fin) mt::integ_fetch_slot(e->I, f.b, e->m_out + f.b * 3 * (size_t)g.n);
        cudaStreamSynchronize((cudaStream_t)mt::integ_stream(e->I));
        for (auto &f : fin) complete(S, g, f.b, f.st, f.values, f.converged);
      }
      g.last_used = S->now();
    }
    // 3. residency and admission, oldest waiting geometry first
    std::vector<Geometry *> order;
    for (Geometry *g : all)
      if (!g->waiting.empty()) order.push_back(g);
    std::sort(order.begin(), order.end(), [](Geometry *a, Geometry *b) {
      return a->waiting.front()->res.t_submit < b->waiting.front()->res.t_submit;
    });
    // a server-wide cap on running jobs (max_running > 0) admits strictly in
    // arrival order: the oldest waiting job goes first or nothing does
    const int cap = S->o.max_running;
    int running = 0;
    for (Geometry *g : all)
      if (g->eng) running += g->eng->occupied;
    for (Geometry *gp : order) {
      Geometry &g = *gp;
      if (cap > 0 && running >= cap) break;
      if (!g.eng && !make_resident(S, g, all)) {
        if (cap > 0) break;
        continue;
      }
      Engine *e = g.eng.get();
      if (!e || e->inflight) {
        if (cap > 0) break;
        continue;
      }
      bool admitted = false;
      for (int b = 0; b < e->B && !g.waiting.empty() && (cap <= 0 || running < cap); ++b) {
        if (e->slot[b]) continue;
        std::shared_ptr<Job> j = g.waiting.front();
        g.waiting.pop_front();
        const size_t n3 = 3 * (size_t)g.n;
        std::memcpy(e->m_in + b * n3, j->m.data(), sizeof(float) * n3);
        const double *ha = j->kind == MT_JOB_SWEEP ? j->fields.data() : j->Ha;
        if (mt::integ_admit(e->I, b, e->m_in + b * n3, j->alpha, ha, j->tol, j->t_max) != MT_OK) {
          fail_job(S, j, MT_ECUDA);
          continue;
        }
        {
          std::lock_guard<std::mutex> lk(S->mu);
          j->res.t_start = S->now();
        }
        e->slot[b] = j;
        e->occupied++;
        running++;
        admitted = true;
      }
      if (admitted) e->need_fresh = true;
      g.last_used = S->now();
    }
    // 4. launch work on every engine with running slots
    bool any_inflight = false;
    for (Geometry *gp : all) {
      Engine *e = gp->eng.get();
      if (!e) continue;
      if (!e->inflight && e->occupied > 0) {
        if (e->need_fresh) {
          mt::integ_init_fresh(e->I);  // one product for every new or re-admitted slot
          e->need_fresh = false;
        }
        mt::integ_replay(e->I, K);
        mt::integ_poll(e->I, e->ctl, e->ev);
        e->inflight = true;
      }
      any_inflight = any_inflight || e->inflight;
    }
    if (any_inflight) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  // drain device work before the engines go away
  for (auto &g : S->geoms)
    if (g->eng) cudaStreamSynchronize((cudaStream_t)mt::integ_stream(g->eng->I));
}

}  // namespace

extern "C" {

mt_status mt_server_create(mt_ctx *ctx, const mt_server_opts *opts, mt_server **out) {
  MT_CHECK(ctx && opts && out, MT_EINVAL, "mt_server_create: NULL argument");
  MT_CHECK(opts->max_batch >= 1 && opts->max_batch <= 128, MT_EINVAL, "mt_server_create: max_batch in 1..128");
  MT_CHECK(opts->prec >= MT_F32 && opts->prec <= MT_BF16_SPLIT, MT_EINVAL,
           "mt_server_create: precision must be FP32, BF16 or split BF16");
  MT_CHECK(opts->layout == MT_LAYOUT_STREAM || opts->layout == MT_LAYOUT_DENSE || opts->layout == MT_LAYOUT_STREAM6 ||
               opts->layout == MT_LAYOUT_STREAM_FULL || opts->layout == MT_LAYOUT_STREAM_HALF,
           MT_EINVAL, "mt_server_create: bad layout %d", (int)opts->layout);
  MT_CHECK(opts->layout != MT_LAYOUT_DENSE || opts->prec != MT_F32, MT_EINVAL,
           "mt_server_create: the dense layout stores BF16 or split BF16");
  MT_CHECK(opts->max_running >= 0, MT_EINVAL, "mt_server_create: max_running must be >= 0");
  mt_server *S = new mt_server();
  S->ctx = ctx;
  ctx->refs++;
  S->o = *opts;
  S->budget = opts->hbm_budget_bytes ? std::min(opts->hbm_budget_bytes, ctx->budget) : ctx->budget;
  S->t0 = Clock::now();
  S->stats.budget = S->budget;
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return MT_OK;
}

mt_status mt_server_add_geometry(mt_server *S, int64_t n, const double *centre, const double *edge, const double *Ms,
                                 const double *Aex, const double *Ku, const double *axis, const int32_t *nbr,
                                 int32_t *geometry_id) {
  MT_CHECK(S && geometry_id && n >= 1 && centre && edge && Ms && Aex && Ku && axis, MT_EINVAL,
           "mt_server_add_geometry: bad argument");
  std::unique_ptr<Geometry> g(new Geometry());
  g->n = n;
  g->centre.assign(centre, centre + 3 * n);
  g->edge.assign(edge, edge + 3 * n);
  g->Ms.assign(Ms, Ms + n);
  g->Aex.assign(Aex, Aex + n);
  g->Ku.assign(Ku, Ku + n);
  g->axis.assign(axis, axis + 3 * n);
  if (nbr) g->nbr.assign(nbr, nbr + 6 * n);
  std::lock_guard<std::mutex> lk(S->mu);
  g->id = (int)S->geoms.size();
  *geometry_id = g->id;
  S->geoms.push_back(std::move(g));
  return MT_OK;
}

mt_status mt_server_submit(mt_server *S, const mt_job *job, uint64_t *job_id) {
  MT_CHECK(S && job && job_id && job->m0, MT_EINVAL, "mt_server_submit: NULL argument");
  std::shared_ptr<Job> j = std::make_shared<Job>();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    MT_CHECK(job->geometry >= 0 && job->geometry < (int)S->geoms.size(), MT_EINVAL,
             "mt_server_submit: unknown geometry %d", job->geometry);
    MT_CHECK(job->tol > 0 && job->t_max > 0 && std::isfinite(job->alpha), MT_EINVAL,
             "mt_server_submit: tol and t_max must be positive");
    MT_CHECK(job->kind == MT_JOB_RELAX || job->kind == MT_JOB_SWEEP, MT_EINVAL, "mt_server_submit: unknown kind %d",
             job->kind);
    if (job->kind == MT_JOB_SWEEP) {
      MT_CHECK(job->fields && job->n_fields >= 1 && job->n_fields <= ((int64_t)1 << 24), MT_EINVAL,
               "mt_server_submit: a sweep needs 1 .. 2^24 field values");
      for (int64_t q = 0; q < 3 * job->n_fields; ++q)
        MT_CHECK(std::isfinite(job->fields[q]), MT_EINVAL, "mt_server_submit: non-finite field value");
      j->fields.assign(job->fields, job->fields + 3 * job->n_fields);
      j->sweep.assign(4 * (size_t)job->n_fields, std::numeric_limits<double>::quiet_NaN());
    } else {
      for (int c = 0; c < 3; ++c)
        MT_CHECK(std::isfinite(job->Ha[c]), MT_EINVAL, "mt_server_submit: non-finite applied field");
    }
    const int64_t n = S->geoms[job->geometry]->n;
    j->m.assign(job->m0, job->m0 + 3 * n);
    j->id = S->next_id++;
    j->geometry = job->geometry;
    j->kind = job->kind;
    j->alpha = job->alpha;
    j->tol = job->tol;
    j->t_max = job->t_max;
    for (int c = 0; c < 3; ++c) j->Ha[c] = job->Ha[c];
    j->res.status = MT_EBUSY;  // in progress
    j->res.geometry = job->geometry;
    j->res.t_submit = S->now();
    S->jobs[j->id] = j;
    S->inbox.push_back(j);
    S->stats.submitted++;
    *job_id = j->id;
  }
  S->cv_work.notify_one();
  return MT_OK;
}

mt_status mt_server_wait(mt_server *S, uint64_t job_id, double timeout_s, mt_job_result *res, float *m_out,
                         double *sweep_out) {
  MT_CHECK(S, MT_EINVAL, "mt_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  MT_CHECK(it != S->jobs.end(), MT_EINVAL, "mt_server_wait: unknown job %llu", (unsigned long long)job_id);
  std::shared_ptr<Job> j = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(std::max(0.0, timeout_s)));
  while (!j->done) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !j->done) {
      mt::set_error("mt_server_wait: job %llu not finished within %.3f s", (unsigned long long)job_id, timeout_s);
      return MT_ETIMEOUT;
    }
  }
  if (res) *res = j->res;
  if (m_out) std::memcpy(m_out, j->m.data(), sizeof(float) * j->m.size());
  if (sweep_out && !j->sweep.empty()) std::memcpy(sweep_out, j->sweep.data(), sizeof(double) * j->sweep.size());
  S->jobs.erase(it);
  return MT_OK;
}

mt_status mt_server_get_stats(mt_server *S, mt_server_stats *st) {
  MT_CHECK(S && st, MT_EINVAL, "mt_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->stats;
  st->bytes_in_use = S->in_use;
  int64_t r = 0;
  for (auto &g : S->geoms) r += g->eng ? 1 : 0;
  st->resident = r;
  return MT_OK;
}

void mt_server_destroy(mt_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &g : S->geoms) {
    destroy_engine(S, *g);
    if (g->tiles) mt_tiles_destroy(g->tiles);
  }
  mt::ctx_release(S->ctx);
  delete S;
}

}  // extern "C"
