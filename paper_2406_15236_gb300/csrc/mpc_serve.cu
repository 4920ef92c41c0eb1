// Serving: a continuous-batching request loop over a batch (C ABI in include/mpc.h).
//
// Jobs wait in arrival order.  Between chunks of steps the loop admits every job that
// has arrived and fits the HBM budget (the batch arena), retires jobs that reached their
// step count (their observables become a Green-Kubo viscosity, their memory returns to
// the arena once the queued work is past it), picks the resident jobs that step in the
// next chunk (by default the least remaining work first, or the oldest first, until the
// GPU is full, or by remaining time minus waiting time; the others hold through their
// step limits), and enqueues the chunk, sized
// so that the next stepping job to finish ends on the chunk boundary.  While a chunk runs, the loop keeps
// admitting arrivals: box creation runs on the batch's side stream and overlaps the
// chunk, and the new members join the next chunk.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "mpc.h"
#include "mpc_host.h"
#include "mpc_internal.h"

using namespace mpc;
using namespace mpc::host;

namespace {

thread_local std::string g_server_create_error;

// default particles the stepping jobs of a chunk should hold: about twenty waves of
// 640-particle bricks on 152 SMs at five CTAs each, so that several jobs step together
// and the last partial wave of one launch overlaps the next (measured on the serving
// trace: 1M-particle fills leave the GPU waiting on launch tails, 16M recover them)
constexpr int64_t kFillParticles = 16000000;

struct Job {
  mpc_job spec{};
  mpc_job_result res{};
  mpc_handle h = nullptr;
  std::vector<double> series;  // kept rows (MPC_JOB_KEEP_SERIES)
  std::vector<uint32_t> X, id;
  std::vector<float> V;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct mpc_server_s {
  mpc_server_config cfg{};
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // result copies that must not wait for queued chunks
  bool det = false, sequential = false, share_all = false, first_come = false, aged = false,
       backfill = false, priority_head = false;
  cudaStream_t head_stream = nullptr;  // priority_head: the head job's own steps
  cudaEvent_t head_done = nullptr;
  cudaEvent_t head_ready = nullptr;  // the batch stream's creations, before the head steps
  Job* head = nullptr;
  double work_done = 0.0;  // particle-steps of the chunks run so far (aged ordering)
  int64_t fill = kFillParticles;
  int chunk = 100;
  mpc_batch batch = nullptr;
  std::vector<Job> jobs;
  size_t next_queued = 0;  // jobs before this index are admitted, done or failed
  bool started = false;
  std::chrono::steady_clock::time_point t0;
  cudaEvent_t chunk_start = nullptr, chunk_done = nullptr;
  mpc_server_stats stats{};
  bool gap_open = false;
  double gap_from = 0.0;
  std::string err;
};

namespace {

mpc_status sfail(mpc_server s, mpc_status st, const std::string& msg) {
  if (s) s->err = msg;
  else g_server_create_error = msg;
  return st;
}

// Green-Kubo shear viscosity from per-step stress rows (Sec. II observables; the MPC
// stress of the streaming and collision parts): eta = (V h / kT) [C(0)/2 + sum_{k=1..K}
// C(k)], C the autocorrelation of each off-diagonal stress about its mean, averaged
// over xy, yx, yz, zy, zx, xz; K = one time unit of steps, round(1 / h): the MPC stress
// autocorrelation has decayed by then (windows of half, one and two time units give the
// same viscosity within the noise), and longer windows only add noise.
void green_kubo(const mpc_params& p, int64_t N, const double* rows, int64_t n, double& eta,
                double& temp) {
  const double vol = (double)p.L[0] * p.L[1] * p.L[2];
  const int kin_of[6] = {4, 4, 5, 5, 6, 6};
  const int col_of[6] = {7, 8, 9, 10, 11, 12};
  temp = 0.0;
  for (int64_t r = 0; r < n; ++r) {
    const double* w = rows + r * kObsWidth;
    const double p2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    temp += N > 1 ? p.m * (w[3] - p2 / (double)N) / (3.0 * ((double)N - 1.0)) : 0.0;
  }
  temp = n > 0 ? temp / (double)n : 0.0;
  eta = 0.0;
  if (n < 4) return;
  const int64_t K = std::min<int64_t>(std::max<int64_t>(std::llround(1.0 / p.h), 1), n - 1);
  std::vector<double> sig((size_t)n);
  double acc = 0.0;
  for (int c = 0; c < 6; ++c) {
    double mean = 0.0;
    for (int64_t r = 0; r < n; ++r) {
      const double* w = rows + r * kObsWidth;
      sig[(size_t)r] = -(p.m / vol) * (w[kin_of[c]] + w[col_of[c]] / p.h);
      mean += sig[(size_t)r];
    }
    mean /= (double)n;
    for (double& v : sig) v -= mean;
    double sum = 0.0;
    for (int64_t k = 0; k <= K; ++k) {
      double ck = 0.0;
      for (int64_t r = 0; r + k < n; ++r) ck += sig[(size_t)r] * sig[(size_t)(r + k)];
      ck /= (double)(n - k);
      sum += (k == 0) ? 0.5 * ck : ck;
    }
    acc += sum;
  }
  eta = (vol * p.h / p.kT) * acc / 6.0;
}

mpc_params job_params(const mpc_server s, const Job& j) {
  mpc_params q = j.spec.params;
  q.flags |= MPC_FLAG_OBSERVABLES;
  if (s->det) q.flags |= MPC_FLAG_DETERMINISTIC;
  q.obs_ring = (int32_t)j.spec.steps;
  return q;
}

// copies the observables (and, if kept, the state) of a job whose box reached its step
// count to the host; the series goes through the server's side stream so that it does
// not wait for work queued on the batch stream
mpc_status fetch(mpc_server s, Job& j) {
  mpc_handle h = j.h;
  const int64_t n = j.spec.steps;
  j.series.resize((size_t)n * kObsWidth);
  if (cudaMemcpyAsync(j.series.data(), h->obs_series, j.series.size() * sizeof(double),
                      cudaMemcpyDeviceToHost, s->side) != cudaSuccess ||
      cudaStreamSynchronize(s->side) != cudaSuccess)
    return sfail(s, MPC_ECUDA, "copy of the job's observables failed");
  if (j.spec.keep & MPC_JOB_KEEP_STATE) {
    j.X.resize((size_t)h->N * 3);
    j.V.resize((size_t)h->N * 3);
    j.id.resize((size_t)h->N);
    // the readout's temporary buffers come from cudaMalloc, not from the budget that
    // the resident jobs fill
    const bool arena = h->has_alloc;
    h->has_alloc = false;
    const mpc_status st = mpc_get_state(h, j.X.data(), j.V.data(), j.id.data(), nullptr, nullptr, 0);
    h->has_alloc = arena;
    if (st != MPC_OK) return sfail(s, st, "job state: " + h->err);
  }
  return MPC_OK;
}

// host-side analysis of fetched observables; the job is done afterwards
void analyse(mpc_server s, Job& j) {
  green_kubo(job_params(s, j), j.res.n_particles, j.series.data(), j.spec.steps, j.res.eta_gk,
             j.res.temperature);
  if (!(j.spec.keep & MPC_JOB_KEEP_SERIES)) std::vector<double>().swap(j.series);
  j.res.status = MPC_JOB_DONE;
  j.res.steps = j.spec.steps;
  j.res.finish_s = now_s(s->t0);
}

void fail_job(Job& j, mpc_status st, double t) {
  j.res.status = MPC_JOB_FAILED;
  j.res.error = st;
  j.res.finish_s = t;
}

// admits arrived jobs in order while they fit; a job that does not fit is passed by
// later ones (it keeps its place for the next round)
void admit(mpc_server s) {
  const double t = now_s(s->t0);
  int active = 0;
  for (const Job& j : s->jobs) active += j.res.status == MPC_JOB_RUNNING;
  for (size_t i = s->next_queued; i < s->jobs.size(); ++i) {
    Job& j = s->jobs[i];
    if (j.res.status != MPC_JOB_QUEUED) continue;
    if (j.spec.arrival_s > t) break;  // jobs are kept in arrival order
    if (active >= (s->cfg.max_active > 0 ? s->cfg.max_active : kMaxBatchBoxes)) break;
    const mpc_params q = job_params(s, j);
    uint64_t steady = 0, peak = 0;
    if (mpc_footprint(&q, &steady, &peak) != MPC_OK) {
      fail_job(j, MPC_EINVAL, t);
      continue;
    }
    if (peak > s->cfg.hbm_budget_bytes) {
      fail_job(j, MPC_ENOMEM, t);  // would not fit even alone
      continue;
    }
    mpc_handle h = nullptr;
    const mpc_status st = mpc_batch_add(s->batch, &q, &h);
    if (st == MPC_ENOMEM) continue;  // wait for memory; later jobs may fit
    if (st != MPC_OK || mpc_set_step_limit(h, j.spec.steps) != MPC_OK) {
      if (h) mpc_batch_remove(s->batch, h);
      fail_job(j, st != MPC_OK ? st : MPC_ECUDA, t);
      continue;
    }
    j.h = h;
    j.res.status = MPC_JOB_RUNNING;
    j.res.admit_s = now_s(s->t0);
    j.res.n_particles = h->N;
    ++active;
  }
  while (s->next_queued < s->jobs.size() && s->jobs[s->next_queued].res.status != MPC_JOB_QUEUED)
    ++s->next_queued;
}

bool all_finished(const mpc_server s) {
  for (const Job& j : s->jobs)
    if (j.res.status == MPC_JOB_QUEUED || j.res.status == MPC_JOB_RUNNING) return false;
  return true;
}

// The head job (MPC_SERVER_PRIORITY_HEAD): detached from the batch, all its remaining
// steps enqueued at once on the high-priority stream, so it runs at its own pace between
// the batch's chunks instead of pausing at each chunk boundary.
mpc_status start_head(mpc_server s, Job* j) {
  s->head = j;
  // the batch stream waits for member creations; no chunk is pending when a head starts
  if (cudaEventRecord(s->head_ready, s->stream) != cudaSuccess ||
      cudaStreamWaitEvent(s->head_stream, s->head_ready, 0) != cudaSuccess)
    return sfail(s, MPC_ECUDA, "event record failed");
  j->h->stream = s->head_stream;
  batch_set_detached(j->h, true);
  if (mpc_status st = mpc_set_step_limit(j->h, j->spec.steps); st != MPC_OK)
    return sfail(s, st, "step limit: " + j->h->err);
  const int64_t n = j->spec.steps - j->h->target_step;
  if (mpc_status st = mpc_step(j->h, n); st != MPC_OK) return sfail(s, st, "head job: " + j->h->err);
  if (cudaEventRecord(s->head_done, s->head_stream) != cudaSuccess)
    return sfail(s, MPC_ECUDA, "event record failed");
  s->work_done += (double)n * (double)j->h->N;
  return MPC_OK;
}

// particle-steps per second of the runs so far (the order keys' time scale)
double work_rate(const mpc_server s) {
  return s->stats.gpu_ms > 0.0 ? s->work_done / (1e-3 * s->stats.gpu_ms) : 4e10;
}

mpc_status run_batched(mpc_server s, double deadline) {
  std::vector<Job*> fetched;  // results on the host, analysis pending
  for (;;) {
    admit(s);
    if (fetched.empty() && all_finished(s)) return MPC_OK;
    if (now_s(s->t0) > deadline) {
      for (Job* j : fetched) analyse(s, *j);
      return sfail(s, MPC_ETIMEOUT, "server run timed out");
    }
    // the jobs that step in this chunk: all resident jobs, or (default) those with the
    // least remaining work -- or the oldest -- until they fill the GPU; the others hold
    // at their step
    std::vector<Job*> resident;  // (retired jobs await analysis with h = NULL)
    for (Job& j : s->jobs)
      if (j.res.status == MPC_JOB_RUNNING && j.h && &j != s->head) resident.push_back(&j);
    if (s->priority_head && !s->head && !resident.empty()) {
      // the oldest resident job (jobs are kept in arrival order) becomes the head
      TRY(start_head(s, resident.front()));
      resident.erase(resident.begin());
    }
    if (s->aged) {
      // remaining time at the measured rate minus the time already waited: a fresh short
      // job goes first, a job that has waited as long as it still needs overtakes it
      const double rate = work_rate(s);
      const double t = now_s(s->t0);
      auto key = [&](const Job* j) {
        return (double)(j->spec.steps - j->h->target_step) * (double)j->h->N / rate -
               (t - j->spec.arrival_s);
      };
      std::stable_sort(resident.begin(), resident.end(),
                       [&](const Job* a, const Job* b) { return key(a) < key(b); });
    } else if (!s->first_come) {
      std::stable_sort(resident.begin(), resident.end(), [](const Job* a, const Job* b) {
        const double wa = (double)(a->spec.steps - a->h->target_step) * (double)a->h->N;
        const double wb = (double)(b->spec.steps - b->h->target_step) * (double)b->h->N;
        return wa < wb;
      });
    }  // else arrival order (jobs are kept in arrival order)
    int64_t min_left = INT64_MAX, filled = 0;
    double chunk_work = 0.0;  // particles stepping in this chunk
    for (Job* j : resident) {
      // backfill: jobs of at most a sixteenth of the fill step whatever the others hold
      const bool light = s->backfill && j->h->N * 16 <= s->fill;
      const bool step = s->share_all || filled < s->fill || light;
      const int64_t want = step ? j->spec.steps : j->h->target_step;
      if (j->h->limit != want) {
        if (mpc_status st = mpc_set_step_limit(j->h, want); st != MPC_OK)
          return sfail(s, st, "step limit: " + j->h->err);
      }
      if (step) {
        filled += j->h->N;
        chunk_work += (double)j->h->N;
        min_left = std::min(min_left, j->spec.steps - j->h->target_step);
      }
    }
    Job* const head = s->head;
    const bool launched = min_left != INT64_MAX;
    if (launched) {
      // the next chunk ends where the first stepping job finishes (at most chunk steps)
      const int64_t n = std::max<int64_t>(1, std::min<int64_t>(min_left, s->chunk));
      if (cudaEventRecord(s->chunk_start, s->stream) != cudaSuccess)
        return sfail(s, MPC_ECUDA, "event record failed");
      if (mpc_status st = mpc_batch_step(s->batch, n); st != MPC_OK)
        return sfail(s, st, std::string("batch step: ") + mpc_batch_last_error(s->batch));
      if (cudaEventRecord(s->chunk_done, s->stream) != cudaSuccess)
        return sfail(s, MPC_ECUDA, "event record failed");
      if (s->gap_open) s->stats.host_gap_ms += 1e3 * (now_s(s->t0) - s->gap_from);
      s->stats.chunks += 1;
      s->stats.chunk_steps += n;
      s->work_done += chunk_work * (double)n;
    }
    // while the chunk runs: analyse the jobs retired after the previous chunk
    for (Job* j : fetched) analyse(s, *j);
    fetched.clear();
    const bool head_running = head && cudaEventQuery(s->head_done) == cudaErrorNotReady;
    if (!launched && !head) {
      s->gap_open = false;  // idle for lack of work, not for the host
      // nothing resident: wait for the next arrival
      double next = 1e300;
      for (size_t i = s->next_queued; i < s->jobs.size(); ++i)
        if (s->jobs[i].res.status == MPC_JOB_QUEUED) next = std::min(next, s->jobs[i].spec.arrival_s);
      const double wait = next - now_s(s->t0);
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.05)));
      continue;
    }
    if (launched) {
      // admit arrivals while the chunk runs; they join the next chunk
      while (cudaEventQuery(s->chunk_done) == cudaErrorNotReady) {
        admit(s);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
      }
      cudaGetLastError();
      s->gap_open = true;  // the GPU is idle from here until the next chunk is enqueued
      s->gap_from = now_s(s->t0);
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, s->chunk_start, s->chunk_done) == cudaSuccess) s->stats.gpu_ms += ms;
      else cudaGetLastError();
      if (mpc_status st = mpc_batch_synchronize(s->batch); st != MPC_OK)
        return sfail(s, st, std::string("batch: ") + mpc_batch_last_error(s->batch));
    } else if (head_running) {
      // only the head steps: poll it, admitting arrivals meanwhile
      admit(s);
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    cudaGetLastError();
    if (head && cudaEventQuery(s->head_done) == cudaSuccess) {
      // the head finished its steps (a capacity repair, if any, completes them here)
      if (mpc_status st = mpc_synchronize(head->h); st != MPC_OK)
        return sfail(s, st, "head job: " + head->h->err);
      batch_set_detached(head->h, false);
      head->h->stream = s->stream;
      s->head = nullptr;
    }
    cudaGetLastError();
    for (Job& j : s->jobs) {
      if (j.res.status != MPC_JOB_RUNNING || !j.h || &j == s->head || j.h->target_step < j.spec.steps)
        continue;
      const mpc_status st = fetch(s, j);
      mpc_batch_remove(s->batch, j.h);
      j.h = nullptr;
      if (st != MPC_OK) fail_job(j, st, now_s(s->t0));
      else fetched.push_back(&j);
    }
  }
}

mpc_status run_sequential(mpc_server s, double deadline) {
  for (Job& j : s->jobs) {
    if (j.res.status != MPC_JOB_QUEUED) continue;
    if (now_s(s->t0) > deadline) return sfail(s, MPC_ETIMEOUT, "server run timed out");
    const double wait = j.spec.arrival_s - now_s(s->t0);
    if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
    const mpc_params q = job_params(s, j);
    mpc_handle h = nullptr;
    j.res.admit_s = now_s(s->t0);
    mpc_status st = mpc_create(&q, s->stream, nullptr, &h);
    if (st != MPC_OK) {
      fail_job(j, st, now_s(s->t0));
      continue;
    }
    j.h = h;
    j.res.status = MPC_JOB_RUNNING;
    j.res.n_particles = h->N;
    st = mpc_step(h, j.spec.steps);
    if (st == MPC_OK) st = mpc_synchronize(h);
    if (st == MPC_OK) st = fetch(s, j);
    mpc_destroy(h);
    j.h = nullptr;
    if (st != MPC_OK) {
      fail_job(j, st, now_s(s->t0));
      continue;
    }
    analyse(s, j);
  }
  return MPC_OK;
}

}  // namespace

extern "C" {

const char* mpc_server_last_error(mpc_server s) {
  return s ? s->err.c_str() : g_server_create_error.c_str();
}

mpc_status mpc_server_destroy(mpc_server s) {
  if (!s) return MPC_OK;
  if (s->batch) mpc_batch_destroy(s->batch);
  if (s->chunk_done) cudaEventDestroy(s->chunk_done);
  if (s->chunk_start) cudaEventDestroy(s->chunk_start);
  if (s->head_done) cudaEventDestroy(s->head_done);
  if (s->head_ready) cudaEventDestroy(s->head_ready);
  if (s->head_stream) cudaStreamDestroy(s->head_stream);
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
  return MPC_OK;
}

mpc_status mpc_server_create(const mpc_server_config* cfg, void* stream, mpc_server* out) {
  if (!cfg || !out) return sfail(nullptr, MPC_EINVAL, "config and out are required");
  *out = nullptr;
  if (cfg->hbm_budget_bytes == 0 || cfg->chunk_steps < 0 || cfg->max_active < 0 ||
      cfg->max_active > kMaxBatchBoxes || cfg->fill_kparticles < 0 ||
      (cfg->flags & ~(uint32_t)(MPC_SERVER_DETERMINISTIC | MPC_SERVER_SEQUENTIAL |
                                MPC_SERVER_SHARE_ALL | MPC_SERVER_FIRST_COME | MPC_SERVER_AGED |
                                MPC_SERVER_BACKFILL | MPC_SERVER_PRIORITY_HEAD)))
    return sfail(nullptr, MPC_EINVAL, "invalid server configuration");
  mpc_server s = new (std::nothrow) mpc_server_s();
  if (!s) return sfail(nullptr, MPC_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  s->stream = static_cast<cudaStream_t>(stream);
  s->det = (cfg->flags & MPC_SERVER_DETERMINISTIC) != 0;
  s->sequential = (cfg->flags & MPC_SERVER_SEQUENTIAL) != 0;
  s->share_all = (cfg->flags & MPC_SERVER_SHARE_ALL) != 0;
  s->first_come = (cfg->flags & MPC_SERVER_FIRST_COME) != 0;
  s->aged = (cfg->flags & MPC_SERVER_AGED) != 0;
  s->backfill = (cfg->flags & MPC_SERVER_BACKFILL) != 0;
  s->priority_head = (cfg->flags & MPC_SERVER_PRIORITY_HEAD) != 0 &&
                     (cfg->flags & MPC_SERVER_SEQUENTIAL) == 0;
  if (cfg->fill_kparticles > 0) s->fill = (int64_t)cfg->fill_kparticles * 1000;
  s->chunk = cfg->chunk_steps > 0 ? cfg->chunk_steps : 100;
  if (cudaEventCreate(&s->chunk_done) != cudaSuccess || cudaEventCreate(&s->chunk_start) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    mpc_server_destroy(s);
    return sfail(nullptr, MPC_ECUDA, "event or stream creation failed");
  }
  if (s->priority_head) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->head_stream, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->head_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->head_ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      mpc_server_destroy(s);
      return sfail(nullptr, MPC_ECUDA, "priority stream creation failed");
    }
  }
  if (!s->sequential) {
    mpc_batch_config bc{};
    bc.arena_bytes = cfg->hbm_budget_bytes;
    bc.graph_steps = s->chunk;
    bc.flags = s->det ? MPC_BATCH_DETERMINISTIC : 0u;
    bc.max_boxes = cfg->max_active;
    if (mpc_status st = mpc_batch_create(&bc, stream, &s->batch); st != MPC_OK) {
      const std::string msg = mpc_batch_last_error(nullptr);
      mpc_server_destroy(s);
      return sfail(nullptr, st, "batch: " + msg);
    }
  }
  *out = s;
  return MPC_OK;
}

mpc_status mpc_server_submit(mpc_server s, const mpc_job* job, int64_t* job_id) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!job) return sfail(s, MPC_EINVAL, "job is NULL");
  if (job->steps < 1 || job->steps > (1 << 24)) return sfail(s, MPC_EINVAL, "steps must lie in [1, 2^24]");
  if (!std::isfinite(job->arrival_s) || job->arrival_s < 0.0)
    return sfail(s, MPC_EINVAL, "arrival_s must be finite and >= 0");
  if (job->reserved != 0 || (job->keep & ~(uint32_t)(MPC_JOB_KEEP_SERIES | MPC_JOB_KEEP_STATE)))
    return sfail(s, MPC_EINVAL, "invalid job flags");
  if (!s->jobs.empty() && job->arrival_s < s->jobs.back().spec.arrival_s)
    return sfail(s, MPC_EINVAL, "jobs must be submitted in arrival order");
  Job j;
  j.spec = *job;
  j.res.status = MPC_JOB_QUEUED;
  j.res.arrival_s = job->arrival_s;
  s->jobs.push_back(std::move(j));
  if (job_id) *job_id = (int64_t)s->jobs.size() - 1;
  return MPC_OK;
}

mpc_status mpc_server_run(mpc_server s, double timeout_s) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!s->started) {
    s->t0 = std::chrono::steady_clock::now();
    s->started = true;
  }
  const double deadline = now_s(s->t0) + (timeout_s > 0 ? timeout_s : 1e300);
  return s->sequential ? run_sequential(s, deadline) : run_batched(s, deadline);
}

mpc_status mpc_server_get_stats(mpc_server s, mpc_server_stats* out) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!out) return sfail(s, MPC_EINVAL, "out is NULL");
  *out = s->stats;
  if (s->batch) {
    mpc_batch_info bi{};
    if (mpc_batch_get_info(s->batch, &bi) == MPC_OK) {
      out->plan_ms = bi.plan_ms;
      out->graph_builds = bi.graph_builds;
    }
  }
  return MPC_OK;
}

mpc_status mpc_server_job(mpc_server s, int64_t job_id, mpc_job_result* out) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!out || job_id < 0 || job_id >= (int64_t)s->jobs.size())
    return sfail(s, MPC_EINVAL, "no such job");
  *out = s->jobs[(size_t)job_id].res;
  return MPC_OK;
}

mpc_status mpc_server_job_series(mpc_server s, int64_t job_id, double* rows, int64_t count) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!rows || job_id < 0 || job_id >= (int64_t)s->jobs.size()) return sfail(s, MPC_EINVAL, "no such job");
  const Job& j = s->jobs[(size_t)job_id];
  if (j.res.status != MPC_JOB_DONE || j.series.empty())
    return sfail(s, MPC_ESTATE, "the job is not done or kept no series");
  if (count < j.spec.steps) return sfail(s, MPC_EINVAL, "count is below the job's steps");
  std::memcpy(rows, j.series.data(), j.series.size() * sizeof(double));
  return MPC_OK;
}

mpc_status mpc_server_job_state(mpc_server s, int64_t job_id, uint32_t* X, float* V, uint32_t* id) {
  if (!s) return sfail(nullptr, MPC_EINVAL, "server is NULL");
  if (!X || !V || !id || job_id < 0 || job_id >= (int64_t)s->jobs.size())
    return sfail(s, MPC_EINVAL, "no such job or NULL buffers");
  const Job& j = s->jobs[(size_t)job_id];
  if (j.res.status != MPC_JOB_DONE || j.X.empty())
    return sfail(s, MPC_ESTATE, "the job is not done or kept no state");
  std::memcpy(X, j.X.data(), j.X.size() * sizeof(uint32_t));
  std::memcpy(V, j.V.data(), j.V.size() * sizeof(float));
  std::memcpy(id, j.id.data(), j.id.size() * sizeof(uint32_t));
  return MPC_OK;
}

}  // extern "C"
