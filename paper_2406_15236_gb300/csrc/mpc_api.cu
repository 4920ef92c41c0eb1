// Host side of the C ABI declared in include/mpc.h: parameter checks, the brick
// geometry, device buffers, graph-captured step chains, overflow repair, and the
// state / observables readers.
#include <algorithm>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "mpc.h"
#include "mpc_host.h"
#include "mpc_internal.h"

using namespace mpc;
using namespace mpc::host;

namespace {
thread_local std::string g_last_create_error;
}  // namespace

namespace mpc {
namespace host {
mpc_status fail(mpc_handle h, mpc_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_last_create_error = msg;
  return st;
}
}  // namespace host
}  // namespace mpc

namespace {
const char* kVersion = "mpc-gb300 0.2 (sm_103a)";
}  // namespace

namespace mpc {
namespace host {

void* dev_alloc(mpc_handle h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->stream);
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) {
    h->allocs.emplace_back(p, bytes);
    h->bytes += bytes;
  }
  return p;
}

void dev_free(mpc_handle h, void* p) {
  if (!p) return;
  for (size_t k = 0; k < h->allocs.size(); ++k) {
    if (h->allocs[k].first == p) {
      const size_t bytes = h->allocs[k].second;
      if (h->has_alloc) h->alloc.release(h->alloc.ctx, p, bytes, (void*)h->stream);
      else cudaFree(p);
      h->bytes -= bytes;
      h->allocs.erase(h->allocs.begin() + (long)k);
      return;
    }
  }
}

template <class T>
mpc_status alloc_array(mpc_handle h, T** out, size_t count, const char* what) {
  *out = static_cast<T*>(dev_alloc(h, count * sizeof(T)));
  if (!*out) return fail(h, MPC_ENOMEM, std::string("device allocation failed: ") + what);
  return MPC_OK;
}

int ceil_log2(int v) {
  int k = 0;
  while ((1LL << k) < (long long)v) ++k;
  return k;
}

// derived brick quantities: log2 of the edges, counts, threads per cell
// tpc_req > 0 fixes the threads per cell; 0 picks the largest power of two that still
// finalises every cell of the brick in one pass
void finish_bricks(Geom& g, int tpc_req) {
  for (int ax = 0; ax < 3; ++ax) g.Bs[ax] = ceil_log2(g.B[ax]);
  g.nbricks = g.nb[0] * g.nb[1] * g.nb[2];
  g.brick_cells = g.B[0] * g.B[1] * g.B[2];
  int tpc = 1;
  while (tpc < 32 && tpc * 2 * g.brick_cells <= kStepThreads) tpc *= 2;
  g.tpc = tpc_req > 0 ? tpc_req : tpc;
}

// cells per brick: powers of two, grown on the shortest axis first, ~tile particles
void choose_bricks(Geom& g, double n_c, int tile, int tpc_req) {
  const int target = std::max(1, (int)std::lround(tile / std::max(n_c, 1e-3)));
  int B[3] = {1, 1, 1};
  for (;;) {
    int best = -1;
    for (int ax = 0; ax < 3; ++ax)
      if (B[ax] * 2 <= g.Lc[ax] && (best < 0 || B[ax] < B[best])) best = ax;
    if (best < 0 || B[0] * B[1] * B[2] * 2 > target) break;
    B[best] *= 2;
  }
  for (int ax = 0; ax < 3; ++ax) {
    g.B[ax] = B[ax];
    g.nb[ax] = (g.Lc[ax] + B[ax] - 1) / B[ax];
  }
  finish_bricks(g, tpc_req);
}

int capacity_for(double mean) {
  const double c = mean + 7.0 * std::sqrt(std::max(mean, 1.0)) + 32.0;
  int cap = (int)std::ceil(c / 32.0) * 32;
  return std::max(cap, 64);
}

mpc_status validate(const mpc_params* p) {
  if (!p) return fail(nullptr, MPC_EINVAL, "params is NULL");
  for (int ax = 0; ax < 3; ++ax)
    if (p->L[ax] < 2 || p->L[ax] > 1024) return fail(nullptr, MPC_EINVAL, "L must lie in [2, 1024]");
  if (p->a != 1.0) return fail(nullptr, MPC_EINVAL, "only a = 1 is supported");
  if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(nullptr, MPC_EINVAL, "h must be > 0");
  if (!(p->kT > 0.0) || !(p->m > 0.0)) return fail(nullptr, MPC_EINVAL, "kT and m must be > 0");
  if (!(p->n_c > 0.0)) return fail(nullptr, MPC_EINVAL, "n_c must be > 0");
  if (p->variant != MPC_SRD && p->variant != MPC_AT_A && p->variant != MPC_SRD_A)
    return fail(nullptr, MPC_EINVAL, "variant must be MPC_SRD, MPC_AT_A or MPC_SRD_A");
  if (p->thermostat && p->variant != MPC_SRD)
    return fail(nullptr, MPC_EINVAL, "the MBS thermostat applies to SRD only");
  if (p->walls_z < 0 || p->walls_z > 2)
    return fail(nullptr, MPC_EINVAL, "walls_z must be 0 (periodic), 1 (no-slip) or 2 (slip)");
  for (int k = 0; k < 2; ++k) {
    if (!std::isfinite(p->wall_u[k])) return fail(nullptr, MPC_EINVAL, "wall_u must be finite");
    if (p->wall_u[k] != 0.0 && p->walls_z != 1)
      return fail(nullptr, MPC_EINVAL, "moving walls need walls_z = 1 (no-slip)");
  }
  for (int ax = 0; ax < 3; ++ax)
    if (!std::isfinite(p->gravity[ax])) return fail(nullptr, MPC_EINVAL, "gravity must be finite");
  const double vol = (double)p->L[0] * p->L[1] * p->L[2];
  const double N = std::llround(vol * p->n_c);
  if (N < 1 || N > 4.0e9) return fail(nullptr, MPC_EINVAL, "particle count must lie in [1, 4e9]");
  if (p->capacity < 0 || p->capacity > 60000) return fail(nullptr, MPC_EINVAL, "capacity must lie in [0, 60000]");
  if (p->graph_steps < 0) return fail(nullptr, MPC_EINVAL, "graph_steps must be >= 0");
  if (p->tile_particles < 0 || p->tile_particles > 16384)
    return fail(nullptr, MPC_EINVAL, "tile_particles must lie in [0, 16384]");
  {
    const int t = p->threads_per_cell;
    if (t < 0 || t > 32 || (t & (t - 1)) != 0)
      return fail(nullptr, MPC_EINVAL, "threads_per_cell must be 0 or a power of two <= 32");
  }
  if (p->reserved != 0) return fail(nullptr, MPC_EINVAL, "reserved must be 0");
  if (p->obs_ring < 0 || p->obs_ring > (1 << 24))
    return fail(nullptr, MPC_EINVAL, "obs_ring must lie in [0, 2^24]");
  if (p->flags & ~(uint32_t)(MPC_FLAG_OBSERVABLES | MPC_FLAG_DEBUG_CELLS | MPC_FLAG_DETERMINISTIC))
    return fail(nullptr, MPC_EINVAL, "unknown flag bits");
  return MPC_OK;
}

StepArgs step_args(mpc_handle h) {
  StepArgs a{};
  a.g = h->g;
  a.buf[0] = h->buf[0];
  a.buf[1] = h->buf[1];
  a.cnt[0] = h->cnt[0];
  a.cnt[1] = h->cnt[1];
  a.ctrl = h->ctrl;
  a.spill = h->spill;
  a.obs_partials = h->obs_partials;
  a.obs_series = h->obs_series;
  a.obs_ring = h->obs_ring;
  a.dbg_counts = h->dbg_counts;
  a.deferred = h->deferred;
  return a;
}

void free_particle_buffers(mpc_handle h) {
  for (int s = 0; s < 2; ++s) {
    for (int ax = 0; ax < 3; ++ax) {
      dev_free(h, h->buf[s].x[ax]);
      dev_free(h, h->buf[s].v[ax]);
    }
    dev_free(h, h->buf[s].id);
    dev_free(h, h->buf[s].cell);
    h->buf[s] = PBuf{};
  }
}

mpc_status alloc_particle_buffers(mpc_handle h) {
  h->buffers_gen += 1;  // step arguments captured elsewhere (graphs, batch tables) are stale
  const size_t n = (size_t)h->g.nbricks * (size_t)h->g.cap;
  for (int s = 0; s < 2; ++s) {
    for (int ax = 0; ax < 3; ++ax) {
      TRY(alloc_array(h, &h->buf[s].x[ax], n, "positions"));
      TRY(alloc_array(h, &h->buf[s].v[ax], n, "velocities"));
    }
    TRY(alloc_array(h, &h->buf[s].id, n, "ids"));
    if (h->g.debug) TRY(alloc_array(h, &h->buf[s].cell, n, "debug cells"));
  }
  return MPC_OK;
}

// contiguous SoA staging area of n particles
struct Staging {
  PBuf b{};
  void* base = nullptr;
};

mpc_status alloc_staging(mpc_handle h, Staging& st, int64_t n, bool with_cell) {
  const size_t a = ((size_t)n * 4 + 255) & ~size_t(255);
  const size_t bytes = a * (with_cell ? 8 : 7);
  st.base = dev_alloc(h, bytes);
  if (!st.base) return fail(h, MPC_ENOMEM, "device allocation failed: staging");
  char* c = static_cast<char*>(st.base);
  for (int ax = 0; ax < 3; ++ax) st.b.x[ax] = reinterpret_cast<uint32_t*>(c + a * ax);
  for (int ax = 0; ax < 3; ++ax) st.b.v[ax] = reinterpret_cast<float*>(c + a * (3 + ax));
  st.b.id = reinterpret_cast<uint32_t*>(c + a * 6);
  st.b.cell = with_cell ? reinterpret_cast<uint32_t*>(c + a * 7) : nullptr;
  return MPC_OK;
}

mpc_status read_ctrl(mpc_handle h) {
  CU(h, cudaMemcpyAsync(h->ctrl_host, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return MPC_OK;
}

mpc_status check_errors(mpc_handle h) {
  const Ctrl& c = *h->ctrl_host;
  if (c.errors & kErrTimeout) return fail(h, MPC_ETIMEOUT, "a bounded device wait gave up (bulk copy)");
  if (c.errors & kErrBinning) return fail(h, MPC_ESTATE, "a particle was found outside its brick");
  if (c.errors & kErrRange) return fail(h, MPC_ESTATE, "a position outside the box was found");
  if (c.errors & kErrFixedRange)
    return fail(h, MPC_ESTATE, "a fixed-point cell-sum term exceeded its range (2^15)");
  if (c.lost) return fail(h, MPC_ESTATE, "brick and spill capacity both overflowed; state lost");
  return MPC_OK;
}

// bins a contiguous particle set (state before step `step`) into buf[step & 1];
// grows the brick capacity first if a brick would overflow
mpc_status bin_into_bricks(mpc_handle h, const PBuf& src, int64_t n, int64_t step) {
  Geom& g = h->g;
  const int par = (int)(step & 1);
  uint32_t* counts = nullptr;
  uint32_t* maxv = nullptr;
  TRY(alloc_array(h, &counts, (size_t)g.nbricks + 1, "bin counts"));
  maxv = counts + g.nbricks;
  CU(h, cudaMemsetAsync(counts, 0, ((size_t)g.nbricks + 1) * 4, h->stream));
  CU(h, cudaMemsetAsync(&h->ctrl->errors, 0, sizeof(int32_t), h->stream));
  CU(h, launch_bin_count(g, n, src.x, src.v, step, counts, &h->ctrl->errors, h->stream));
  CU(h, launch_max_u32(counts, g.nbricks, maxv, h->stream));
  uint32_t mx = 0;
  CU(h, cudaMemcpyAsync(&mx, maxv, 4, cudaMemcpyDeviceToHost, h->stream));
  TRY(read_ctrl(h));
  dev_free(h, counts);
  if (h->ctrl_host->errors & kErrRange) return fail(h, MPC_EINVAL, "a position lies outside [0, L << F)");
  if ((int)mx > g.cap) {
    // automatic capacity keeps 7 sigma of headroom above the largest brick seen; an
    // explicit capacity is honoured as tightly as the current state allows
    const int want = h->p.capacity > 0 ? (int)((mx + 3u) & ~3u) : capacity_for((double)mx);
    Geom trial = g;
    trial.cap = want;
    if (want > 60000 || step_smem_bytes(trial) > h->smem_limit)
      return fail(h, MPC_ESTATE, "a brick holds more particles than shared memory allows");
    free_particle_buffers(h);
    g.cap = want;
    TRY(alloc_particle_buffers(h));
    CU(h, configure_step_kernels(h->smem_limit));
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
  }
  CU(h, cudaMemsetAsync(h->cnt[0], 0, (size_t)g.nbricks * 4, h->stream));
  CU(h, cudaMemsetAsync(h->cnt[1], 0, (size_t)g.nbricks * 4, h->stream));
  CU(h, launch_bin_scatter(g, n, src.x, src.v, src.id, src.cell, step, h->buf[par], h->cnt[par],
                           &h->ctrl->errors, h->stream));
  TRY(read_ctrl(h));
  if (h->ctrl_host->errors) return fail(h, MPC_ESTATE, "binning into bricks failed");
  return MPC_OK;
}

mpc_status reset_ctrl(mpc_handle h, int64_t step) {
  Ctrl c{};
  c.step = step;
  h->limit = std::max(h->limit, step);
  c.limit = h->limit;
  *h->ctrl_host = c;
  CU(h, cudaMemcpyAsync(h->ctrl, h->ctrl_host, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (h->obs_partials)
    CU(h, cudaMemsetAsync(h->obs_partials, 0, sizeof(double) * kObsSlots * kObsWidth, h->stream));
  h->target_step = step;
  return MPC_OK;
}

mpc_status build_graph(mpc_handle h) {
  if (h->graph) return MPC_OK;
  const StepArgs a = step_args(h);
  cudaGraph_t graph = nullptr;
  CU(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
  for (int k = 0; k < h->graph_steps; ++k) {
    cudaError_t e = cudaSuccess;
    // external event-record nodes: recorded each time the graph runs (a plain record
    // during capture would only express a dependency)
    if (h->profiling)
      e = cudaEventRecordWithFlags(h->ev_begin[(size_t)k], h->cap_stream, cudaEventRecordExternal);
    if (e == cudaSuccess) e = launch_step(a, h->cap_stream);
    if (e == cudaSuccess && h->profiling)
      e = cudaEventRecordWithFlags(h->ev_end[(size_t)k], h->cap_stream, cudaEventRecordExternal);
    if (e == cudaSuccess) e = launch_advance(a, h->cap_stream);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(h->cap_stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      return fail(h, MPC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
  }
  CU(h, cudaStreamEndCapture(h->cap_stream, &graph));
  cudaError_t e = cudaGraphInstantiate(&h->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(h, MPC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MPC_OK;
}

mpc_status enqueue_steps(mpc_handle h, int64_t n) {
  if (n <= 0) return MPC_OK;
  const StepArgs a = step_args(h);
  if (n >= h->graph_steps) {
    TRY(build_graph(h));
    while (n >= h->graph_steps) {
      CU(h, cudaGraphLaunch(h->graph, h->stream));
      n -= h->graph_steps;
      if (h->profiling) {
        h->ev_recorded = h->graph_steps;
        h->ev_next = 0;
      }
    }
  }
  for (int64_t k = 0; k < n; ++k) {
    if (h->profiling) {
      const size_t slot = (size_t)h->ev_next;
      CU(h, cudaEventRecord(h->ev_begin[slot], h->stream));
      CU(h, launch_step(a, h->stream));
      CU(h, cudaEventRecord(h->ev_end[slot], h->stream));
      h->ev_next = (h->ev_next + 1) % h->graph_steps;
      h->ev_recorded = std::min(h->graph_steps, h->ev_recorded + 1);
    } else {
      CU(h, launch_step(a, h->stream));
    }
    CU(h, launch_advance(a, h->stream));
  }
  return MPC_OK;
}

// gathers the current state (after `step` completed steps) into a contiguous staging
// area: bricks of buf[step & 1] (counts clamped to capacity) followed by the spill list
mpc_status gather(mpc_handle h, Staging& st, bool with_cell) {
  Geom& g = h->g;
  const int64_t step = h->ctrl_host->step;
  const int par = (int)(step & 1);
  TRY(alloc_staging(h, st, h->N, with_cell));
  uint32_t* offs = nullptr;
  const size_t tmpw = scan_tmp_words(g.nbricks);
  TRY(alloc_array(h, &offs, (size_t)g.nbricks + 1 + tmpw, "gather offsets"));
  // clamp counts into offs, scan in place, compact
  std::vector<uint32_t> cnt((size_t)g.nbricks);
  CU(h, cudaMemcpyAsync(cnt.data(), h->cnt[par], (size_t)g.nbricks * 4, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  uint64_t total = 0;
  std::vector<uint32_t> off((size_t)g.nbricks);
  for (int b = 0; b < g.nbricks; ++b) {
    off[(size_t)b] = (uint32_t)total;
    total += std::min<uint32_t>(cnt[(size_t)b], (uint32_t)g.cap);
  }
  const uint32_t spill = std::min<uint32_t>(h->ctrl_host->spill_count, h->spill.capacity);
  if ((int64_t)(total + spill) != h->N) {
    dev_free(h, offs);
    return fail(h, MPC_ESTATE, "particle count changed (bricks + spill != N)");
  }
  CU(h, cudaMemcpyAsync(offs, off.data(), (size_t)g.nbricks * 4, cudaMemcpyHostToDevice, h->stream));
  PBuf src = h->buf[par];
  if (!with_cell) src.cell = nullptr;
  CU(h, launch_compact(g, src, h->cnt[par], offs, st.b, h->stream));
  Spill sp = h->spill;
  if (!with_cell) sp.cell = nullptr;
  CU(h, launch_append_spill(sp, spill, total, st.b, h->stream));
  CU(h, launch_unstream(g, h->N, st.b, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  dev_free(h, offs);
  return MPC_OK;
}

mpc_status repair_overflow(mpc_handle h) {
  Staging st;
  TRY(gather(h, st, h->g.debug != 0));
  const int64_t step = h->ctrl_host->step;
  // grow the capacity by a quarter and rebin
  Geom& g = h->g;
  Geom trial = g;
  trial.cap = std::min(60000, (int)std::ceil(g.cap * 1.25 / 32.0) * 32);
  if (step_smem_bytes(trial) > h->smem_limit) {
    // grow only as far as shared memory allows; bin_into_bricks reports a true overflow
    while (trial.cap > g.cap + 32 && step_smem_bytes(trial) > h->smem_limit) trial.cap -= 32;
  }
  free_particle_buffers(h);
  g.cap = trial.cap;
  TRY(alloc_particle_buffers(h));
  CU(h, configure_step_kernels(h->smem_limit));
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  const int64_t target = h->target_step;
  TRY(reset_ctrl(h, step));
  TRY(bin_into_bricks(h, st.b, h->N, step));
  dev_free(h, st.base);
  h->target_step = target;
  h->recoveries += 1;
  return MPC_OK;
}

mpc_status sync_and_repair(mpc_handle h) {
  for (int rounds = 0; rounds < 64; ++rounds) {
    TRY(read_ctrl(h));
    TRY(check_errors(h));
    if (!h->ctrl_host->halted) {
      if (h->ctrl_host->step != h->target_step)
        return fail(h, MPC_ESTATE, "step counter does not match the requested steps");
      return MPC_OK;
    }
    TRY(repair_overflow(h));
    TRY(enqueue_steps(h, h->target_step - h->ctrl_host->step));
  }
  return fail(h, MPC_ESTATE, "capacity overflow repeated too often");
}

mpc_status set_device(mpc_handle h) {
  CU(h, cudaSetDevice(h->device));
  return MPC_OK;
}

size_t device_smem_limit(int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (size_t)optin - 2048;  // room for the kernel's static shared memory
}

mpc_status plan_box(const mpc_params* p, size_t smem_limit, Geom& g, int64_t& N) {
  TRY(validate(p));
  g = Geom{};
  g.F = fixed_bits_for(p->L);
  g.mask = (1u << g.F) - 1u;
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = p->L[ax];
    g.Lc[ax] = p->L[ax];
    g.P[ax] = (uint32_t)p->L[ax] << g.F;
    g.gh[ax] = (float)(p->gravity[ax] * p->h);
  }
  g.walls = p->walls_z;
  g.wall_u[0] = (float)p->wall_u[0];
  g.wall_u[1] = (float)p->wall_u[1];
  if (g.walls) g.Lc[2] += 1;
  g.hs = (float)std::ldexp(p->h, g.F);
  g.inv2F = (float)std::ldexp(1.0, -g.F);
  g.variant = p->variant;
  g.thermostat = p->thermostat ? 1 : 0;
  const double alpha = p->alpha_deg * M_PI / 180.0;
  g.cos_a = (float)std::cos(alpha);
  g.sin_a = (float)std::sin(alpha);
  g.sigma = (float)std::sqrt(p->kT / p->m);
  g.kT = (float)p->kT;
  g.m = (float)p->m;
  g.n_c = p->n_c;
  g.key0 = (uint32_t)(p->seed & 0xffffffffu);
  g.key1 = (uint32_t)(p->seed >> 32);
  round_keys(g);
  g.box = p->box_id;
  g.obs = (p->flags & MPC_FLAG_OBSERVABLES) ? 1 : 0;
  g.debug = (p->flags & MPC_FLAG_DEBUG_CELLS) ? 1 : 0;
  g.det = (p->flags & MPC_FLAG_DETERMINISTIC) ? 1 : 0;
  g.ncells = (int64_t)g.Lc[0] * g.Lc[1] * g.Lc[2];
  const int tile = p->tile_particles > 0 ? p->tile_particles : kBrickParticles;
  choose_bricks(g, p->n_c, tile, p->threads_per_cell);
  g.cap = p->capacity > 0 ? ((p->capacity + 3) & ~3) : capacity_for(p->n_c * g.brick_cells);
  // shrink the brick until one brick's particles fit in shared memory
  while (step_smem_bytes(g) > smem_limit && g.brick_cells > 1 && p->capacity == 0) {
    int ax = 0;
    for (int k = 1; k < 3; ++k)
      if (g.B[k] > g.B[ax]) ax = k;
    g.B[ax] /= 2;
    g.nb[ax] = (g.Lc[ax] + g.B[ax] - 1) / g.B[ax];
    finish_bricks(g, p->threads_per_cell);
    g.cap = capacity_for(p->n_c * g.brick_cells);
  }
  if (step_smem_bytes(g) > smem_limit) return fail(nullptr, MPC_EINVAL, "brick capacity exceeds shared memory");
  N = std::llround((double)p->L[0] * p->L[1] * p->L[2] * p->n_c);
  return MPC_OK;
}

namespace {
size_t rounded(size_t bytes) { return ((bytes ? bytes : 256) + 255) & ~size_t(255); }
uint32_t spill_capacity(int64_t N) { return (uint32_t)std::max<int64_t>(4096, N / 256); }
}  // namespace

void box_footprint(const Geom& g, int64_t N, size_t& steady, size_t& peak) {
  const size_t n = (size_t)g.nbricks * (size_t)g.cap;
  const size_t sp = spill_capacity(N);
  size_t s = rounded(sizeof(Ctrl)) + 2 * rounded((size_t)g.nbricks * 4);
  s += 8 * rounded(sp * 4) + (g.debug ? rounded(sp * 4) : 0);  // x, v, id, dest (+ cell)
  s += rounded(sizeof(double) * kObsSlots * kObsWidth);
  if (g.debug) s += rounded((size_t)g.ncells * 4);
  s += rounded(((size_t)g.nbricks + 2) * 4);  // deferred bricks
  s += 2 * (7 + (g.debug ? 1 : 0)) * rounded(n * 4);
  steady = s;
  // creation: contiguous staging (7 arrays) + init sums + bin counts
  const size_t a = ((size_t)N * 4 + 255) & ~size_t(255);
  peak = s + rounded(a * 7) + rounded(sizeof(double) * 3 * 64) + rounded(((size_t)g.nbricks + 1) * 4);
}

mpc_status create_box(const mpc_params* p, cudaStream_t stream, const mpc_allocator* alloc,
                      Ctrl* ctrl_slot, mpc_handle* out) {
  if (!out) return fail(nullptr, MPC_EINVAL, "out is NULL");
  *out = nullptr;
  TRY(validate(p));
  if (alloc && (!alloc->alloc || !alloc->release))
    return fail(nullptr, MPC_EINVAL, "allocator needs alloc and release");
  mpc_handle h = new (std::nothrow) mpc_s();
  if (!h) return fail(nullptr, MPC_ENOMEM, "host allocation failed");
  auto bail = [&](mpc_status st) {
    g_last_create_error = h->err;
    destroy_box(h, true);
    return st;
  };
  h->p = *p;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, MPC_ECUDA, "no CUDA device");
  }
  h->stream = stream;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, "stream creation failed"));
  if (ctrl_slot) {
    h->ctrl_host = ctrl_slot;
    h->ctrl_host_owned = false;
  } else if (cudaMallocHost(&h->ctrl_host, sizeof(Ctrl)) != cudaSuccess) {
    h->ctrl_host = nullptr;
    return bail(fail(h, MPC_ENOMEM, "pinned host allocation failed"));
  }
  h->graph_steps = p->graph_steps > 0 ? p->graph_steps : 16;
  h->obs_ring = p->obs_ring > 0 ? p->obs_ring : 1024;
  h->smem_limit = device_smem_limit(h->device);
  if (h->smem_limit == 0) return bail(fail(h, MPC_ECUDA, "cannot query shared memory per block"));
  {
    mpc_status st = plan_box(p, h->smem_limit, h->g, h->N);
    if (st != MPC_OK) return bail(fail(h, st, g_last_create_error));
  }
  Geom& g = h->g;

  mpc_status st;
  if ((st = alloc_array(h, &h->ctrl, 1, "control block")) != MPC_OK) return bail(st);
  for (int s = 0; s < 2; ++s)
    if ((st = alloc_array(h, &h->cnt[s], (size_t)g.nbricks, "brick counts")) != MPC_OK) return bail(st);
  h->spill.capacity = spill_capacity(h->N);
  for (int ax = 0; ax < 3; ++ax) {
    if ((st = alloc_array(h, &h->spill.x[ax], h->spill.capacity, "spill")) != MPC_OK) return bail(st);
    if ((st = alloc_array(h, &h->spill.v[ax], h->spill.capacity, "spill")) != MPC_OK) return bail(st);
  }
  if ((st = alloc_array(h, &h->spill.id, h->spill.capacity, "spill")) != MPC_OK) return bail(st);
  if ((st = alloc_array(h, &h->spill.dest, h->spill.capacity, "spill")) != MPC_OK) return bail(st);
  if (g.debug && (st = alloc_array(h, &h->spill.cell, h->spill.capacity, "spill")) != MPC_OK) return bail(st);
  if ((st = alloc_array(h, &h->obs_partials, (size_t)kObsSlots * kObsWidth, "observables")) != MPC_OK) return bail(st);
  if ((st = alloc_array(h, &h->obs_series, (size_t)h->obs_ring * kObsWidth, "observables")) != MPC_OK) return bail(st);
  if (g.debug && (st = alloc_array(h, &h->dbg_counts, (size_t)g.ncells, "debug counts")) != MPC_OK) return bail(st);
  if ((st = alloc_array(h, &h->deferred, (size_t)g.nbricks + 2, "deferred bricks")) != MPC_OK) return bail(st);
  if (cudaMemsetAsync(h->deferred, 0, ((size_t)g.nbricks + 2) * 4, h->stream) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, "memset"));
  if ((st = alloc_particle_buffers(h)) != MPC_OK) return bail(st);
  if (configure_step_kernels(h->smem_limit) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, "cannot configure the step kernel (shared memory)"));
  if (cudaMemsetAsync(h->obs_series, 0, sizeof(double) * h->obs_ring * kObsWidth, h->stream) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, "memset"));
  if ((st = reset_ctrl(h, 0)) != MPC_OK) return bail(st);

  // initial state (Sec. II): uniform positions, Maxwell-Boltzmann velocities, zero
  // net momentum, consecutive ids -- generated contiguous, then binned for step 0
  Staging stg;
  if ((st = alloc_staging(h, stg, h->N, false)) != MPC_OK) return bail(st);
  double* sums = nullptr;
  if ((st = alloc_array(h, &sums, 3 * 64, "init sums")) != MPC_OK) return bail(st);
  if (cudaMemsetAsync(sums, 0, sizeof(double) * 3 * 64, h->stream) != cudaSuccess ||
      launch_init_particles(g, h->N, stg.b.x, stg.b.v, stg.b.id, sums, h->stream) != cudaSuccess ||
      launch_sub_mean(h->N, stg.b.v, sums, h->stream) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, std::string("init: ") + cudaGetErrorString(cudaGetLastError())));
  if ((st = bin_into_bricks(h, stg.b, h->N, 0)) != MPC_OK) return bail(st);
  dev_free(h, sums);
  dev_free(h, stg.base);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess)
    return bail(fail(h, MPC_ECUDA, std::string("init: ") + cudaGetErrorString(cudaGetLastError())));
  *out = h;
  return MPC_OK;
}

void destroy_box(mpc_handle h, bool sync) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (sync) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (cudaEvent_t e : h->ev_begin) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_end) cudaEventDestroy(e);
  while (!h->allocs.empty()) dev_free(h, h->allocs.back().first);
  if (h->ctrl_host && h->ctrl_host_owned) cudaFreeHost(h->ctrl_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

mpc_status set_step_limit(mpc_handle h, int64_t limit) {
  if (limit < h->target_step) return fail(h, MPC_EINVAL, "the limit lies before the steps already requested");
  h->limit = limit;
  CU(h, launch_store_i64(&h->ctrl->limit, limit, h->stream));
  return MPC_OK;
}

}  // namespace host
}  // namespace mpc

namespace mpc {
// lets entry points that take no handle report through mpc_last_error(NULL)
void set_null_handle_error(const std::string& msg) { g_last_create_error = msg; }
}  // namespace mpc

extern "C" {

const char* mpc_version(void) { return kVersion; }

const char* mpc_last_error(mpc_handle h) {
  return h ? h->err.c_str() : g_last_create_error.c_str();
}

mpc_status mpc_create(const mpc_params* p, void* stream, const mpc_allocator* alloc, mpc_handle* out) {
  return create_box(p, static_cast<cudaStream_t>(stream), alloc, nullptr, out);
}

mpc_status mpc_destroy(mpc_handle h) {
  if (!h) return MPC_OK;
  if (h->batch) return fail(h, MPC_EINVAL, "the box belongs to a batch: use mpc_batch_remove");
  destroy_box(h, true);
  return MPC_OK;
}

mpc_status mpc_step(mpc_handle h, int64_t nsteps) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, MPC_EINVAL, "nsteps must be >= 0");
  TRY(set_device(h));
  const int64_t n = std::min(nsteps, h->limit - h->target_step);
  h->target_step += n;
  return enqueue_steps(h, n);
}

mpc_status mpc_set_step_limit(mpc_handle h, int64_t limit) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  TRY(set_device(h));
  return set_step_limit(h, limit);
}

mpc_status mpc_footprint(const mpc_params* p, uint64_t* steady_bytes, uint64_t* peak_bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MPC_ECUDA, "no CUDA device");
  }
  const size_t lim = device_smem_limit(dev);
  if (lim == 0) return fail(nullptr, MPC_ECUDA, "cannot query shared memory per block");
  Geom g;
  int64_t N = 0;
  TRY(plan_box(p, lim, g, N));
  size_t steady = 0, peak = 0;
  box_footprint(g, N, steady, peak);
  const size_t ring = (((size_t)(p->obs_ring > 0 ? p->obs_ring : 1024) * kObsWidth * 8) + 255) & ~size_t(255);
  if (steady_bytes) *steady_bytes = steady + ring;
  if (peak_bytes) *peak_bytes = peak + ring;
  return MPC_OK;
}

mpc_status mpc_synchronize(mpc_handle h) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  TRY(set_device(h));
  return sync_and_repair(h);
}

mpc_status mpc_get_state(mpc_handle h, uint32_t* X, float* V, uint32_t* id, uint32_t* cell,
                         int64_t* step, int device_ptrs) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!X || !V) return fail(h, MPC_EINVAL, "X and V are required");
  if (cell && !h->g.debug) return fail(h, MPC_ESTATE, "cells need MPC_FLAG_DEBUG_CELLS");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  Geom& g = h->g;
  const int64_t N = h->N;
  Staging st;
  TRY(gather(h, st, cell != nullptr));
  // counting sort by unshifted cell
  const int64_t C = (int64_t)g.L[0] * g.L[1] * g.L[2];
  uint32_t* hist = nullptr;
  const size_t tmpw = scan_tmp_words(C);
  TRY(alloc_array(h, &hist, (size_t)C + tmpw, "cell histogram"));
  CU(h, cudaMemsetAsync(hist, 0, (size_t)C * 4, h->stream));
  CU(h, launch_cell_hist(g, N, st.b.x, hist, h->stream));
  CU(h, launch_scan(hist, hist, C, hist + C, h->stream));
  Staging out;
  PBuf dst{};
  if (device_ptrs) {
    for (int ax = 0; ax < 3; ++ax) {
      dst.x[ax] = X + (size_t)ax * N;
      dst.v[ax] = V + (size_t)ax * N;
    }
    dst.id = id;
    dst.cell = cell;
  } else {
    TRY(alloc_staging(h, out, N, cell != nullptr));
    dst = out.b;
    if (!id) dst.id = nullptr;
  }
  PBuf src = st.b;
  if (!dst.id) src.id = nullptr;
  if (!id && dst.id) dst.id = nullptr;
  CU(h, launch_cell_scatter(g, N, src, hist, dst, h->stream));
  if (!device_ptrs) {
    for (int ax = 0; ax < 3; ++ax) {
      CU(h, cudaMemcpyAsync(X + (size_t)ax * N, out.b.x[ax], (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
      CU(h, cudaMemcpyAsync(V + (size_t)ax * N, out.b.v[ax], (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
    }
    if (id) CU(h, cudaMemcpyAsync(id, out.b.id, (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
    if (cell) CU(h, cudaMemcpyAsync(cell, out.b.cell, (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
  }
  CU(h, cudaStreamSynchronize(h->stream));
  if (!device_ptrs) dev_free(h, out.base);
  dev_free(h, hist);
  dev_free(h, st.base);
  if (step) *step = h->ctrl_host->step;
  return MPC_OK;
}

mpc_status mpc_set_state(mpc_handle h, const uint32_t* X, const float* V, const uint32_t* id,
                         int64_t step, int device_ptrs) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!X || !V || !id) return fail(h, MPC_EINVAL, "X, V and id are required");
  if (step < 0 || step >= (1LL << 32)) return fail(h, MPC_EINVAL, "step must lie in [0, 2^32)");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  const int64_t N = h->N;
  Staging st;
  TRY(alloc_staging(h, st, N, false));
  const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int ax = 0; ax < 3; ++ax) {
    CU(h, cudaMemcpyAsync(st.b.x[ax], X + (size_t)ax * N, (size_t)N * 4, kind, h->stream));
    CU(h, cudaMemcpyAsync(st.b.v[ax], V + (size_t)ax * N, (size_t)N * 4, kind, h->stream));
  }
  CU(h, cudaMemcpyAsync(st.b.id, id, (size_t)N * 4, kind, h->stream));
  TRY(reset_ctrl(h, step));
  CU(h, launch_check_range(h->g, N, st.b.x, &h->ctrl->errors, h->stream));
  TRY(read_ctrl(h));
  if (h->ctrl_host->errors & kErrRange) {
    dev_free(h, st.base);
    TRY(reset_ctrl(h, step));
    return fail(h, MPC_EINVAL, "a position lies outside [0, L << F)");
  }
  mpc_status s = bin_into_bricks(h, st.b, N, step);
  dev_free(h, st.base);
  if (s != MPC_OK) return s;
  h->target_step = step;
  return MPC_OK;
}

mpc_status mpc_get_cell_counts(mpc_handle h, uint32_t* counts, int device_ptrs) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!counts) return fail(h, MPC_EINVAL, "counts is NULL");
  if (!h->g.debug) return fail(h, MPC_ESTATE, "per-cell counts need MPC_FLAG_DEBUG_CELLS");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  CU(h, cudaMemcpyAsync(counts, h->dbg_counts, (size_t)h->g.ncells * 4,
                        device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return MPC_OK;
}

mpc_status mpc_velocity_profile(mpc_handle h, int32_t nbins, double* out) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!out) return fail(h, MPC_EINVAL, "out is NULL");
  if (nbins < 1 || nbins > 65536) return fail(h, MPC_EINVAL, "nbins must lie in [1, 65536]");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  double* part = nullptr;
  TRY(alloc_array(h, &part, (size_t)nbins * 4, "velocity profile"));
  const int par = (int)(h->ctrl_host->step & 1);
  cudaError_t e = cudaMemsetAsync(part, 0, sizeof(double) * 4 * (size_t)nbins, h->stream);
  if (e == cudaSuccess) e = launch_velocity_profile(h->g, h->buf[par], h->cnt[par], nbins, part, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, part, sizeof(double) * 4 * (size_t)nbins, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, part);
  if (e != cudaSuccess) return fail(h, MPC_ECUDA, std::string("velocity profile: ") + cudaGetErrorString(e));
  return MPC_OK;
}

mpc_status mpc_observables(mpc_handle h, mpc_obs* out) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!out) return fail(h, MPC_EINVAL, "out is NULL");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  std::memset(out, 0, sizeof(*out));
  const int64_t step = h->ctrl_host->step;
  const double m = h->p.m;
  const double vol = (double)h->p.L[0] * h->p.L[1] * h->p.L[2];
  double px, py, pz, s2;
  if (h->g.obs && step > 0) {
    double row[kObsWidth];
    CU(h, cudaMemcpyAsync(row, h->obs_series + (size_t)((step - 1) % h->obs_ring) * kObsWidth,
                          sizeof(row), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    px = row[0]; py = row[1]; pz = row[2]; s2 = row[3];
    for (int k = 0; k < 3; ++k) out->stress_kin[k] = -m * row[4 + k] / vol;
    for (int k = 0; k < 6; ++k) out->stress_col[k] = -m * row[7 + k] / (vol * h->p.h);
    out->has_stress = 1;
  } else {
    double* part = nullptr;
    TRY(alloc_array(h, &part, (size_t)kObsSlots * 4, "observables"));
    CU(h, cudaMemsetAsync(part, 0, sizeof(double) * kObsSlots * 4, h->stream));
    const int par = (int)(step & 1);
    CU(h, launch_reduce_obs(h->g, h->buf[par], h->cnt[par], part, h->stream));
    std::vector<double> host((size_t)kObsSlots * 4);
    CU(h, cudaMemcpyAsync(host.data(), part, sizeof(double) * kObsSlots * 4, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    dev_free(h, part);
    px = py = pz = s2 = 0.0;
    for (int k = 0; k < kObsSlots; ++k) {
      px += host[(size_t)k * 4 + 0];
      py += host[(size_t)k * 4 + 1];
      pz += host[(size_t)k * 4 + 2];
      s2 += host[(size_t)k * 4 + 3];
    }
  }
  const double N = (double)h->N;
  out->momentum[0] = m * px;
  out->momentum[1] = m * py;
  out->momentum[2] = m * pz;
  out->ekin = 0.5 * m * s2;
  out->temperature = h->N > 1 ? m * (s2 - (px * px + py * py + pz * pz) / N) / (3.0 * (N - 1.0)) : 0.0;
  out->n_particles = h->N;
  out->step = step;
  return MPC_OK;
}

mpc_status mpc_observable_series(mpc_handle h, double* rows, int64_t count, int64_t* written) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!rows || count < 0) return fail(h, MPC_EINVAL, "rows is NULL or count < 0");
  if (!h->g.obs) return fail(h, MPC_ESTATE, "the series needs MPC_FLAG_OBSERVABLES");
  TRY(set_device(h));
  TRY(sync_and_repair(h));
  const int64_t step = h->ctrl_host->step;
  int64_t n = std::min<int64_t>(count, std::min<int64_t>(step, h->obs_ring));
  std::vector<double> ring((size_t)h->obs_ring * kObsWidth);
  CU(h, cudaMemcpyAsync(ring.data(), h->obs_series, ring.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  for (int64_t k = 0; k < n; ++k) {
    const int64_t s = step - n + k;  // row of step s (state after s+1 steps)
    std::memcpy(rows + k * kObsWidth, ring.data() + (size_t)(s % h->obs_ring) * kObsWidth,
                sizeof(double) * kObsWidth);
  }
  if (written) *written = n;
  return MPC_OK;
}

mpc_status mpc_set_profiling(mpc_handle h, int enable) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  TRY(set_device(h));
  const bool on = enable != 0;
  if (on && h->ev_begin.empty()) {
    for (int k = 0; k < h->graph_steps; ++k) {
      cudaEvent_t b, e;
      CU(h, cudaEventCreate(&b));
      CU(h, cudaEventCreate(&e));
      h->ev_begin.push_back(b);
      h->ev_end.push_back(e);
    }
  }
  if (on != h->profiling) {
    CU(h, cudaStreamSynchronize(h->stream));
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    h->profiling = on;
    h->ev_recorded = 0;
    h->ev_next = 0;
  }
  return MPC_OK;
}

mpc_status mpc_profile_step_kernel(mpc_handle h, double* mean_ms, int32_t* samples) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!mean_ms) return fail(h, MPC_EINVAL, "mean_ms is NULL");
  if (!h->profiling) return fail(h, MPC_ESTATE, "profiling is off");
  TRY(set_device(h));
  CU(h, cudaStreamSynchronize(h->stream));
  double total = 0.0;
  for (int k = 0; k < h->ev_recorded; ++k) {
    float ms = 0.0f;
    CU(h, cudaEventElapsedTime(&ms, h->ev_begin[(size_t)k], h->ev_end[(size_t)k]));
    total += ms;
  }
  *mean_ms = h->ev_recorded ? total / h->ev_recorded : 0.0;
  if (samples) *samples = h->ev_recorded;
  return MPC_OK;
}

mpc_status mpc_get_info(mpc_handle h, mpc_info* out) {
  if (!h) return fail(nullptr, MPC_EINVAL, "handle is NULL");
  if (!out) return fail(h, MPC_EINVAL, "out is NULL");
  std::memset(out, 0, sizeof(*out));
  out->n_particles = h->N;
  out->n_cells = h->g.ncells;
  out->step = h->target_step;
  out->fixed_bits = h->g.F;
  out->capacity = h->g.cap;
  for (int ax = 0; ax < 3; ++ax) {
    out->brick[ax] = h->g.B[ax];
    out->n_bricks[ax] = h->g.nb[ax];
  }
  out->device_bytes = h->bytes;
  out->recoveries = h->recoveries;
  out->threads_per_cell = h->g.tpc;
  return MPC_OK;
}

}  // extern "C"
