// Batches of independent MPC boxes (C ABI in include/mpc.h) and the kernel autotuner.
//
// One batch step advances every member by one MPC step:
//   - members large enough to fill the GPU alone (at least two waves of bricks) get
//     their own launch of the single-box kernel;
//   - the other members are packed, grouped by variant and brick geometry (kPackGroup
//     boxes at most per group), and each group is one persistent launch of the packed
//     kernel (with the geometry compiled in when it is a default one), which
//     carries the boxes' arguments in kernel parameter space and lets its CTAs claim
//     the group's bricks from a counter;
//   - one small launch closes the step of every member (step counter, observables).
// Members at their step limit are left out of the launches.  A batch step is captured
// in a CUDA graph of graph_steps steps once the same launch plan is used a second time;
// the plan (and the graph) change when members, their buffers or their stepping state
// change.
//
// Member device memory can come from one arena allocated up front.  Memory a member
// releases returns to the arena only after the stream it was released on has passed the
// release point (an event per release), so a member can be removed while steps that
// still read it are queued.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mpc.h"
#include "mpc_host.h"
#include "mpc_internal.h"

using namespace mpc;
using namespace mpc::host;

namespace {

thread_local std::string g_batch_create_error;

// First/best-fit suballocator over one device allocation with deferred release.
class Arena {
 public:
  ~Arena() {
    reclaim(true);
    for (cudaEvent_t e : events_) cudaEventDestroy(e);
    if (base_) cudaFree(base_);
  }

  bool init(size_t bytes) {
    bytes &= ~size_t(255);
    if (bytes == 0) return false;
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }

  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    reclaim(false);
    void* p = take(bytes);
    if (!p && !pending_.empty()) {
      reclaim(true);
      p = take(bytes);
    }
    return p;
  }

  void release(void* p, size_t bytes, cudaStream_t s) {
    bytes = (bytes + 255) & ~size_t(255);
    const size_t off = static_cast<char*>(p) - static_cast<char*>(base_);
    cudaEvent_t e = event();
    if (e && cudaEventRecord(e, s) == cudaSuccess) {
      pending_.push_back({off, bytes, e});
    } else {
      cudaGetLastError();
      cudaStreamSynchronize(s);
      if (e) events_.push_back(e);
      give_back(off, bytes);
    }
  }

  // returns released blocks whose streams have passed the release (wait: all of them)
  void reclaim(bool wait) {
    size_t k = 0;
    while (k < pending_.size()) {
      Pending& q = pending_[k];
      const cudaError_t r = wait ? cudaEventSynchronize(q.ev) : cudaEventQuery(q.ev);
      if (r == cudaSuccess) {
        give_back(q.off, q.len);
        events_.push_back(q.ev);
        pending_[k] = pending_.back();
        pending_.pop_back();
      } else {
        if (r != cudaErrorNotReady) cudaGetLastError();
        ++k;
      }
    }
  }

  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t pending() const {
    size_t b = 0;
    for (const Pending& q : pending_) b += q.len;
    return b;
  }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }

 private:
  struct Pending {
    size_t off, len;
    cudaEvent_t ev;
  };

  void* take(size_t bytes) {
    auto best = free_.end();
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes && (best == free_.end() || it->second < best->second)) best = it;
    if (best == free_.end()) return nullptr;
    const size_t off = best->first, len = best->second;
    free_.erase(best);
    if (len > bytes) free_[off + bytes] = len - bytes;
    used_ += bytes;
    return static_cast<char*>(base_) + off;
  }

  void give_back(size_t off, size_t len) {
    used_ -= len;
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

  cudaEvent_t event() {
    if (!events_.empty()) {
      cudaEvent_t e = events_.back();
      events_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }

  void* base_ = nullptr;
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length, coalesced
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> events_;
};

void* arena_alloc(void* ctx, size_t bytes, void*) { return static_cast<Arena*>(ctx)->alloc(bytes); }
void arena_release(void* ctx, void* p, size_t bytes, void* stream) {
  static_cast<Arena*>(ctx)->release(p, bytes, static_cast<cudaStream_t>(stream));
}

constexpr int kTableBuffers = 3;  // pinned host copies of the member table in rotation
constexpr int kBranches = 2;      // concurrent streams for the launches of one step
constexpr int kSoloWaves = 2;     // members with this many waves of bricks run solo
constexpr int kWaveCtasPerSm = 6; // CTAs per SM of a wave (the AT+a kernel's occupancy)

}  // namespace

struct mpc_batch_s {
  int device = 0;
  cudaStream_t stream = nullptr;      // steps
  cudaStream_t adm_stream = nullptr;  // member creation (overlaps queued steps)
  cudaStream_t cap_stream = nullptr;  // graph capture
  cudaStream_t branch[kBranches] = {};  // forked streams of one step's launches
  cudaEvent_t fork_ev = nullptr, join_ev[kBranches] = {};
  std::vector<int> unit_branch;  // branch of each solo launch, then of each packed group
  int n_branches = 0;
  bool det = false, autotune = false;
  int graph_steps = 100;
  int max_boxes = kMaxBatchBoxes;
  Arena* arena = nullptr;
  mpc_allocator alloc{};
  std::vector<mpc_handle> boxes;
  std::vector<uint64_t> gens;  // buffers_gen of each member at the last table upload
  std::vector<char> stepping;  // members below their step limit at the last plan
  Ctrl* ctrl_slab = nullptr;  // pinned control mirrors, one slot per member
  std::vector<int> free_slots;
  std::map<mpc_handle, int> slot_of;
  BatchTable* table_dev = nullptr;  // all members' arguments (closing kernel)
  BatchTable* table_host[kTableBuffers] = {};
  cudaEvent_t table_ev[kTableBuffers] = {};
  bool table_ev_live[kTableBuffers] = {};
  int table_next = 0;
  bool dirty = true;
  int total_items = 0;              // bricks of the packed members
  int64_t total_particles = 0;
  int num_sms = 0;
  int adv_grid = 0;
  uint32_t* counters = nullptr;     // one work-claiming counter per packed group
  struct Group {
    int variant = 0;
    int tier = 0;  // brick geometry compiled into the launch (0: any)
    size_t smem = 0;
    int grid = 0, ctas_per_sm = 0;
    PackTable table{};
  };
  std::vector<Group> groups;
  std::vector<StepArgs> solo_args;  // arguments of the solo members' launches
  int solo_bricks = 0;              // members with at least this many bricks run solo
  bool pack_all = false;
  cudaGraphExec_t graph = nullptr;
  bool graph_stale = true;
  int plan_uses = 0;  // batch-step calls on the current plan; graphs from the second on
  int graph_builds = 0;
  double plan_ms = 0.0;  // host time spent re-planning and capturing graphs
  std::map<std::string, std::pair<int, int>> tuned;
  std::string err;
};

namespace {

mpc_status bfail(mpc_batch b, mpc_status st, const std::string& msg) {
  if (b) b->err = msg;
  else g_batch_create_error = msg;
  return st;
}

#define BCU(b, call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bfail((b), MPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

size_t table_bytes(int nboxes) {
  return offsetof(BatchTable, args) + sizeof(StepArgs) * (size_t)nboxes;
}

// The launches of one step (solo members and packed groups) are independent: they are
// spread over up to kBranches forked streams (largest first, each to the least loaded
// branch) so that one launch's last partial wave overlaps the next launch.
void assign_branches(mpc_batch b) {
  const size_t units = b->solo_args.size() + b->groups.size();
  b->unit_branch.assign(units, 0);
  b->n_branches = (int)std::min<size_t>(units, kBranches);
  if (b->n_branches <= 1) return;
  std::vector<std::pair<int64_t, size_t>> work;  // (bricks, unit)
  for (size_t i = 0; i < b->solo_args.size(); ++i) work.push_back({b->solo_args[i].g.nbricks, i});
  for (size_t i = 0; i < b->groups.size(); ++i)
    work.push_back({b->groups[i].table.begin[b->groups[i].table.n], b->solo_args.size() + i});
  std::stable_sort(work.begin(), work.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<int64_t> load((size_t)b->n_branches, 0);
  for (const auto& w : work) {
    const size_t k = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
    b->unit_branch[w.second] = (int)k;
    load[k] += w.first;
  }
}

// Rebuilds the launch plan when members or their buffers changed: solo members, packed
// groups (sorted by variant and shared-memory need, kPackGroup boxes at most), and the
// device table of all members for the closing kernel.
mpc_status refresh(mpc_batch b) {
  // a member repaired or re-binned through its own handle has new buffers; a member at
  // its step limit is left out of the launches until its limit moves
  for (size_t i = 0; i < b->boxes.size() && !b->dirty; ++i) {
    const mpc_handle h = b->boxes[i];
    if (b->gens[i] != h->buffers_gen || b->stepping[i] != (!h->detached && h->limit > h->target_step))
      b->dirty = true;
  }
  if (!b->dirty) return MPC_OK;
  const int k = b->table_next;  // a pinned buffer whose previous upload has executed
  b->table_next = (k + 1) % kTableBuffers;
  if (b->table_ev_live[k]) BCU(b, cudaEventSynchronize(b->table_ev[k]));
  BatchTable* t = b->table_host[k];
  const int n = (int)b->boxes.size();
  std::vector<mpc_handle> packed;
  b->solo_args.clear();
  b->total_particles = 0;
  int nt = 0;  // members the closing kernel advances (detached ones step on their own)
  for (int i = 0; i < n; ++i) {
    mpc_handle h = b->boxes[(size_t)i];
    b->gens[(size_t)i] = h->buffers_gen;
    b->stepping[(size_t)i] = !h->detached && h->limit > h->target_step;
    if (!h->detached) t->args[nt++] = step_args(h);
    b->total_particles += h->N;
    if (!b->stepping[(size_t)i]) continue;
    if (!b->pack_all && h->g.nbricks >= b->solo_bricks) b->solo_args.push_back(t->args[nt - 1]);
    else packed.push_back(h);
  }
  t->nboxes = nt;
  std::stable_sort(packed.begin(), packed.end(), [](mpc_handle x, mpc_handle y) {
    if (x->g.variant != y->g.variant) return x->g.variant < y->g.variant;
    const int tx = brick_tier(x->g), ty = brick_tier(y->g);
    if (tx != ty) return tx > ty;
    return step_smem_bytes(x->g) < step_smem_bytes(y->g);
  });
  b->groups.clear();
  int64_t items = 0;
  for (size_t i = 0; i < packed.size(); ++i) {
    mpc_handle h = packed[i];
    const int tier = brick_tier(h->g);
    if (b->groups.empty() || b->groups.back().variant != h->g.variant ||
        b->groups.back().tier != tier || b->groups.back().table.n == kPackGroup) {
      b->groups.emplace_back();
      b->groups.back().variant = h->g.variant;
      b->groups.back().tier = tier;
    }
    mpc_batch_s::Group& G = b->groups.back();
    PackTable& P = G.table;
    if (P.n == 0) P.begin[0] = 0;
    P.args[P.n] = step_args(h);
    P.begin[P.n + 1] = P.begin[P.n] + h->g.nbricks;
    P.n += 1;
    G.smem = std::max(G.smem, step_smem_bytes(h->g));
    items += h->g.nbricks;
  }
  if ((int)b->groups.size() > b->max_boxes) return bfail(b, MPC_EINVAL, "too many packed groups");
  BCU(b, configure_step_kernels(device_smem_limit(b->device)));
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    mpc_batch_s::Group& G = b->groups[gi];
    G.table.counter = b->counters + gi;
    BCU(b, packed_kernel_occupancy(G.variant, G.tier, b->det, G.smem, &G.ctas_per_sm));
    if (G.ctas_per_sm < 1) return bfail(b, MPC_EINVAL, "the packed step kernel does not fit on an SM");
    G.grid = (int)std::min<int64_t>(G.table.begin[G.table.n], (int64_t)G.ctas_per_sm * b->num_sms);
  }
  b->total_items = (int)std::min<int64_t>(items, INT32_MAX);
  BCU(b, cudaMemcpyAsync(b->table_dev, t, table_bytes(n), cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaEventRecord(b->table_ev[k], b->stream));
  b->table_ev_live[k] = true;
  assign_branches(b);
  b->graph_stale = true;
  b->plan_uses = 0;
  b->dirty = false;
  return MPC_OK;
}

// one batch step: the solo members' own kernels, one persistent launch per packed
// group (their claim counters zeroed first), then the closing of every member's step
cudaError_t launch_batch_step(mpc_batch b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const int nb = b->n_branches;
  if (!b->groups.empty()) e = cudaMemsetAsync(b->counters, 0, sizeof(uint32_t) * b->groups.size(), s);
  if (e == cudaSuccess && nb > 1) {
    e = cudaEventRecord(b->fork_ev, s);
    for (int k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->branch[k], b->fork_ev, 0);
  }
  auto on = [&](size_t unit) { return nb > 1 ? b->branch[b->unit_branch[unit]] : s; };
  for (size_t i = 0; i < b->solo_args.size() && e == cudaSuccess; ++i)
    e = launch_step(b->solo_args[i], on(i));
  for (size_t i = 0; i < b->groups.size() && e == cudaSuccess; ++i) {
    const mpc_batch_s::Group& G = b->groups[i];
    e = launch_step_packed(G.table, G.variant, G.tier, b->det, G.grid, G.smem, on(b->solo_args.size() + i));
  }
  if (e == cudaSuccess && nb > 1) {
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b->join_ev[k], b->branch[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join_ev[k], 0);
    }
  }
  if (e == cudaSuccess) e = launch_advance_batch(b->table_dev, b->adv_grid, s);
  return e;
}

mpc_status build_graph(mpc_batch b) {
  if (b->graph && !b->graph_stale) return MPC_OK;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  BCU(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
  for (int k = 0; k < b->graph_steps; ++k) {
    const cudaError_t e = launch_batch_step(b, b->cap_stream);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(b->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      return bfail(b, MPC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
  }
  BCU(b, cudaStreamEndCapture(b->cap_stream, &g));
  const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, MPC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  b->graph_stale = false;
  b->graph_builds += 1;
  return MPC_OK;
}

std::string class_key(const mpc_params& p) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "v%d n%.6g t%d w%d f%u", p.variant, p.n_c, p.thermostat, p.walls_z,
                p.flags);
  return buf;
}

}  // namespace

namespace mpc {
namespace host {
void batch_set_detached(mpc_handle h, bool detached) {
  if (!h || h->detached == detached) return;
  h->detached = detached;
  if (h->batch) h->batch->dirty = true;
}
}  // namespace host
}  // namespace mpc

extern "C" {

mpc_status mpc_autotune(const mpc_params* p, void* stream, uint64_t max_smem_bytes,
                        int32_t* tile_particles, int32_t* threads_per_cell,
                        double* ns_per_particle_step) {
  if (!p || !tile_particles || !threads_per_cell)
    return fail(nullptr, MPC_EINVAL, "params and outputs are required");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MPC_ECUDA, "no CUDA device");
  }
  const size_t lim = device_smem_limit(dev);
  if (lim == 0) return fail(nullptr, MPC_ECUDA, "cannot query shared memory per block");
  // a cubic box of about 8M particles with p's physics
  mpc_params q = *p;
  const int edge = std::max(8, std::min(1024, (int)std::lround(std::cbrt(8.0e6 / std::max(p->n_c, 1e-3)))));
  q.L[0] = q.L[1] = q.L[2] = edge;
  q.capacity = 0;
  q.graph_steps = 8;
  q.flags &= ~(uint32_t)MPC_FLAG_DEBUG_CELLS;
  double best = 1e300;
  int best_tile = 0, best_tpc = 0;
  for (int tile : {320, 640, 1280}) {
    Geom g;
    int64_t N = 0;
    q.tile_particles = tile;
    q.threads_per_cell = 0;
    TRY(plan_box(&q, lim, g, N));
    if (max_smem_bytes && step_smem_bytes(g) > max_smem_bytes) continue;
    const int t0 = g.tpc;
    for (int tpc : {t0 / 2, t0, t0 * 2, t0 * 4}) {
      if (tpc < 1 || tpc > 32) continue;
      const int groups = kStepThreads / tpc;
      if ((g.brick_cells + groups - 1) / groups > 4) continue;
      q.threads_per_cell = tpc;
      mpc_handle h = nullptr;
      TRY(create_box(&q, static_cast<cudaStream_t>(stream), nullptr, nullptr, &h));
      double ms = 0.0;
      int32_t n = 0;
      mpc_status st = mpc_set_profiling(h, 1);
      if (st == MPC_OK) st = mpc_step(h, 3);
      if (st == MPC_OK) st = mpc_synchronize(h);
      if (st == MPC_OK) st = mpc_step(h, 8);
      if (st == MPC_OK) st = mpc_synchronize(h);
      if (st == MPC_OK) st = mpc_profile_step_kernel(h, &ms, &n);
      const std::string msg = h->err;
      destroy_box(h, true);
      if (st != MPC_OK) return fail(nullptr, st, "autotune: " + msg);
      const double ns = ms * 1e6 / (double)N;
      if (n > 0 && ns < best) {
        best = ns;
        best_tile = tile;
        best_tpc = tpc;
      }
    }
  }
  if (best_tile == 0) return fail(nullptr, MPC_ESTATE, "autotune found no candidate");
  *tile_particles = best_tile;
  *threads_per_cell = best_tpc;
  if (ns_per_particle_step) *ns_per_particle_step = best;
  return MPC_OK;
}

const char* mpc_batch_last_error(mpc_batch b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

mpc_status mpc_batch_destroy(mpc_batch b) {
  if (!b) return MPC_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  for (mpc_handle h : b->boxes) {
    h->batch = nullptr;
    destroy_box(h, true);
  }
  b->boxes.clear();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  delete b->arena;
  if (b->table_dev) cudaFree(b->table_dev);
  if (b->counters) cudaFree(b->counters);
  for (int k = 0; k < kTableBuffers; ++k) {
    if (b->table_host[k]) cudaFreeHost(b->table_host[k]);
    if (b->table_ev[k]) cudaEventDestroy(b->table_ev[k]);
  }
  if (b->ctrl_slab) cudaFreeHost(b->ctrl_slab);
  if (b->adm_stream) cudaStreamDestroy(b->adm_stream);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int k = 0; k < kBranches; ++k) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  delete b;
  return MPC_OK;
}

mpc_status mpc_batch_create(const mpc_batch_config* cfg, void* stream, mpc_batch* out) {
  if (!out) return bfail(nullptr, MPC_EINVAL, "out is NULL");
  *out = nullptr;
  mpc_batch_config c{};
  if (cfg) c = *cfg;
  if (c.graph_steps < 0 || c.max_boxes < 0 || c.max_boxes > kMaxBatchBoxes || c.reserved != 0 ||
      (c.flags & ~(uint32_t)(MPC_BATCH_DETERMINISTIC | MPC_BATCH_AUTOTUNE | MPC_BATCH_PACK_ALL)))
    return bfail(nullptr, MPC_EINVAL, "invalid batch configuration");
  mpc_batch b = new (std::nothrow) mpc_batch_s();
  if (!b) return bfail(nullptr, MPC_ENOMEM, "host allocation failed");
  auto bail = [&](mpc_status st, const std::string& msg) {
    mpc_batch_destroy(b);
    return bfail(nullptr, st, msg);
  };
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return bfail(nullptr, MPC_ECUDA, "no CUDA device");
  }
  b->stream = static_cast<cudaStream_t>(stream);
  b->det = (c.flags & MPC_BATCH_DETERMINISTIC) != 0;
  b->autotune = (c.flags & MPC_BATCH_AUTOTUNE) != 0;
  b->pack_all = (c.flags & MPC_BATCH_PACK_ALL) != 0;
  b->graph_steps = c.graph_steps > 0 ? c.graph_steps : 100;
  b->max_boxes = c.max_boxes > 0 ? c.max_boxes : kMaxBatchBoxes;
  if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return bail(MPC_ECUDA, "cannot query the SM count");

  b->adv_grid = b->num_sms;
  b->solo_bricks = kSoloWaves * kWaveCtasPerSm * b->num_sms;
  if (cudaStreamCreateWithFlags(&b->adm_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return bail(MPC_ECUDA, "stream creation failed");
  for (int k = 0; k < kBranches; ++k)
    if (cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(MPC_ECUDA, "stream creation failed");
  if (cudaMallocHost(&b->ctrl_slab, sizeof(Ctrl) * (size_t)b->max_boxes) != cudaSuccess) {
    b->ctrl_slab = nullptr;
    return bail(MPC_ENOMEM, "pinned host allocation failed");
  }
  for (int k = b->max_boxes - 1; k >= 0; --k) b->free_slots.push_back(k);
  if (cudaMalloc(&b->table_dev, sizeof(BatchTable)) != cudaSuccess) {
    b->table_dev = nullptr;
    return bail(MPC_ENOMEM, "device allocation failed: member table");
  }
  if (cudaMalloc(&b->counters, sizeof(uint32_t) * (size_t)b->max_boxes) != cudaSuccess) {
    b->counters = nullptr;
    return bail(MPC_ENOMEM, "device allocation failed: claim counters");
  }
  for (int k = 0; k < kTableBuffers; ++k) {
    if (cudaMallocHost(&b->table_host[k], sizeof(BatchTable)) != cudaSuccess) {
      b->table_host[k] = nullptr;
      return bail(MPC_ENOMEM, "pinned host allocation failed: member table");
    }
    if (cudaEventCreateWithFlags(&b->table_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(MPC_ECUDA, "event creation failed");
  }
  if (c.arena_bytes > 0) {
    b->arena = new (std::nothrow) Arena();
    if (!b->arena || !b->arena->init(c.arena_bytes))
      return bail(MPC_ENOMEM, "device allocation failed: arena");
    b->alloc.ctx = b->arena;
    b->alloc.alloc = arena_alloc;
    b->alloc.release = arena_release;
  }
  *out = b;
  return MPC_OK;
}

mpc_status mpc_batch_add(mpc_batch b, const mpc_params* p, mpc_handle* out) {
  if (!b) return bfail(nullptr, MPC_EINVAL, "batch is NULL");
  if (!p || !out) return bfail(b, MPC_EINVAL, "params and out are required");
  *out = nullptr;
  if ((int)b->boxes.size() >= b->max_boxes || b->free_slots.empty())
    return bfail(b, MPC_EINVAL, "the batch is full");
  BCU(b, cudaSetDevice(b->device));
  mpc_params q = *p;
  if (b->det) q.flags |= MPC_FLAG_DETERMINISTIC;
  else if (q.flags & MPC_FLAG_DETERMINISTIC)
    return bfail(b, MPC_EINVAL, "deterministic boxes need a batch created with MPC_BATCH_DETERMINISTIC");
  if (b->autotune && q.tile_particles == 0 && q.threads_per_cell == 0) {
    const std::string key = class_key(q);
    auto it = b->tuned.find(key);
    if (it == b->tuned.end()) {
      int32_t tile = 0, tpc = 0;
      double ns = 0.0;
      if (mpc_autotune(&q, b->adm_stream, 0, &tile, &tpc, &ns) != MPC_OK)
        return bfail(b, MPC_ECUDA, std::string("autotune: ") + mpc_last_error(nullptr));
      it = b->tuned.emplace(key, std::make_pair((int)tile, (int)tpc)).first;
    }
    q.tile_particles = it->second.first;
    q.threads_per_cell = it->second.second;
  }
  if (b->arena) {
    // quick refusal before touching the device: the arena cannot hold the creation peak
    uint64_t steady = 0, peak = 0;
    if (mpc_footprint(&q, &steady, &peak) != MPC_OK)
      return bfail(b, MPC_EINVAL, mpc_last_error(nullptr));
    b->arena->reclaim(false);
    if (peak > b->arena->size() - b->arena->used() + b->arena->pending())
      return bfail(b, MPC_ENOMEM, "the arena cannot hold the box");
  }
  const int slot = b->free_slots.back();
  mpc_handle h = nullptr;
  const mpc_status st = create_box(&q, b->adm_stream, b->arena ? &b->alloc : nullptr,
                                   b->ctrl_slab + slot, &h);
  if (st != MPC_OK) return bfail(b, st, mpc_last_error(nullptr));
  b->free_slots.pop_back();
  // the steps enqueued from now on see the created box
  cudaEvent_t ev = nullptr;
  BCU(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  BCU(b, cudaEventRecord(ev, b->adm_stream));
  BCU(b, cudaStreamWaitEvent(b->stream, ev, 0));
  cudaEventDestroy(ev);
  h->stream = b->stream;
  h->batch = b;
  b->slot_of[h] = slot;
  b->boxes.push_back(h);
  b->gens.push_back(h->buffers_gen);
  b->stepping.push_back(1);
  b->dirty = true;
  *out = h;
  return MPC_OK;
}

mpc_status mpc_batch_remove(mpc_batch b, mpc_handle h) {
  if (!b) return bfail(nullptr, MPC_EINVAL, "batch is NULL");
  auto it = std::find(b->boxes.begin(), b->boxes.end(), h);
  if (!h || it == b->boxes.end()) return bfail(b, MPC_EINVAL, "not a member of this batch");
  BCU(b, cudaSetDevice(b->device));
  b->gens.erase(b->gens.begin() + (it - b->boxes.begin()));
  b->stepping.erase(b->stepping.begin() + (it - b->boxes.begin()));
  b->boxes.erase(it);
  const int slot = b->slot_of[h];
  b->slot_of.erase(h);
  h->batch = nullptr;
  // with an arena, released blocks wait for an event on the batch stream; without one,
  // wait for the queued steps before cudaFree
  destroy_box(h, b->arena == nullptr);
  b->free_slots.push_back(slot);
  b->dirty = true;
  return MPC_OK;
}


mpc_status mpc_batch_step(mpc_batch b, int64_t nsteps) {
  if (!b) return bfail(nullptr, MPC_EINVAL, "batch is NULL");
  if (nsteps < 0) return bfail(b, MPC_EINVAL, "nsteps must be >= 0");
  BCU(b, cudaSetDevice(b->device));
  if (nsteps == 0 || b->boxes.empty()) return MPC_OK;
  const auto t_plan = std::chrono::steady_clock::now();
  if (mpc_status st = refresh(b); st != MPC_OK) return st;
  for (mpc_handle h : b->boxes)
    if (!h->detached) h->target_step += std::min(nsteps, h->limit - h->target_step);
  int64_t n = nsteps;
  // a plan used once (e.g. between admissions of a serving loop) is launched directly;
  // from its second use on it is captured
  const bool graphed = n >= b->graph_steps && b->plan_uses++ >= 1;
  if (graphed)
    if (mpc_status st = build_graph(b); st != MPC_OK) return st;
  b->plan_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count();
  if (graphed) {
    for (; n >= b->graph_steps; n -= b->graph_steps) BCU(b, cudaGraphLaunch(b->graph, b->stream));
  }
  for (; n > 0; --n) BCU(b, launch_batch_step(b, b->stream));
  return MPC_OK;
}

mpc_status mpc_batch_synchronize(mpc_batch b) {
  if (!b) return bfail(nullptr, MPC_EINVAL, "batch is NULL");
  BCU(b, cudaSetDevice(b->device));
  BCU(b, cudaStreamSynchronize(b->stream));
  mpc_status first = MPC_OK;
  for (mpc_handle h : b->boxes) {
    const mpc_status st = sync_and_repair(h);  // refresh() sees reallocated buffers
    if (st != MPC_OK && first == MPC_OK) {
      first = st;
      b->err = "member box: " + h->err;
    }
  }
  return first;
}

mpc_status mpc_batch_get_info(mpc_batch b, mpc_batch_info* out) {
  if (!b) return bfail(nullptr, MPC_EINVAL, "batch is NULL");
  if (!out) return bfail(b, MPC_EINVAL, "out is NULL");
  std::memset(out, 0, sizeof(*out));
  int64_t parts = 0;
  for (mpc_handle h : b->boxes) parts += h->N;
  out->n_boxes = (int32_t)b->boxes.size();
  out->work_items = b->total_items;
  out->n_particles = parts;
  if (b->arena) {
    b->arena->reclaim(false);
    out->arena_bytes = b->arena->size();
    out->arena_used = b->arena->used();
    out->arena_largest_free = b->arena->largest_free();
  }
  for (const mpc_batch_s::Group& G : b->groups) {
    out->grid += G.grid;
    out->ctas_per_sm = std::max(out->ctas_per_sm, G.ctas_per_sm);
    out->smem_bytes = std::max(out->smem_bytes, (int32_t)G.smem);
  }
  out->packed_launches = (int32_t)b->groups.size();
  out->plan_ms = (float)b->plan_ms;
  out->graph_builds = b->graph_builds;
  out->tuned_classes = (int32_t)b->tuned.size();
  out->solo_boxes = (int32_t)b->solo_args.size();
  return MPC_OK;
}

}  // extern "C"
