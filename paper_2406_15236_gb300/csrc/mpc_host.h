// Host-side internals shared by the single-box API (mpc_api.cu) and the batch and
// serving layers (mpc_batch.cu): the handle, its helpers and their error conventions.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "mpc.h"
#include "mpc_internal.h"

struct mpc_batch_s;

struct mpc_s {
  mpc_params p{};
  mpc::Geom g{};
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  mpc_allocator alloc{};
  bool has_alloc = false;
  int64_t N = 0;
  mpc::PBuf buf[2]{};
  uint32_t* cnt[2]{};
  mpc::Ctrl* ctrl = nullptr;
  mpc::Ctrl* ctrl_host = nullptr;  // pinned mirror
  bool ctrl_host_owned = true;     // false: a slot of a batch's pinned slab
  mpc::Spill spill{};
  double* obs_partials = nullptr;
  double* obs_series = nullptr;
  int obs_ring = 1024;
  uint32_t* dbg_counts = nullptr;
  uint32_t* deferred = nullptr;    // bricks deferred to the full-capacity pass
  int64_t target_step = 0;
  int64_t limit = INT64_MAX;       // the box stops advancing at this step
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 16;
  int recoveries = 0;
  size_t smem_limit = 0;
  mpc_batch_s* batch = nullptr;    // owning batch (members are destroyed through it)
  bool detached = false;           // a batch member stepped on its own (left out of the
                                   // batch's launches and closing kernel)
  uint64_t buffers_gen = 0;        // bumped whenever the particle buffers are reallocated
  // profiling: event pairs around step-kernel launches (graph nodes and single launches)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_begin, ev_end;
  int ev_next = 0;       // next slot for a single launch
  int ev_recorded = 0;   // valid pairs
  std::string err;
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;
};

namespace mpc {
namespace host {

mpc_status fail(mpc_handle h, mpc_status st, const std::string& msg);

#define CU(h, call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ::mpc::host::fail((h), MPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)                    \
  do {                               \
    mpc_status s_ = (expr);          \
    if (s_ != MPC_OK) return s_;     \
  } while (0)

// Geometry of a box before any allocation: brick shape, capacity, thread split, and the
// shared-memory budget of the device.  Fails with MPC_EINVAL like mpc_create.
mpc_status plan_box(const mpc_params* p, size_t smem_limit, Geom& g, int64_t& N);
size_t device_smem_limit(int device);  // opt-in shared memory per block minus static use

// Device bytes of a box's allocations without its observables ring: steady (held while
// it lives) and peak (during creation, which also holds the contiguous initial state
// and binning counts).
void box_footprint(const Geom& g, int64_t N, size_t& steady, size_t& peak);

// Creates a box on `stream`; ctrl_slot (pinned, may be NULL) replaces the handle's own
// pinned control mirror.
mpc_status create_box(const mpc_params* p, cudaStream_t stream, const mpc_allocator* alloc,
                      Ctrl* ctrl_slot, mpc_handle* out);
// Releases the handle; sync = false skips waiting for its stream (the caller guarantees
// that released device memory is not reused before queued work is done).
void destroy_box(mpc_handle h, bool sync);

StepArgs step_args(mpc_handle h);
mpc_status read_ctrl(mpc_handle h);
mpc_status sync_and_repair(mpc_handle h);
mpc_status set_step_limit(mpc_handle h, int64_t limit);
// detaches a member from its batch's steps (the caller steps it with mpc_step on a stream
// of its own) or attaches it again; the batch rebuilds its launch plan
void batch_set_detached(mpc_handle h, bool detached);

}  // namespace host
}  // namespace mpc
