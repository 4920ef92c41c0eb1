// mpc_sort_by_cell_noalloc: the checkpoint ordering of mpc_get_state (particles sorted
// by unshifted cell, Sec. III.G.2 of the paper) for callers that cannot allocate device
// memory when they need it.  Such callers exist: a serving loop that hands all HBM to
// its own memory pool at start-up cannot get more from cudaMalloc, and code that runs
// while other streams keep the GPU busy must not pay the device-wide synchronisation
// that cudaFree implies.  This entry point therefore uses a fixed scratch area that is
// part of the library image instead of asking for memory: the caller passes the input
// and output arrays, and the histogram and scan partials live in `g_sort_scratch`.
//
// The array is a device symbol.  Host code cannot use its name as an address (on the
// host the name denotes a host-side shadow), so the device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, and cached.
#include <cstring>
#include <mutex>
#include <string>

#include "mpc.h"
#include "mpc_internal.h"

namespace mpc {
void set_null_handle_error(const std::string& msg);  // mpc_api.cu
}

namespace {

using namespace mpc;

// Largest box the scratch covers: 2^21 = 2,097,152 cells (e.g. 128^3).
constexpr int64_t kMaxCells = int64_t(1) << 21;
// Scan partials: scan_tmp_words(2^21) = 1025 words; keep a margin.
constexpr int64_t kScanWords = 4096;
constexpr int64_t kErrorWord = kMaxCells + kScanWords;

// Histogram / cursors (kMaxCells words), scan partials, one error word: 8.4 MB held on
// every device that loads the library, until the process exits.
static __device__ __align__(256) uint32_t g_sort_scratch[kMaxCells + kScanWords + 64];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

mpc_status fail(mpc_status st, const std::string& msg) {
  set_null_handle_error(msg);
  return st;
}

// device address of the scratch array on the current device (set up on first use and
// kept for the life of the process: a device reset after that first call is not supported)
mpc_status scratch_for_current_device(uint32_t** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MPC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MPC_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p)
      return fail(MPC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MPC_OK;
}

}  // namespace

extern "C" mpc_status mpc_sort_by_cell_noalloc(const int32_t L[3], int64_t n, const uint32_t* X,
                                               const float* V, const uint32_t* id, uint32_t* X_out,
                                               float* V_out, uint32_t* id_out, void* stream) {
  if (!L) return fail(MPC_EINVAL, "L is NULL");
  for (int ax = 0; ax < 3; ++ax)
    if (L[ax] < 2 || L[ax] > 1024) return fail(MPC_EINVAL, "L must lie in [2, 1024]");
  const int64_t cells = (int64_t)L[0] * L[1] * L[2];
  if (cells > kMaxCells)
    return fail(MPC_EINVAL, "box has " + std::to_string(cells) +
                                " cells; mpc_sort_by_cell_noalloc supports at most 2097152");
  if (n < 0 || n > 0xFFFFFFFFLL) return fail(MPC_EINVAL, "n must lie in [0, 2^32)");
  if (!X || !V || !X_out || !V_out) return fail(MPC_EINVAL, "X, V, X_out and V_out are required");
  if ((id == nullptr) != (id_out == nullptr)) return fail(MPC_EINVAL, "pass both id and id_out or neither");
  if (n == 0) return MPC_OK;

  uint32_t* scratch = nullptr;
  mpc_status st = scratch_for_current_device(&scratch);
  if (st != MPC_OK) return st;
  uint32_t* hist = scratch;
  uint32_t* scan_tmp = scratch + kMaxCells;
  int32_t* err_word = reinterpret_cast<int32_t*>(scratch + kErrorWord);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  Geom g{};
  g.F = fixed_bits_for(L);
  g.mask = (1u << g.F) - 1u;
  for (int ax = 0; ax < 3; ++ax) {
    g.L[ax] = L[ax];
    g.Lc[ax] = L[ax];
    g.P[ax] = (uint32_t)L[ax] << g.F;
  }
  g.ncells = cells;

  uint32_t* const xin[3] = {const_cast<uint32_t*>(X), const_cast<uint32_t*>(X) + n,
                            const_cast<uint32_t*>(X) + 2 * n};
  PBuf src{};
  PBuf dst{};
  for (int ax = 0; ax < 3; ++ax) {
    src.x[ax] = xin[ax];
    src.v[ax] = const_cast<float*>(V) + ax * n;
    dst.x[ax] = X_out + ax * n;
    dst.v[ax] = V_out + ax * n;
  }
  src.id = const_cast<uint32_t*>(id);
  dst.id = id_out;

  // positions outside the box would index past the histogram: reject them first
  int32_t host_err = 0;
  cudaError_t e = cudaMemsetAsync(err_word, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = launch_check_range(g, n, xin, err_word, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, err_word, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(MPC_ECUDA, std::string("range check: ") + cudaGetErrorString(e));
  if (host_err) return fail(MPC_EINVAL, "a position lies outside [0, L << F)");

  // the histogram keeps the previous call's counts: clear the part this box uses
  e = cudaMemsetAsync(hist, 0, (size_t)cells * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = launch_cell_hist(g, n, xin, hist, s);
  if (e == cudaSuccess) e = launch_scan(hist, hist, cells, scan_tmp, s);
  if (e == cudaSuccess) e = launch_cell_scatter(g, n, src, hist, dst, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(MPC_ECUDA, std::string("sort: ") + cudaGetErrorString(e));
  return MPC_OK;
}
