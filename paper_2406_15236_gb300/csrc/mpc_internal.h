// Internal types shared by the host API and the kernels of the MPC library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mpc {

// Everything a kernel needs to know about one box (passed by value).
struct Geom {
  int L[3];          // box edge in cells
  int Lc[3];         // extent of the collision-cell grid (Lz + 1 layers with walls)
  uint32_t P[3];     // L << F
  int F;             // fixed-point fraction bits
  uint32_t mask;     // 2^F - 1
  float hs;          // float32(h 2^F)
  float gh[3];       // float32(g h)
  float inv2F;       // 2^-F
  int walls;         // walls at z = 0, Lz: 0 none, 1 no-slip, 2 slip
  float wall_u[2];   // x velocity of the no-slip walls at z = 0 and z = Lz
  int B[3];          // cells per brick (powers of two)
  int Bs[3];         // log2 B
  int nb[3];         // bricks per axis
  int nbricks;
  int cap;           // particles per brick buffer
  int brick_cells;   // B[0] B[1] B[2]
  int tpc;           // threads cooperating on one cell in the finalisation
  int variant;       // 0 SRD, 1 AT+a, 2 SRD+a
  int thermostat;    // MBS after SRD
  float cos_a, sin_a;
  float sigma;       // sqrt(kT / m)
  float kT, m;
  double n_c;        // mean density (phantom particles)
  uint32_t key0, key1, box;
  uint32_t rk[20];   // Philox round keys: (key0 + r 0x9E3779B9, key1 + r 0xBB67AE85), r < 10
  int obs;           // accumulate observables
  int debug;         // keep collision cells and per-cell counts
  int det;           // fixed-point (order-independent) cell sums and observables
  int64_t ncells;    // Lc[0] Lc[1] Lc[2]
};

// Device-side control block of a box; written by the step kernels.
struct Ctrl {
  int64_t step;           // completed steps
  int64_t limit;          // steps stop (are skipped) once step reaches limit
  int32_t halted;         // a brick overflowed: later steps are skipped until repaired
  int32_t overflow;       // set during the step that overflowed
  int32_t lost;           // the spill area overflowed as well (state unrecoverable)
  int32_t errors;         // bit flags, see kErr*
  uint32_t spill_count;
  uint32_t pad;
};

enum : int32_t { kErrBinning = 1, kErrTimeout = 2, kErrRange = 4, kErrFixedRange = 8 };

// Particle buffer set: structure of arrays, nbricks * cap entries each.
struct PBuf {
  uint32_t* x[3];
  float* v[3];
  uint32_t* id;
  uint32_t* cell;  // collision cell of the last step (debug only, else nullptr)
};

struct Spill {
  uint32_t* x[3];
  float* v[3];
  uint32_t* id;
  uint32_t* cell;
  uint32_t* dest;
  uint32_t capacity;
};

constexpr int kStepThreads = 128;  // threads per CTA of the fused step kernel
constexpr int kBrickParticles = 640;  // target mean particles per brick
constexpr int kObsSlots = 128;   // partial-sum slots per step (spreads FP64 atomics)
constexpr int kObsWidth = 16;    // doubles per observables row

struct StepArgs {
  Geom g;
  PBuf buf[2];
  uint32_t* cnt[2];
  Ctrl* ctrl;
  Spill spill;
  double* obs_partials;   // kObsSlots * kObsWidth
  double* obs_series;     // ring * kObsWidth
  int obs_ring;
  uint32_t* dbg_counts;   // ncells (debug)
  // bricks left to the full-capacity pass of a step (their particles did not fit the
  // smaller shared-memory tile of the kernel that runs more CTAs per SM): word 0 counts
  // them, word 1 counts the CTAs of that pass that finished, words 2.. hold brick indices
  // (nbricks + 2 words, zero between steps)
  uint32_t* deferred;
};

// Step arguments of every member of a batch (device memory), for the kernel that
// closes each member's step.
constexpr int kMaxBatchBoxes = 4096;
struct BatchTable {
  int32_t nboxes;
  StepArgs args[kMaxBatchBoxes];
};

// Boxes of one packed launch, passed by value in kernel parameter space (at most 32 KB):
// box k owns the work items [begin[k], begin[k+1]).
constexpr int kPackGroup = 48;
struct PackTable {
  int32_t n;
  uint32_t* counter;  // work-claiming counter, zero when the launch starts
  int32_t begin[kPackGroup + 1];
  StepArgs args[kPackGroup];
};
static_assert(sizeof(PackTable) <= 32000, "PackTable must fit in kernel parameter space");

// Fixed-point fraction bits per cell of a box (the position contract): the largest
// F with max(L) 2^F <= 2^31, so every position and its sum with a lattice shift fits in
// 32 bits.  The one rule used by box planning, checkpoint files and the no-allocation sort.
inline int fixed_bits_for(const int L[3]) {
  const int lmax = L[0] > L[1] ? (L[0] > L[2] ? L[0] : L[2]) : (L[1] > L[2] ? L[1] : L[2]);
  int k = 0;
  while ((1LL << k) < (long long)lmax) ++k;
  return 31 - k;
}

// Philox4x32-10 round keys of a seed (the key schedule of Salmon et al., SC'11)
inline void round_keys(Geom& g) {
  for (int r = 0; r < 10; ++r) {
    g.rk[2 * r] = g.key0 + (uint32_t)r * 0x9E3779B9u;
    g.rk[2 * r + 1] = g.key1 + (uint32_t)r * 0xBB67AE85u;
  }
}

// launchers (mpc_step.cu)
size_t step_smem_bytes(const Geom& g);
// raises the dynamic shared-memory cap of every step kernel to the device limit
cudaError_t configure_step_kernels(size_t max_dynamic_smem);
cudaError_t launch_step(const StepArgs& a, cudaStream_t s);
cudaError_t launch_advance(const StepArgs& a, cudaStream_t s);
cudaError_t launch_store_i64(int64_t* p, int64_t v, cudaStream_t s);
// packed step of many small boxes of one variant and brick tier (all boxes of a launch
// share the tier; tier 0 = any geometry): CTAs of the kernel per SM, launch
int brick_tier(const Geom& g);
cudaError_t packed_kernel_occupancy(int variant, int tier, bool det, size_t smem_bytes, int* ctas_per_sm);
cudaError_t launch_step_packed(const PackTable& t, int variant, int tier, bool det, int grid,
                               size_t smem_bytes, cudaStream_t s);
// closes the step of every member of a batch
cudaError_t launch_advance_batch(const BatchTable* t, int grid, cudaStream_t s);

// launchers (mpc_layout.cu)
cudaError_t launch_init_particles(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                                  uint32_t* id, double* sums, cudaStream_t s);
cudaError_t launch_sub_mean(int64_t N, float* const v[3], const double* sums, cudaStream_t s);
cudaError_t launch_bin_count(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                             int64_t step, uint32_t* counts, int32_t* errors, cudaStream_t s);
cudaError_t launch_bin_scatter(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                               const uint32_t* id, const uint32_t* cell, int64_t step,
                               const PBuf& dst, uint32_t* cnt, int32_t* errors, cudaStream_t s);
cudaError_t launch_check_range(const Geom& g, int64_t N, uint32_t* const x[3], int32_t* errors,
                               cudaStream_t s);
cudaError_t launch_max_u32(const uint32_t* in, int64_t n, uint32_t* out, cudaStream_t s);
// exclusive scan of n uint32 into out (may alias in); tmp must hold scan_tmp_words(n)
size_t scan_tmp_words(int64_t n);
cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                        cudaStream_t s);
cudaError_t launch_compact(const Geom& g, const PBuf& src, const uint32_t* cnt,
                           const uint32_t* offsets, const PBuf& dst, cudaStream_t s);
cudaError_t launch_append_spill(const Spill& sp, uint32_t count, uint64_t base, const PBuf& dst,
                                cudaStream_t s);
// bricks hold streamed positions; converts a gathered set back to the state contract
cudaError_t launch_unstream(const Geom& g, int64_t N, const PBuf& b, cudaStream_t s);
cudaError_t launch_cell_hist(const Geom& g, int64_t N, uint32_t* const x[3], uint32_t* hist,
                             cudaStream_t s);
cudaError_t launch_cell_scatter(const Geom& g, int64_t N, const PBuf& src, uint32_t* cursor,
                                const PBuf& dst, cudaStream_t s);
cudaError_t launch_reduce_obs(const Geom& g, const PBuf& b, const uint32_t* cnt, double* out,
                              cudaStream_t s);
// per slab of nbins along z: count, sum vx, sum vy, sum vz (out: 4 nbins doubles, zeroed)
cudaError_t launch_velocity_profile(const Geom& g, const PBuf& b, const uint32_t* cnt, int nbins,
                                    double* out, cudaStream_t s);

}  // namespace mpc
