// Layout kernels around the fused step: initial state, binning of a contiguous particle
// set into brick buffers (create / set_state / overflow repair), brick compaction,
// the counting sort by unshifted cell used for checkpoints (Sec. III.G.2), an
// exclusive scan, and small reductions.
#include <cstdio>

#include "mpc_device.cuh"
#include "mpc_internal.h"

namespace mpc {

namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(int64_t n, int per_block = kBlock) {
  int64_t b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// warp-aggregated atomic increment of counter[key]: lanes with equal keys elect one
// leader that adds the group size; returns this lane's slot
__device__ __forceinline__ uint32_t aggregated_inc(uint32_t* counter, uint32_t key) {
  const uint32_t active = __activemask();
  const uint32_t peers = __match_any_sync(active, key);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&counter[key], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// streams a particle for step `step` (in place) and returns the brick of its collision
// cell in that step
__device__ __forceinline__ uint32_t stream_to_brick(const Geom& g, uint32_t& x, uint32_t& y, uint32_t& z,
                                                    float vx, float vy, float vz, uint3 S) {
  stream(g, x, y, z, vx, vy, vz);
  const int cx = cell_axis(g, x, S.x, 0), cy = cell_axis(g, y, S.y, 1),
            cz = cell_axis(g, z & ~kCrossedBit, S.z, 2);
  return (uint32_t)((cx >> g.Bs[0]) + g.nb[0] * ((cy >> g.Bs[1]) + g.nb[1] * (cz >> g.Bs[2])));
}

__global__ void k_init_particles(const Geom g, int64_t N, uint32_t* x0, uint32_t* x1, uint32_t* x2,
                                 float* v0, float* v1, float* v2, uint32_t* id, double* sums) {
  __shared__ double red[3][kBlock / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (i < N) {
    const uint4 r = draw(g, (uint32_t)i, 0u, kTagInitX, 0u);
    x0[i] = __umulhi(r.x, g.P[0]);
    x1[i] = __umulhi(r.y, g.P[1]);
    x2[i] = __umulhi(r.z, g.P[2]);
    const uint4 q = draw(g, (uint32_t)i, 0u, kTagInitV, 0u);
    const float2 a = normal2(q.x, q.y);
    const float b = normal2(q.z, q.w).x;
    vx = g.sigma * a.x;
    vy = g.sigma * a.y;
    vz = g.sigma * b;
    v0[i] = vx; v1[i] = vy; v2[i] = vz;
    id[i] = (uint32_t)i;
  }
  double dx = vx, dy = vy, dz = vz;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dx += __shfl_xor_sync(0xffffffffu, dx, o);
    dy += __shfl_xor_sync(0xffffffffu, dy, o);
    dz += __shfl_xor_sync(0xffffffffu, dz, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = dx; red[1][w] = dy; red[2][w] = dz; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) s += red[threadIdx.x][k];
    atomicAdd(&sums[threadIdx.x + 3 * (blockIdx.x % 64)], s);
  }
}

__global__ void k_sub_mean(int64_t N, float* v0, float* v1, float* v2, const double* sums) {
  __shared__ float mean[3];
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < 64; ++k) s += sums[threadIdx.x + 3 * k];
    mean[threadIdx.x] = (float)(s / (double)N);
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    v0[i] -= mean[0];
    v1[i] -= mean[1];
    v2[i] -= mean[2];
  }
}

__global__ void k_bin_count(const Geom g, int64_t N, const uint32_t* x0, const uint32_t* x1,
                            const uint32_t* x2, const float* v0, const float* v1, const float* v2,
                            uint32_t step, uint32_t* counts, int32_t* errors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (x0[i] >= g.P[0] || x1[i] >= g.P[1] || x2[i] >= g.P[2]) {
    atomicOr(errors, kErrRange);
    return;
  }
  const uint3 S = lattice_shift(g, step);
  uint32_t x = x0[i], y = x1[i], z = x2[i];
  const uint32_t b = stream_to_brick(g, x, y, z, v0[i], v1[i], v2[i], S);
  aggregated_inc(counts, b);
}

__global__ void k_bin_scatter(const Geom g, int64_t N, const uint32_t* x0, const uint32_t* x1,
                              const uint32_t* x2, const float* v0, const float* v1, const float* v2,
                              const uint32_t* id, const uint32_t* cell, uint32_t step, PBuf dst,
                              uint32_t* cnt, int32_t* errors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint3 S = lattice_shift(g, step);
  uint32_t x = x0[i], y = x1[i], z = x2[i];
  const uint32_t b = stream_to_brick(g, x, y, z, v0[i], v1[i], v2[i], S);
  const uint32_t slot = aggregated_inc(cnt, b);
  if (slot >= (uint32_t)g.cap) {
    atomicOr(errors, kErrRange);
    return;
  }
  // bricks hold positions already streamed for the coming step (see mpc_step.cuh)
  const size_t o = (size_t)b * g.cap + slot;
  dst.x[0][o] = x; dst.x[1][o] = y; dst.x[2][o] = z;
  dst.v[0][o] = v0[i]; dst.v[1][o] = v1[i]; dst.v[2][o] = v2[i];
  dst.id[o] = id[i];
  if (dst.cell) dst.cell[o] = cell ? cell[i] : 0xFFFFFFFFu;
}

__global__ void k_check_range(const Geom g, int64_t N, const uint32_t* x0, const uint32_t* x1,
                              const uint32_t* x2, int32_t* errors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N && (x0[i] >= g.P[0] || x1[i] >= g.P[1] || x2[i] >= g.P[2])) atomicOr(errors, kErrRange);
}

__global__ void k_max_u32(const uint32_t* in, int64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, in[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---- exclusive scan: tiles of 2048 (256 threads x 8) ----
constexpr int kScanPer = 8;
constexpr int kScanTile = kBlock * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint32_t wbase = 0, all = 0;
  for (int k = 0; k < kBlock / 32; ++k) {
    if (k < w) wbase += warp_tot[k];
    all += warp_tot[k];
  }
  __syncthreads();
  *total = all;
  return wbase + incl - v;
}

__global__ void k_scan_reduce(const uint32_t* in, int64_t n, uint32_t* block_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint32_t tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const uint32_t* in, uint32_t* out, int64_t n, const uint32_t* offsets) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  uint32_t v[kScanPer];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + k;
    v[k] = (i < n) ? in[i] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t run = block_exclusive(s, &tot) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

__global__ void k_compact(const Geom g, PBuf src, const uint32_t* cnt, const uint32_t* offsets, PBuf dst) {
  const int b = blockIdx.x;
  const uint32_t c = min(cnt[b], (uint32_t)g.cap);
  const size_t so = (size_t)b * g.cap;
  const size_t dof = offsets[b];
  for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
    dst.x[0][dof + k] = src.x[0][so + k];
    dst.x[1][dof + k] = src.x[1][so + k];
    dst.x[2][dof + k] = src.x[2][so + k];
    dst.v[0][dof + k] = src.v[0][so + k];
    dst.v[1][dof + k] = src.v[1][so + k];
    dst.v[2][dof + k] = src.v[2][so + k];
    dst.id[dof + k] = src.id[so + k];
    if (dst.cell && src.cell) dst.cell[dof + k] = src.cell[so + k];
  }
}

__global__ void k_append_spill(Spill sp, uint32_t count, uint64_t base, PBuf dst) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const size_t o = base + k;
  dst.x[0][o] = sp.x[0][k]; dst.x[1][o] = sp.x[1][k]; dst.x[2][o] = sp.x[2][k];
  dst.v[0][o] = sp.v[0][k]; dst.v[1][o] = sp.v[1][k]; dst.v[2][o] = sp.v[2][k];
  dst.id[o] = sp.id[k];
  if (dst.cell && sp.cell) dst.cell[o] = sp.cell[k];
}

// bricks store streamed positions: back to the state before the coming step
__global__ void k_unstream(const Geom g, int64_t N, PBuf b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  uint32_t x = b.x[0][i], y = b.x[1][i], z = b.x[2][i];
  unstream(g, x, y, z, b.v[0][i], b.v[1][i], b.v[2][i]);
  b.x[0][i] = x; b.x[1][i] = y; b.x[2][i] = z;
}

__device__ __forceinline__ uint32_t unshifted_cell(const Geom& g, uint32_t x, uint32_t y, uint32_t z) {
  return (x >> g.F) + (uint32_t)g.L[0] * ((y >> g.F) + (uint32_t)g.L[1] * (z >> g.F));
}

__global__ void k_cell_hist(const Geom g, int64_t N, const uint32_t* x0, const uint32_t* x1,
                            const uint32_t* x2, uint32_t* hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  aggregated_inc(hist, unshifted_cell(g, x0[i], x1[i], x2[i]));
}

__global__ void k_cell_scatter(const Geom g, int64_t N, PBuf src, uint32_t* cursor, PBuf dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t c = unshifted_cell(g, src.x[0][i], src.x[1][i], src.x[2][i]);
  const uint32_t o = aggregated_inc(cursor, c);
  dst.x[0][o] = src.x[0][i]; dst.x[1][o] = src.x[1][i]; dst.x[2][o] = src.x[2][i];
  dst.v[0][o] = src.v[0][i]; dst.v[1][o] = src.v[1][i]; dst.v[2][o] = src.v[2][i];
  if (dst.id) dst.id[o] = src.id[i];
  if (dst.cell && src.cell) dst.cell[o] = src.cell[i];
}

__global__ void k_reduce_obs(const Geom g, PBuf b, const uint32_t* cnt, double* out) {
  __shared__ double red[4][kBlock / 32];
  const int br = blockIdx.x;
  const uint32_t c = min(cnt[br], (uint32_t)g.cap);
  const size_t o = (size_t)br * g.cap;
  float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
    const float vx = b.v[0][o + k], vy = b.v[1][o + k], vz = b.v[2][o + k];
    s0 += vx; s1 += vy; s2 += vz;
    s3 += vx * vx + vy * vy + vz * vz;
  }
  double d[4] = {s0, s1, s2, s3};
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], off);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) red[q][w] = d[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) s += red[threadIdx.x][k];
    atomicAdd(&out[(br % kObsSlots) * 4 + threadIdx.x], s);
  }
}

// Velocity profile across the box along z: nbins equal slabs of [0, L_z); per slab the
// particle count and the sums of the velocity components, at the positions of the state
// contract (the stored, streamed positions unstreamed).  Global double atomics: an
// analysis pass, not part of the step.
__global__ void k_velocity_profile(const Geom g, PBuf b, const uint32_t* cnt, int nbins, double* out) {
  const int br = blockIdx.x;
  const uint32_t c = min(cnt[br], (uint32_t)g.cap);
  const size_t o = (size_t)br * g.cap;
  for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
    uint32_t x = b.x[0][o + k], y = b.x[1][o + k], z = b.x[2][o + k];
    const float vx = b.v[0][o + k], vy = b.v[1][o + k], vz = b.v[2][o + k];
    unstream(g, x, y, z, vx, vy, vz);
    const uint64_t slab = ((uint64_t)z * (uint64_t)nbins) / (uint64_t)g.P[2];
    double* q = out + 4 * min((int)slab, nbins - 1);
    atomicAdd(q, 1.0);
    atomicAdd(q + 1, (double)vx);
    atomicAdd(q + 2, (double)vy);
    atomicAdd(q + 3, (double)vz);
  }
}

}  // namespace

cudaError_t launch_velocity_profile(const Geom& g, const PBuf& b, const uint32_t* cnt, int nbins,
                                    double* out, cudaStream_t s) {
  k_velocity_profile<<<g.nbricks, kBlock, 0, s>>>(g, b, cnt, nbins, out);
  return cudaGetLastError();
}

cudaError_t launch_init_particles(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                                  uint32_t* id, double* sums, cudaStream_t s) {
  k_init_particles<<<grid_for(N), kBlock, 0, s>>>(g, N, x[0], x[1], x[2], v[0], v[1], v[2], id, sums);
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(int64_t N, float* const v[3], const double* sums, cudaStream_t s) {
  k_sub_mean<<<grid_for(N), kBlock, 0, s>>>(N, v[0], v[1], v[2], sums);
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                             int64_t step, uint32_t* counts, int32_t* errors, cudaStream_t s) {
  k_bin_count<<<grid_for(N), kBlock, 0, s>>>(g, N, x[0], x[1], x[2], v[0], v[1], v[2],
                                             (uint32_t)step, counts, errors);
  return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const Geom& g, int64_t N, uint32_t* const x[3], float* const v[3],
                               const uint32_t* id, const uint32_t* cell, int64_t step,
                               const PBuf& dst, uint32_t* cnt, int32_t* errors, cudaStream_t s) {
  k_bin_scatter<<<grid_for(N), kBlock, 0, s>>>(g, N, x[0], x[1], x[2], v[0], v[1], v[2], id, cell,
                                               (uint32_t)step, dst, cnt, errors);
  return cudaGetLastError();
}

cudaError_t launch_check_range(const Geom& g, int64_t N, uint32_t* const x[3], int32_t* errors,
                               cudaStream_t s) {
  k_check_range<<<grid_for(N), kBlock, 0, s>>>(g, N, x[0], x[1], x[2], errors);
  return cudaGetLastError();
}

cudaError_t launch_max_u32(const uint32_t* in, int64_t n, uint32_t* out, cudaStream_t s) {
  unsigned blocks = grid_for(n);
  if (blocks > 4096) blocks = 4096;
  k_max_u32<<<blocks, kBlock, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

size_t scan_tmp_words(int64_t n) {
  if (n <= kScanTile) return 0;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)nb + scan_tmp_words(nb);
}

cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n <= kScanTile) {
    k_scan_apply<<<1, kBlock, 0, s>>>(in, out, n, nullptr);
    return cudaGetLastError();
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<<<(unsigned)nb, kBlock, 0, s>>>(in, n, tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(tmp, tmp, nb, tmp + nb, s);
  if (e != cudaSuccess) return e;
  k_scan_apply<<<(unsigned)nb, kBlock, 0, s>>>(in, out, n, tmp);
  return cudaGetLastError();
}

cudaError_t launch_compact(const Geom& g, const PBuf& src, const uint32_t* cnt,
                           const uint32_t* offsets, const PBuf& dst, cudaStream_t s) {
  k_compact<<<g.nbricks, kBlock, 0, s>>>(g, src, cnt, offsets, dst);
  return cudaGetLastError();
}

cudaError_t launch_append_spill(const Spill& sp, uint32_t count, uint64_t base, const PBuf& dst,
                                cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_append_spill<<<grid_for(count), kBlock, 0, s>>>(sp, count, base, dst);
  return cudaGetLastError();
}

cudaError_t launch_unstream(const Geom& g, int64_t N, const PBuf& b, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_unstream<<<grid_for(N), kBlock, 0, s>>>(g, N, b);
  return cudaGetLastError();
}

cudaError_t launch_cell_hist(const Geom& g, int64_t N, uint32_t* const x[3], uint32_t* hist,
                             cudaStream_t s) {
  k_cell_hist<<<grid_for(N), kBlock, 0, s>>>(g, N, x[0], x[1], x[2], hist);
  return cudaGetLastError();
}

cudaError_t launch_cell_scatter(const Geom& g, int64_t N, const PBuf& src, uint32_t* cursor,
                                const PBuf& dst, cudaStream_t s) {
  k_cell_scatter<<<grid_for(N), kBlock, 0, s>>>(g, N, src, cursor, dst);
  return cudaGetLastError();
}

cudaError_t launch_reduce_obs(const Geom& g, const PBuf& b, const uint32_t* cnt, double* out,
                              cudaStream_t s) {
  k_reduce_obs<<<g.nbricks, kBlock, 0, s>>>(g, b, cnt, out);
  return cudaGetLastError();
}

}  // namespace mpc
