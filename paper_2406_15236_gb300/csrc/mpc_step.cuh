// The fused MPC step: one CTA per brick of collision cells.
//
// Particles live in fixed-capacity brick buffers, binned by the collision cell they
// will occupy in the coming step, with their positions already streamed for that step
// (Eq. 1 with gravity kick and periodic / bounce-back walls; a wall crossing is kept in
// bit 31 of z) and the velocity they streamed with.  For step n a CTA
//   1. pulls its brick's particles (x, y, z, vx, vy, vz: 24 B each; the 4-byte ids too
//      for AT+a, whose random velocities are keyed by them) into shared memory with
//      bulk-async (TMA) copies,
//   2. finds their cell on the lattice shifted by S(n) -- inside this brick by
//      construction -- and counting-sorts them by cell in shared memory (integer
//      atomics give each particle its rank in its cell; a scan gives offsets),
//   3. finalises every cell from its contiguous member list with register reductions
//      over a few cooperating threads: SRD axis and MBS factor (Eqs. 2, 5-7) with
//      phantom particles in wall cells, or the AT+a angular velocity from the moments
//      about the cell's centre of mass,
//   4. applies the collision to every particle, streams it for step n+1 (its only
//      streaming per step), finds the brick of its next collision cell and ranks it
//      within its warp's group for that destination (shared-memory atomics),
//   5. per warp, without a block barrier (a thread writes out the particles it
//      collided): reserves the warp's run in each destination with one global atomic
//      and writes its particles out in contiguous runs, the ids read again from the
//      source brick (an L2 hit).
// HBM traffic per particle-step is one read and one write of the 28-byte particle: no
// global per-cell arrays, no second sweep, no separate reorder pass (the permanent
// reorder of Sec. III.B.3 happens in every step as part of the write).  Keeping the ids
// out of shared memory after the AT+a draws and 16-bit tags bring a brick to 26.5 KB
// (SRD) and 36.8 KB (AT+a) of dynamic shared memory: 8 and 6 CTAs per SM.
#pragma once

#include <cstdio>

#include "mpc_device.cuh"
#include "mpc_internal.h"

namespace mpc {

constexpr int kThreads = kStepThreads;

template <int VAR>
struct CellParams;
template <>
struct CellParams<0> {  // SRD: v_cm (3), rotation axis (3), kappa
  static constexpr int kParams = 7;
  static constexpr bool kStoresRandomVelocity = false;
};
template <>
struct CellParams<1> {  // AT+a: <w> - omega x rho_cm (3) with <w> = v_cm - <v_ran>, omega (3)
  static constexpr int kParams = 6;
  static constexpr bool kStoresRandomVelocity = true;
};
template <>
struct CellParams<2> {  // SRD+a: v_cm (3), omega (3), rho_cm (3), rotation axis (3)
  static constexpr int kParams = 12;
  static constexpr bool kStoresRandomVelocity = false;
};

// Dynamic shared memory of one brick.  The `stage` region is reused over the phases of
// a step: the particle ids for the AT+a random-velocity draws, then the member lists and
// cell parameters.
struct Layout {
  size_t x, y, z, vx, vy, vz, gcell, ux, uy, uz, tag, count, cstart, perm, params, total;
};

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ constexpr size_t max_sz(size_t a, size_t b) { return a > b ? a : b; }

__host__ __device__ constexpr Layout make_layout(int cap, int bc, int nparams, bool vran, int debug,
                                                 int tag_bytes) {
  Layout L{};
  size_t o = 0;
  const size_t a4 = align16(size_t(cap) * 4);
  L.x = o; o += a4;
  L.y = o; o += a4;
  L.z = o; o += a4;
  L.vx = o; o += a4;
  L.vy = o; o += a4;
  L.vz = o; o += a4;
  L.gcell = o; o += debug ? a4 : 0;
  L.ux = o; o += vran ? a4 : 0;
  L.uy = o; o += vran ? a4 : 0;
  L.uz = o; o += vran ? a4 : 0;
  L.tag = o; o += align16(size_t(cap) * tag_bytes);
  // cells: member counts and list offsets
  L.count = o;
  L.cstart = o + align16(size_t(bc) * 4);
  o += align16(size_t(bc) * 4) + align16(size_t(bc + 1) * 4);
  // stage: AT+a ids, then member lists and cell parameters
  const size_t lists = align16(size_t(cap) * 2) + align16(size_t(bc) * 4 * nparams);
  L.perm = o;
  L.params = o + align16(size_t(cap) * 2);
  o += max_sz(lists, vran ? a4 : 0);
  L.total = o;
  return L;
}


// Brick geometries compiled in: the default ~640-particle tiles (capacity 864) of
// 4x4x2, 4x4x4 and 8x4x4 cells.  With the shared-memory layout and the brick shape as
// constants, array addresses and cell arithmetic fold into immediates (about 6 % faster
// than reading them from the Geom).  TIER 0 takes everything from the Geom.
//
// scap: the shared-memory tile of the deferring kernel (MPC-AT+a on large boxes).  A
// brick's count is Poisson-like with mean 640 and deviation 25; a tile of 736 slots
// (3.8 deviations above the mean) instead of the full 864 brings an AT+a brick to 31.5 KB
// of shared memory, 7 CTAs per SM instead of 6.  The ~7e-5 of the bricks that hold more
// are deferred to a full-capacity pass after the main launch.
template <int TIER>
struct TierShape {
  static constexpr int cap = 0, scap = 0, Bs0 = 0, Bs1 = 0, Bs2 = 0;
};
template <>
struct TierShape<1> {
  static constexpr int cap = 864, scap = 736, Bs0 = 2, Bs1 = 2, Bs2 = 1;
};
template <>
struct TierShape<2> {
  static constexpr int cap = 864, scap = 736, Bs0 = 2, Bs1 = 2, Bs2 = 2;
};
template <>
struct TierShape<3> {
  static constexpr int cap = 864, scap = 736, Bs0 = 3, Bs1 = 2, Bs2 = 2;
};

// Boxes of an angular-momentum-conserving variant between no-slip walls take TIER 0: only
// that body carries the phantom particles' code, which costs the others 3 %.
__host__ __device__ inline int tier_of(const Geom& g) {
  if (g.cap != 864 || g.debug || (g.walls == 1 && g.variant != 0)) return 0;
  const int s0 = g.Bs[0], s1 = g.Bs[1], s2 = g.Bs[2];
  if (s0 == 2 && s1 == 2 && s2 == 1) return 1;
  if (s0 == 2 && s1 == 2 && s2 == 2) return 2;
  if (s0 == 3 && s1 == 2 && s2 == 2) return 3;
  return 0;
}

// Per-particle tag: collision cell in the brick | rank in that cell (phases 2-4), then
// destination code | rank in the destination group << 5 (phases 4-6).  Bricks of at
// most 64 cells and 864 slots fit both in 16 bits (cell: low log2(cells) bits, rank
// below 864); the others use 32 bits with the cell in the low 16.
template <int TIER>
struct TagOf {
  using type = uint32_t;
  static constexpr int kCellBits = 16;
};
template <>
struct TagOf<1> {
  using type = uint16_t;
  static constexpr int kCellBits = 5;
};
template <>
struct TagOf<2> {
  using type = uint16_t;
  static constexpr int kCellBits = 6;
};
constexpr uint32_t kNoCell = 0xFFFFu;  // tag of a particle not binned in this brick

template <int VAR>
__host__ __device__ inline Layout layout_for(const Geom& g) {
  const int t = tier_of(g);
  return make_layout(g.cap, g.brick_cells, CellParams<VAR>::kParams,
                     CellParams<VAR>::kStoresRandomVelocity, g.debug, (t == 1 || t == 2) ? 2 : 4);
}

// --- small PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// bounded wait on phase `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the `tpc` consecutive lanes that cooperate on one cell (tpc a power of two)
__device__ __forceinline__ float group_sum(float v, int tpc) {
  for (int o = tpc >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of 16 values at once: at each butterfly level a lane keeps half of its
// values and adds the partner's copy of that half (the other half goes to the partner),
// so 16 + 8 + 4 + 2 + 1 exchanges replace 16 x 5.  Lanes 2j and 2j + 1 end with the sum
// of value j over the warp.
template <class T>
__device__ __forceinline__ T warp_reduce_scatter16(T (&v)[16], int lane) {
  const bool hi8 = lane & 16, hi4 = lane & 8, hi2 = lane & 4, hi1 = lane & 2;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const T send = hi8 ? v[k] : v[k + 8];
    const T keep = hi8 ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T send = hi4 ? v[k] : v[k + 4];
    const T keep = hi4 ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T send = hi2 ? v[k] : v[k + 2];
    const T keep = hi2 ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const T send = hi1 ? v[0] : v[1];
    const T keep = hi1 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// brick-axis offset of a neighbour: 0 same, +-1 adjacent (with periodic wrap), 9 other
__device__ __forceinline__ int brick_delta(int q, int b, int nb, bool periodic) {
  int d = q - b;
  if (periodic) {
    if (d > 1) d -= nb;
    else if (d < -1) d += nb;
  }
  return (d >= -1 && d <= 1) ? d : 9;
}

// Fixed-point cell sums (deterministic mode, Sec. III.B "Reproducibility"): every
// per-particle term is converted to a 64-bit integer with 32 fraction bits and summed
// exactly, so a cell's sums do not depend on the order of its members, on the brick
// geometry or on the number of cooperating threads.  Terms must stay below 2^15 in
// magnitude (|t| n < 2^31 for the largest admissible cell); larger terms raise
// kErrFixedRange.  A float32 term above 2^-9 converts without rounding (smaller terms are
// truncated toward zero at 2^-32).
constexpr float kUnFx = 2.3283064365386963e-10f;   // 2^-32
constexpr float kFxLimit = 32768.0f;
// observables: 24 fraction bits (sums over whole boxes of up to ~2^30 particles)
constexpr double kObsUnFx = 5.9604644775390625e-08; // 2^-24

// v * 2^S as a 64-bit integer, from the IEEE-754 fields with integer operations only (the
// float-to-int64 conversion instruction issues at the FP64 rate on this GPU and made the
// deterministic step twice as slow): exact when v * 2^S is an integer, else truncated
// toward zero; |v| < 2^(38 - S) assumed (the callers' range checks flag larger terms).
template <int S>
__device__ __forceinline__ long long fixed_of(float v) {
  const uint32_t b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xFFu);
  const unsigned long long m = (b & 0x7FFFFFu) | (e != 0 ? 0x800000u : 0u);
  const int sh = e - (127 + 23 - S);  // v * 2^S = m * 2^sh
  const unsigned long long r = sh >= 0 ? (m << min(sh, 38)) : (m >> min(-sh, 32));
  const long long q = (long long)r;
  return (b >> 31) ? -q : q;
}

__device__ __forceinline__ long long to_fx(float v) { return fixed_of<32>(v); }
__device__ __forceinline__ float from_fx(long long s) { return __ll2float_rn(s) * kUnFx; }

__device__ __forceinline__ long long group_sum_fx(long long v, int tpc) {
  for (int o = tpc >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum_fx(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// position relative to the cell centre as an integer number of 2^-F units
__device__ __forceinline__ int rho_int(const Geom& g, uint32_t x, uint32_t s) {
  return (int)((x + s) & g.mask) - (int)(1u << (g.F - 1));
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Block-wide scalars of one brick's processing (static shared memory).
struct BrickShared {
  uint64_t bar;
  uint32_t cnt, halt;
  int64_t step;
  uint32_t wcount[4 * 28];  // per warp: particles bound for each destination code
  uint32_t shift[6];  // lattice shifts of this step and the next
};

// omega = J^-1 L for the moments M = sum r r^T and L = sum r x w about a cell's centre of
// mass (J = tr(M) 1 - M): the adjugate for n >= 3 (zero when det J <= 0, a collinear
// cell), the pseudo-inverse on the plane normal to the pair for n = 2, zero for n < 2
__device__ __forceinline__ float3 solve_omega(int n, float Mxx, float Myy, float Mzz, float Mxy,
                                              float Myz, float Mzx, float Lx, float Ly, float Lz) {
  const float tr = Mxx + Myy + Mzz;
  float3 om = make_float3(0.0f, 0.0f, 0.0f);
  if (n >= 3) {
    const float Jxx = tr - Mxx, Jyy = tr - Myy, Jzz = tr - Mzz;
    const float Jxy = -Mxy, Jyz = -Myz, Jzx = -Mzx;
    const float A00 = Jyy * Jzz - Jyz * Jyz, A01 = Jzx * Jyz - Jxy * Jzz,
                A02 = Jxy * Jyz - Jzx * Jyy, A11 = Jxx * Jzz - Jzx * Jzx,
                A12 = Jzx * Jxy - Jxx * Jyz, A22 = Jxx * Jyy - Jxy * Jxy;
    const float det = Jxx * A00 + Jxy * A01 + Jzx * A02;
    if (det > 0.0f) {
      const float id = 1.0f / det;
      om.x = (A00 * Lx + A01 * Ly + A02 * Lz) * id;
      om.y = (A01 * Lx + A11 * Ly + A12 * Lz) * id;
      om.z = (A02 * Lx + A12 * Ly + A22 * Lz) * id;
    }
  } else if (n == 2 && tr > 0.0f) {
    // pair: J = tr(M) (1 - d d^T/|d|^2); pseudo-inverse on the plane normal to d
    const float it = 1.0f / tr;
    const float mLx = (Mxx * Lx + Mxy * Ly + Mzx * Lz) * it;
    const float mLy = (Mxy * Lx + Myy * Ly + Myz * Lz) * it;
    const float mLz = (Mzx * Lx + Myz * Ly + Mzz * Lz) * it;
    om.x = (Lx - mLx) * it;
    om.y = (Ly - mLy) * it;
    om.z = (Lz - mLz) * it;
  }
  return om;
}

// --- one brick of one box ---------------------------------------------------------
// Processes brick b of the box described by `a`.  PERSIST: the caller initialised
// sh.bar once and tracks its phase (persistent kernels); otherwise the barrier is
// initialised here and phase must be 0.  DEFER (TIER > 0): the shared-memory tile holds
// T::scap particles, and a brick holding more is appended to a.deferred and left
// untouched (its count slot too) for the full-capacity pass.  PLAIN: the box is periodic,
// without gravity, with power-of-two extents (periodic_pow2_box): the kick, the wall
// handling and the general wrap are compiled out (5 % of the AT+a and SRD step).
// Returns false after a bounded wait gave up (the CTA must stop).
template <int VAR, bool DET, bool PERSIST, int TIER = 0, bool DEFER = false, bool PLAIN = false>
__device__ __forceinline__ bool step_brick(const StepArgs& a, const int b, unsigned char* smem,
                                           BrickShared& sh, uint32_t& phase) {
  const Geom& g = a.g;
  using T = TierShape<TIER>;
  static_assert(!DEFER || TIER > 0, "deferral needs a compiled-in brick tier");
  // the compiled-in tiers serve no debug boxes (tier_of), so their debug paths compile out
  const bool debug = TIER == 0 && g.debug;
  // brick geometry: compile-time constants for TIER > 0, else from the Geom
  const int cap = TIER ? T::cap : g.cap;
  // particles the shared-memory tile holds (the global brick slots hold cap)
  constexpr int kTile = DEFER ? T::scap : T::cap;
  const int Bs0 = TIER ? T::Bs0 : g.Bs[0], Bs1 = TIER ? T::Bs1 : g.Bs[1], Bs2 = TIER ? T::Bs2 : g.Bs[2];
  const int B0 = 1 << Bs0, B1 = 1 << Bs1, B2 = 1 << Bs2;
  using Tag = typename TagOf<TIER>::type;
  constexpr int kCellBits = TagOf<TIER>::kCellBits;
  constexpr uint32_t kCellMask = (1u << kCellBits) - 1u;
  const Layout lay = TIER ? make_layout(kTile, 1 << (T::Bs0 + T::Bs1 + T::Bs2), CellParams<VAR>::kParams,
                                        CellParams<VAR>::kStoresRandomVelocity, 0, (int)sizeof(Tag))
                          : make_layout(g.cap, g.brick_cells, CellParams<VAR>::kParams,
                                        CellParams<VAR>::kStoresRandomVelocity, g.debug, (int)sizeof(Tag));

  uint32_t* sx = reinterpret_cast<uint32_t*>(smem + lay.x);
  uint32_t* sy = reinterpret_cast<uint32_t*>(smem + lay.y);
  uint32_t* sz = reinterpret_cast<uint32_t*>(smem + lay.z);
  float* svx = reinterpret_cast<float*>(smem + lay.vx);  // SRD: v; AT+a: w = v - v_ran
  float* svy = reinterpret_cast<float*>(smem + lay.vy);
  float* svz = reinterpret_cast<float*>(smem + lay.vz);
  uint32_t* sid = reinterpret_cast<uint32_t*>(smem + lay.perm);  // stage: AT+a ids (phases 1-2)
  uint32_t* sgc = reinterpret_cast<uint32_t*>(smem + lay.gcell);
  float* sux = reinterpret_cast<float*>(smem + lay.ux);  // AT+a: v_ran
  float* suy = reinterpret_cast<float*>(smem + lay.uy);
  float* suz = reinterpret_cast<float*>(smem + lay.uz);
  Tag* stag = reinterpret_cast<Tag*>(smem + lay.tag);
  uint16_t* sperm = reinterpret_cast<uint16_t*>(smem + lay.perm);  // stage: member lists
  uint32_t* scount = reinterpret_cast<uint32_t*>(smem + lay.count);
  uint32_t* scstart = reinterpret_cast<uint32_t*>(smem + lay.cstart);
  float* spar = reinterpret_cast<float*>(smem + lay.params);

  uint32_t* wcount = sh.wcount;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int bc = TIER ? (1 << (T::Bs0 + T::Bs1 + T::Bs2)) : g.brick_cells;

  // ---- 1. load the brick: thread 0 reads the step, its limit, the halt flag and both
  // count slots in one round trip, then starts the bulk copies ----
  if (tid == 0) {
    // the barrier's init fence goes first, with no memory operation of its own to wait for
    if (!PERSIST) mbar_init(&sh.bar, 1);
    const int64_t st = *(volatile int64_t*)&a.ctrl->step;
    const int64_t lim = *(volatile int64_t*)&a.ctrl->limit;
    const int32_t halted = *(volatile int32_t*)&a.ctrl->halted;
    const uint32_t c_even = a.cnt[0][b], c_odd = a.cnt[1][b];
    const bool skip = halted || st >= lim;
    sh.step = st;
    sh.halt = skip;
    uint32_t c = 0;
    const int p = (int)(st & 1);
    if (!skip) {
      c = p ? c_odd : c_even;
      if (c > (uint32_t)cap) c = cap;
    }
    if (DEFER && !skip && c > (uint32_t)kTile) {
      // too many for this tile: the full-capacity pass takes the brick (its count stays)
      const uint32_t k = atomicAdd(&a.deferred[0], 1u);
      a.deferred[2 + k] = (uint32_t)b;
      sh.halt = 1;
      c = 0;
    } else if (!skip) {
      const uint32_t bytes = (uint32_t)(((c + 3) & ~3u) * 4);
      // AT+a draws its random velocities from the ids now; the other variants need the
      // ids only for the write-out, which reads them from the source brick (into L2 now)
      mbar_expect_tx(&sh.bar, (VAR == 1 ? 7u : 6u) * bytes);
      if (bytes) {
        const PBuf& sb = a.buf[p];
        const size_t off = (size_t)b * cap;
        bulk_g2s(sx, sb.x[0] + off, bytes, &sh.bar);
        bulk_g2s(sy, sb.x[1] + off, bytes, &sh.bar);
        bulk_g2s(sz, sb.x[2] + off, bytes, &sh.bar);
        bulk_g2s(svx, sb.v[0] + off, bytes, &sh.bar);
        bulk_g2s(svy, sb.v[1] + off, bytes, &sh.bar);
        bulk_g2s(svz, sb.v[2] + off, bytes, &sh.bar);
        if (VAR == 1) bulk_g2s(sid, sb.id + off, bytes, &sh.bar);
        else bulk_prefetch_l2(sb.id + off, bytes);
      }
      a.cnt[p][b] = 0;  // this buffer becomes the destination of the next step
    }
    sh.cnt = c;
  }
  if (tid < 4 * 28) wcount[tid] = 0;
  for (int c = tid; c < bc; c += kThreads) scount[c] = 0;
  __syncthreads();
  if (sh.halt) return true;
  const int64_t step64 = sh.step;
  const uint32_t step = (uint32_t)step64;
  const int par = (int)(step64 & 1);
  const PBuf& dst = a.buf[par ^ 1];
  uint32_t* cnt_dst = a.cnt[par ^ 1];
  const int cnt = (int)sh.cnt;
  // lattice shifts of this step and the next, drawn by one thread each while the bulk
  // copies are in flight; the barrier after the wait publishes them
  if (tid == 0 || tid == 32) {
    const uint3 t = lattice_shift(g, step + (tid >> 5));
    uint32_t* o = sh.shift + 3 * (tid >> 5);
    o[0] = t.x; o[1] = t.y; o[2] = t.z;
  }
  {
    // every thread waits (bounded); the block leaves together if any wait gave up
    const bool ok = mbar_wait(&sh.bar, phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(&a.ctrl->errors, kErrTimeout);
      if (!ok) mbar_wait(&sh.bar, phase);  // one more bounded chance for copies in flight
      return false;
    }
    phase ^= 1u;
  }
  const uint32_t S0x = sh.shift[0], S0y = sh.shift[1], S0z = sh.shift[2];
  const uint32_t S1x = sh.shift[3], S1y = sh.shift[4], S1z = sh.shift[5];

  const int bx = b % g.nb[0];
  const int by = (b / g.nb[0]) % g.nb[1];
  const int bz = b / (g.nb[0] * g.nb[1]);
  const int ox = bx << Bs0, oy = by << Bs1, oz = bz << Bs2;
  // bricks whose lower neighbour exists and whose upper neighbour is a whole brick inside
  // the box, on every axis: the cells a particle of this brick can reach within one brick
  // need no periodic wrap, so brick deltas follow from one shift per axis (a ragged box's
  // partial last brick is too narrow for that: one step past it wraps to cell 0)
  const bool inner = TIER > 0 && bx >= 1 && ((bx + 2) << Bs0) <= g.Lc[0] && by >= 1 &&
                     ((by + 2) << Bs1) <= g.Lc[1] && bz >= 1 && ((bz + 2) << Bs2) <= g.Lc[2];
  const uint32_t Ox = (uint32_t)ox << g.F, Oy = (uint32_t)oy << g.F, Oz = (uint32_t)oz << g.F;

  // ---- 2. rank each particle within its collision cell ----
  // Stored positions are already streamed for this step (the previous step streamed
  // them when it predicted their brick); the stored velocity is the one they streamed
  // with, before the kick.
  bool binerr = false;
  for (int i = tid; i < cnt; i += kThreads) {
    const uint32_t zraw = sz[i];
    const uint32_t x = sx[i], y = sy[i], z = zraw & ~kCrossedBit;
    float vx = svx[i], vy = svy[i], vz = svz[i];
    if constexpr (!PLAIN) collision_velocity(g, zraw, vx, vy, vz);
    int cx = 0, cy = 0, cz = 0, lx, ly, lz;
    if (inner) {
      lx = (int)(x + S0x - Ox) >> g.F;
      ly = (int)(y + S0y - Oy) >> g.F;
      lz = (int)(z + S0z - Oz) >> g.F;
    } else {
      cx = cell_axis(g, x, S0x, 0); cy = cell_axis(g, y, S0y, 1); cz = cell_axis(g, z, S0z, 2);
      lx = cx - ox; ly = cy - oy; lz = cz - oz;
    }
    // a particle outside the brick's cells is kept but skips its collision (kNoCell)
    const bool in = (unsigned)lx < (unsigned)B0 && (unsigned)ly < (unsigned)B1 && (unsigned)lz < (unsigned)B2;
    const uint32_t lc = in ? (uint32_t)(lx | (ly << Bs0) | (lz << (Bs0 + Bs1))) : 0u;
    uint32_t rank = 0;
    if (in) rank = atomicAdd(&scount[lc], 1u);
    const uint32_t lcr = in ? (lc | (rank << kCellBits)) : kNoCell;
    binerr |= !in;
    stag[i] = (Tag)lcr;
    if (debug) sgc[i] = (uint32_t)cx + (uint32_t)g.Lc[0] * ((uint32_t)cy + (uint32_t)g.Lc[1] * (uint32_t)cz);
    if constexpr (VAR == 1) {
      // AT+a: keep v_ran and w = v - v_ran
      const float3 u = normal3_at(draw(g, sid[i], step, kTagAtVel, 0u), g.sigma);
      const float ux = u.x, uy = u.y, uz = u.z;
      sux[i] = ux; suy[i] = uy; suz[i] = uz;
      vx -= ux; vy -= uy; vz -= uz;
    }
    svx[i] = vx; svy[i] = vy; svz[i] = vz;
  }
  if (binerr) atomicOr(&a.ctrl->errors, kErrBinning);
  __syncthreads();

  // ---- 3a. offsets of the cells' member lists ----
  if (tid < 32) {
    const int per = (bc + 31) >> 5;
    const int c0 = lane * per;
    uint32_t s = 0;
    for (int k = 0; k < per; ++k)
      if (c0 + k < bc) s += scount[c0 + k];
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t run = incl - s;
    for (int k = 0; k < per; ++k)
      if (c0 + k < bc) {
        scstart[c0 + k] = run;
        run += scount[c0 + k];
      }
    if (lane == 31) scstart[bc] = incl;
  }
  __syncthreads();
  for (int i = tid; i < cnt; i += kThreads) {
    const uint32_t lcr = stag[i];
    if (lcr != kNoCell) sperm[scstart[lcr & kCellMask] + (lcr >> kCellBits)] = (uint16_t)i;
  }
  __syncthreads();

  // ---- 3b. finalise every cell: `tpc` lanes reduce over its member list ----
  {
    const int tpc = g.tpc;
    const int groups = kThreads / tpc;
    const int grp = tid / tpc, sub = tid & (tpc - 1);
    const int leader = lane & ~(tpc - 1);
    float fxbig = 0.0f;  // deterministic mode: largest fixed-point term seen by this lane
    for (int c0 = 0; c0 < bc; c0 += groups) {
      const int lc = c0 + grp;
      const int cx = ox + (lc & (B0 - 1));
      const int cy = oy + ((lc >> Bs0) & (B1 - 1));
      const int cz = oz + (lc >> (Bs0 + Bs1));
      const bool exists = lc < bc && cx < g.Lc[0] && cy < g.Lc[1] && cz < g.Lc[2];
      const uint32_t cg = (uint32_t)cx + (uint32_t)g.Lc[0] * ((uint32_t)cy + (uint32_t)g.Lc[1] * (uint32_t)cz);
      const int n = exists ? (int)scount[lc] : 0;
      const int base = exists ? (int)scstart[lc] : 0;
      if (exists && sub == 0 && debug) a.dbg_counts[cg] = (uint32_t)n;
      if constexpr (VAR == 0) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        if constexpr (DET) {
          long long q0 = 0, q1 = 0, q2 = 0;
          for (int k = sub; k < n; k += tpc) {
            const int i = sperm[base + k];
            const float v0 = svx[i], v1 = svy[i], v2 = svz[i];
            fxbig = fmaxf(fxbig, fmaxf(fabsf(v0), fmaxf(fabsf(v1), fabsf(v2))));
            q0 += to_fx(v0); q1 += to_fx(v1); q2 += to_fx(v2);
          }
          q0 = group_sum_fx(q0, tpc); q1 = group_sum_fx(q1, tpc); q2 = group_sum_fx(q2, tpc);
          s0 = from_fx(q0); s1 = from_fx(q1); s2 = from_fx(q2);
        } else {
          for (int k = sub; k < n; k += tpc) {
            const int i = sperm[base + k];
            s0 += svx[i]; s1 += svy[i]; s2 += svz[i];
          }
          s0 = group_sum(s0, tpc); s1 = group_sum(s1, tpc); s2 = group_sum(s2, tpc);
        }
        // phantom particles fill the wall part of a cut cell at the mean density
        // (Sec. II, Boundary conditions): Poisson count, Gaussian total momentum, and
        // an internal kinetic energy ~ kT chi^2(3(n_ph - 1)); drawn by the group leader
        float nph = 0.f, Px = 0.f, Py = 0.f, Pz = 0.f, Kint = 0.f;
        if (!PLAIN && exists && n > 0 && sub == 0 && g.walls == 1 && (cz == 0 || cz == g.L[2])) {
          const double sz_ = (double)S0z * (double)g.inv2F;
          const double phi = (cz == 0) ? sz_ : 1.0 - sz_;
          const uint4 r = draw(g, cg, step, kTagPhantom, 0u);
          const uint4 r1 = draw(g, cg, step, kTagPhantom, 1u);
          const int k = poisson_inv((double)u01(r.x), g.n_c * phi);
          nph = (float)k;
          const float2 zxy = normal2(r.y, r.z);
          const float zz = normal2(r1.x, r1.y).x;
          const float sp = g.m * sqrtf(nph * g.kT / g.m);
          // phantoms move with their wall on average
          Px = sp * zxy.x + g.m * nph * g.wall_u[cz == 0 ? 0 : 1];
          Py = sp * zxy.y; Pz = sp * zz;
          if (k >= 2) Kint = g.kT * 2.0f * gamma_mt(g, cg, step, kTagPhGamma, 1.5f * (float)(k - 1));
        }
        if (tpc > 1) {
          nph = __shfl_sync(0xffffffffu, nph, leader);
          Px = __shfl_sync(0xffffffffu, Px, leader);
          Py = __shfl_sync(0xffffffffu, Py, leader);
          Pz = __shfl_sync(0xffffffffu, Pz, leader);
        }
        const float ntot = (float)n + nph;
        const float inv = 1.0f / (g.m * fmaxf(ntot, 1.0f));
        const float vcx = (g.m * s0 + Px) * inv, vcy = (g.m * s1 + Py) * inv,
                    vcz = (g.m * s2 + Pz) * inv;
        float kappa = 1.0f;
        if (g.thermostat) {
          // MBS, Eqs. (5)-(7): relative kinetic energy about v_cm (second pass)
          float q = 0.f;
          if constexpr (DET) {
            long long qq = 0;
            for (int k = sub; k < n; k += tpc) {
              const int i = sperm[base + k];
              const float dx = svx[i] - vcx, dy = svy[i] - vcy, dz = svz[i] - vcz;
              const float t = dx * dx + dy * dy + dz * dz;
              fxbig = fmaxf(fxbig, t);
              qq += to_fx(t);
            }
            q = from_fx(group_sum_fx(qq, tpc));
          } else {
            for (int k = sub; k < n; k += tpc) {
              const int i = sperm[base + k];
              const float dx = svx[i] - vcx, dy = svy[i] - vcy, dz = svz[i] - vcz;
              q += dx * dx + dy * dy + dz * dz;
            }
            q = group_sum(q, tpc);
          }
          if (exists && n > 0 && sub == 0 && ntot >= 2.0f) {
            float Krel = g.m * q;
            if (nph > 0.0f) {
              const float dx = Px / (g.m * nph) - vcx, dy = Py / (g.m * nph) - vcy,
                          dz = Pz / (g.m * nph) - vcz;
              Krel += Kint + nph * g.m * (dx * dx + dy * dy + dz * dz);
            }
            const float Ek = g.kT * gamma_mt(g, cg, step, kTagMbs, 1.5f * (ntot - 1.0f));
            if (Krel > 0.0f) kappa = sqrtf(2.0f * Ek / Krel);
          }
        }
        if (exists && n > 0 && sub == 0) {
          const uint4 r = draw(g, cg, step, kTagAxis, 0u);
          const float ct = 2.0f * u01(r.x) - 1.0f;
          const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
          float sphi, cphi;
          sincospif(2.0f * u01(r.y), &sphi, &cphi);
          float* P = spar + lc;
          P[0 * bc] = vcx; P[1 * bc] = vcy; P[2 * bc] = vcz;
          P[3 * bc] = st * cphi; P[4 * bc] = st * sphi; P[5 * bc] = ct;
          P[6 * bc] = kappa;
        }
      } else {
        // angular-momentum-conserving variants.  First pass: centre of mass and mean of
        // w (AT+a: w = v - v_ran; SRD+a: w = v, so the mean is v_cm).  In a cell cut by a
        // no-slip wall the phantom particles of the wall part are members too (drawn one
        // by one: their positions enter the moments); the group's lanes share them like
        // the fluid members
        float r0 = 0.f, r1 = 0.f, r2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
        constexpr bool kOnePass = VAR == 1 && !DET;
        int nph = 0;
        const int pwall = cz == 0 ? 0 : 1;
        if (TIER == 0 && g.walls == 1 && exists && n > 0 && (cz == 0 || cz == g.L[2])) {
          const double sz_ = (double)S0z * (double)g.inv2F;
          const double phi = (cz == 0) ? sz_ : 1.0 - sz_;
          nph = poisson_inv((double)u01(draw(g, cg, step, kTagPhantom, 0u).x), g.n_c * phi);
        }
        float o_m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if constexpr (DET) {
          // positions sum exactly as integers; velocities in fixed point
          long long R0 = 0, R1 = 0, R2 = 0, W0 = 0, W1 = 0, W2 = 0;
          for (int k = sub; k < n; k += tpc) {
            const int i = sperm[base + k];
            R0 += rho_int(g, sx[i], S0x); R1 += rho_int(g, sy[i], S0y);
            R2 += rho_int(g, sz[i] & ~kCrossedBit, S0z);
            const float v0 = svx[i], v1 = svy[i], v2 = svz[i];
            fxbig = fmaxf(fxbig, fmaxf(fabsf(v0), fmaxf(fabsf(v1), fabsf(v2))));
            W0 += to_fx(v0); W1 += to_fx(v1); W2 += to_fx(v2);
          }
          for (int j = sub; j < nph; j += tpc) {
            const PhantomParticle q = phantom_particle(g, cg, step, j, S0z, pwall);
            R0 += q.ix; R1 += q.iy; R2 += q.iz;
            const float v0 = VAR == 1 ? q.vx - q.ux : q.vx, v1 = VAR == 1 ? q.vy - q.uy : q.vy,
                        v2 = VAR == 1 ? q.vz - q.uz : q.vz;
            fxbig = fmaxf(fxbig, fmaxf(fabsf(v0), fmaxf(fabsf(v1), fabsf(v2))));
            W0 += to_fx(v0); W1 += to_fx(v1); W2 += to_fx(v2);
          }
          R0 = group_sum_fx(R0, tpc); R1 = group_sum_fx(R1, tpc); R2 = group_sum_fx(R2, tpc);
          W0 = group_sum_fx(W0, tpc); W1 = group_sum_fx(W1, tpc); W2 = group_sum_fx(W2, tpc);
          r0 = __ll2float_rn(R0) * g.inv2F; r1 = __ll2float_rn(R1) * g.inv2F;
          r2 = __ll2float_rn(R2) * g.inv2F;
          w0 = from_fx(W0); w1 = from_fx(W1); w2 = from_fx(W2);
        } else {
          // positions in units of 2^-F (integers, exact in float32): the sums are scaled by
          // the powers of two at the end, which changes no rounding
          auto first_term = [&](float px, float py, float pz, float vx, float vy, float vz) {
            r0 += px; r1 += py; r2 += pz;
            w0 += vx; w1 += vy; w2 += vz;
            if constexpr (kOnePass) {
              o_m[0] = fmaf(px, px, o_m[0]); o_m[1] = fmaf(py, py, o_m[1]); o_m[2] = fmaf(pz, pz, o_m[2]);
              o_m[3] = fmaf(px, py, o_m[3]); o_m[4] = fmaf(py, pz, o_m[4]); o_m[5] = fmaf(pz, px, o_m[5]);
              o_m[6] = fmaf(-pz, vy, fmaf(py, vz, o_m[6]));
              o_m[7] = fmaf(-px, vz, fmaf(pz, vx, o_m[7]));
              o_m[8] = fmaf(-py, vx, fmaf(px, vy, o_m[8]));
            }
          };
          for (int k = sub; k < n; k += tpc) {
            const int i = sperm[base + k];
            first_term((float)rho_int(g, sx[i], S0x), (float)rho_int(g, sy[i], S0y),
                       (float)rho_int(g, sz[i] & ~kCrossedBit, S0z), svx[i], svy[i], svz[i]);
          }
          for (int j = sub; j < nph; j += tpc) {
            const PhantomParticle q = phantom_particle(g, cg, step, j, S0z, pwall);
            first_term((float)q.ix, (float)q.iy, (float)q.iz, VAR == 1 ? q.vx - q.ux : q.vx,
                       VAR == 1 ? q.vy - q.uy : q.vy, VAR == 1 ? q.vz - q.uz : q.vz);
          }
          r0 = group_sum(r0, tpc); r1 = group_sum(r1, tpc); r2 = group_sum(r2, tpc);
          w0 = group_sum(w0, tpc); w1 = group_sum(w1, tpc); w2 = group_sum(w2, tpc);
          r0 *= g.inv2F; r1 *= g.inv2F; r2 *= g.inv2F;
          if constexpr (kOnePass) {
            const float s2 = g.inv2F * g.inv2F;
#pragma unroll
            for (int q = 0; q < 9; ++q) o_m[q] = group_sum(o_m[q], tpc) * (q < 6 ? s2 : g.inv2F);
          }
        }
        const int nt = n + nph;  // members: fluid and phantom particles
        const float inv = 1.0f / fmaxf((float)nt, 1.0f);
        const float rcx = r0 * inv, rcy = r1 * inv, rcz = r2 * inv;
        const float wmx = w0 * inv, wmy = w1 * inv, wmz = w2 * inv;
        // float AT+a takes the moments from the first pass's raw sums about the cell
        // centre, M = sum rho rho^T - n rho_c rho_c^T and L = sum rho x w - n rho_c x <w>;
        // where the members sit close together away from the centre these differences
        // cancel (sum |rho|^2 > 4 tr M), and such cells take the second pass about the
        // centre of mass
        float Mxx = 0.f, Myy = 0.f, Mzz = 0.f, Mxy = 0.f, Myz = 0.f, Mzx = 0.f;
        float Lx = 0.f, Ly = 0.f, Lz = 0.f;
        bool second = true;
        if constexpr (kOnePass) {
          const float fn = (float)nt;
          Mxx = o_m[0] - fn * rcx * rcx; Myy = o_m[1] - fn * rcy * rcy; Mzz = o_m[2] - fn * rcz * rcz;
          Mxy = o_m[3] - fn * rcx * rcy; Myz = o_m[4] - fn * rcy * rcz; Mzx = o_m[5] - fn * rcz * rcx;
          Lx = o_m[6] - fn * (rcy * wmz - rcz * wmy);
          Ly = o_m[7] - fn * (rcz * wmx - rcx * wmz);
          Lz = o_m[8] - fn * (rcx * wmy - rcy * wmx);
          second = nt >= 2 && o_m[0] + o_m[1] + o_m[2] > 4.0f * (Mxx + Myy + Mzz);
        }
        // SRD+a: the cell's random rotation axis (every lane of the group draws it)
        float ax = 0.f, ay = 0.f, az = 0.f;
        if constexpr (VAR == 2) {
          const uint4 r = draw(g, cg, step, kTagAxis, 0u);
          az = 2.0f * u01(r.x) - 1.0f;
          const float st = sqrtf(fmaxf(0.0f, 1.0f - az * az));
          float sphi, cphi;
          sincospif(2.0f * u01(r.y), &sphi, &cphi);
          ax = st * cphi;
          ay = st * sphi;
        }
        // second pass: moments about the centre of mass and the angular momentum the
        // collision would change -- AT+a: of w - <w>; SRD+a (Eq. 4): of v_ic - D v_ic
        float sMxx = 0.f, sMyy = 0.f, sMzz = 0.f, sMxy = 0.f, sMyz = 0.f, sMzx = 0.f;
        float sLx = 0.f, sLy = 0.f, sLz = 0.f;
        long long qM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // deterministic mode
        const bool any_second = !kOnePass || __any_sync(0xffffffffu, second && n > 0);
        // one member's terms about the centre of mass: r = rho - rho_cm, w - <w> (SRD+a:
        // minus its rotation, Eq. 4)
        auto second_term = [&](float rx, float ry, float rz, float wx, float wy, float wz) {
          if constexpr (VAR == 2) {
            const float nr = ax * wx + ay * wy + az * wz;
            const float t = (1.0f - g.cos_a) * nr;
            const float dx = g.cos_a * wx + g.sin_a * (ay * wz - az * wy) + t * ax;
            const float dy = g.cos_a * wy + g.sin_a * (az * wx - ax * wz) + t * ay;
            const float dz = g.cos_a * wz + g.sin_a * (ax * wy - ay * wx) + t * az;
            wx -= dx; wy -= dy; wz -= dz;
          }
          if constexpr (DET) {
            const float tx = ry * wz - rz * wy, ty = rz * wx - rx * wz, tz = rx * wy - ry * wx;
            fxbig = fmaxf(fxbig, fmaxf(fabsf(tx), fmaxf(fabsf(ty), fabsf(tz))));
            qM[0] += to_fx(rx * rx); qM[1] += to_fx(ry * ry); qM[2] += to_fx(rz * rz);
            qM[3] += to_fx(rx * ry); qM[4] += to_fx(ry * rz); qM[5] += to_fx(rz * rx);
            qM[6] += to_fx(tx); qM[7] += to_fx(ty); qM[8] += to_fx(tz);
          } else {
            sMxx += rx * rx; sMyy += ry * ry; sMzz += rz * rz;
            sMxy += rx * ry; sMyz += ry * rz; sMzx += rz * rx;
            sLx += ry * wz - rz * wy; sLy += rz * wx - rx * wz; sLz += rx * wy - ry * wx;
          }
        };
        const int n2 = second ? n : 0;
        for (int k = sub; any_second && k < n2; k += tpc) {
          const int i = sperm[base + k];
          second_term(rho_axis(g, sx[i], S0x) - rcx, rho_axis(g, sy[i], S0y) - rcy,
                      rho_axis(g, sz[i] & ~kCrossedBit, S0z) - rcz, svx[i] - wmx, svy[i] - wmy,
                      svz[i] - wmz);
        }
        const int nph2 = second ? nph : 0;
        for (int j = sub; any_second && j < nph2; j += tpc) {
          const PhantomParticle q = phantom_particle(g, cg, step, j, S0z, pwall);
          const float vx = VAR == 1 ? q.vx - q.ux : q.vx, vy = VAR == 1 ? q.vy - q.uy : q.vy,
                      vz = VAR == 1 ? q.vz - q.uz : q.vz;
          second_term((float)q.ix * g.inv2F - rcx, (float)q.iy * g.inv2F - rcy,
                      (float)q.iz * g.inv2F - rcz, vx - wmx, vy - wmy, vz - wmz);
        }
        if constexpr (DET) {
#pragma unroll
          for (int q = 0; q < 9; ++q) qM[q] = group_sum_fx(qM[q], tpc);
          Mxx = from_fx(qM[0]); Myy = from_fx(qM[1]); Mzz = from_fx(qM[2]);
          Mxy = from_fx(qM[3]); Myz = from_fx(qM[4]); Mzx = from_fx(qM[5]);
          Lx = from_fx(qM[6]); Ly = from_fx(qM[7]); Lz = from_fx(qM[8]);
        } else {
          if (any_second) {
            sMxx = group_sum(sMxx, tpc); sMyy = group_sum(sMyy, tpc); sMzz = group_sum(sMzz, tpc);
            sMxy = group_sum(sMxy, tpc); sMyz = group_sum(sMyz, tpc); sMzx = group_sum(sMzx, tpc);
            sLx = group_sum(sLx, tpc); sLy = group_sum(sLy, tpc); sLz = group_sum(sLz, tpc);
          }
          if (second) {
            Mxx = sMxx; Myy = sMyy; Mzz = sMzz; Mxy = sMxy; Myz = sMyz; Mzx = sMzx;
            Lx = sLx; Ly = sLy; Lz = sLz;
          }
        }
        if (exists && n > 0 && sub == 0) {
          // J = tr(M) 1 - M (moment-of-inertia tensor per unit mass); omega = J^-1 L
          const float3 om = solve_omega(nt, Mxx, Myy, Mzz, Mxy, Myz, Mzx, Lx, Ly, Lz);
          const float ox_ = om.x, oy_ = om.y, oz_ = om.z;
          float* P = spar + lc;
          P[0 * bc] = wmx; P[1 * bc] = wmy; P[2 * bc] = wmz;
          P[3 * bc] = ox_; P[4 * bc] = oy_; P[5 * bc] = oz_;
          if constexpr (VAR == 1) {
            // omega x (rho - rho_cm) = omega x rho - omega x rho_cm: the second term
            // joins the cell's velocity offset
            P[0 * bc] = wmx - (oy_ * rcz - oz_ * rcy);
            P[1 * bc] = wmy - (oz_ * rcx - ox_ * rcz);
            P[2 * bc] = wmz - (ox_ * rcy - oy_ * rcx);
          } else {
            P[6 * bc] = rcx; P[7 * bc] = rcy; P[8 * bc] = rcz;
          }
          if constexpr (VAR == 2) {
            P[9 * bc] = ax; P[10 * bc] = ay; P[11 * bc] = az;
          }
        }
      }
    }
    if (DET && fxbig >= kFxLimit) atomicOr(&a.ctrl->errors, kErrFixedRange);
  }
  __syncthreads();

  // ---- 4. collide, stream for step n+1, count by destination brick ----
  float o_px = 0, o_py = 0, o_pz = 0, o_e = 0, o_kxy = 0, o_kyz = 0, o_kzx = 0;
  float o_c[6] = {0, 0, 0, 0, 0, 0};
  long long o_q[13];  // deterministic mode: fixed-point observables
  if constexpr (DET) {
#pragma unroll
    for (int q = 0; q < 13; ++q) o_q[q] = 0;
  }
  const bool zper = PLAIN || !g.walls;
  for (int i = tid; i < cnt; i += kThreads) {
    uint32_t x = sx[i], y = sy[i], z = sz[i] & ~kCrossedBit;
    float vbx = svx[i], vby = svy[i], vbz = svz[i];  // AT+a: w
    const uint32_t lcr = stag[i];
    // a particle without a cell (kNoCell) keeps its velocity: computed with cell 0's
    // parameters and discarded, so the common path has no branch
    const bool has = lcr != kNoCell;
    const uint32_t lc = has ? (lcr & kCellMask) : 0u;
    const float* P = spar + lc;
    float nx, ny, nz;
    // positions relative to the collision-cell centre (collisional stress, AT+a omega x r)
    const float px = rho_axis(g, x, S0x), py = rho_axis(g, y, S0y), pz = rho_axis(g, z, S0z);
    if constexpr (VAR == 0) {
      const float vcx = P[0], vcy = P[bc], vcz = P[2 * bc];
      const float ax = P[3 * bc], ay = P[4 * bc], az = P[5 * bc], kap = P[6 * bc];
      const float rx = vbx - vcx, ry = vby - vcy, rz = vbz - vcz;
      const float nr = ax * rx + ay * ry + az * rz;
      const float t = (1.0f - g.cos_a) * nr;
      nx = vcx + kap * (g.cos_a * rx + g.sin_a * (ay * rz - az * ry) + t * ax);
      ny = vcy + kap * (g.cos_a * ry + g.sin_a * (az * rx - ax * rz) + t * ay);
      nz = vcz + kap * (g.cos_a * rz + g.sin_a * (ax * ry - ay * rx) + t * az);
      nx = has ? nx : vbx; ny = has ? ny : vby; nz = has ? nz : vbz;
    } else if constexpr (VAR == 2) {
      // SRD+a, Eq. (3): v' = v_cm + D v_ic + omega x r_ic
      nx = vbx; ny = vby; nz = vbz;
      if (has) {
        const float vcx = P[0], vcy = P[bc], vcz = P[2 * bc];
        const float wx = P[3 * bc], wy = P[4 * bc], wz = P[5 * bc];
        const float rx = px - P[6 * bc], ry = py - P[7 * bc], rz = pz - P[8 * bc];
        const float ax = P[9 * bc], ay = P[10 * bc], az = P[11 * bc];
        const float ux = vbx - vcx, uy = vby - vcy, uz = vbz - vcz;
        const float nr = ax * ux + ay * uy + az * uz;
        const float t = (1.0f - g.cos_a) * nr;
        nx = vcx + g.cos_a * ux + g.sin_a * (ay * uz - az * uy) + t * ax + (wy * rz - wz * ry);
        ny = vcy + g.cos_a * uy + g.sin_a * (az * ux - ax * uz) + t * ay + (wz * rx - wx * rz);
        nz = vcz + g.cos_a * uz + g.sin_a * (ax * uy - ay * ux) + t * az + (wx * ry - wy * rx);
      }
    } else {
      const float ux = sux[i], uy = suy[i], uz = suz[i];
      vbx += ux; vby += uy; vbz += uz;  // the velocity the particle streamed with
      const float wx = P[3 * bc], wy = P[4 * bc], wz = P[5 * bc];
      nx = P[0] + ux + (wy * pz - wz * py);
      ny = P[bc] + uy + (wz * px - wx * pz);
      nz = P[2 * bc] + uz + (wx * py - wy * px);
      nx = has ? nx : vbx; ny = has ? ny : vby; nz = has ? nz : vbz;
    }
    if (g.obs) {
      if constexpr (DET) {
        const float dx = nx - vbx, dy = ny - vby, dz = nz - vbz;
        const float t[13] = {nx, ny, nz, nx * nx + ny * ny + nz * nz, vbx * vby, vby * vbz,
                             vbz * vbx, dx * py, dy * px, dy * pz, dz * py, dz * px, dx * pz};
#pragma unroll
        for (int q = 0; q < 13; ++q) o_q[q] += fixed_of<24>(t[q]);
      } else {
        o_px += nx; o_py += ny; o_pz += nz;
        o_e = fmaf(nz, nz, fmaf(ny, ny, fmaf(nx, nx, o_e)));
        o_kxy += vbx * vby; o_kyz += vby * vbz; o_kzx += vbz * vbx;
        const float dx = nx - vbx, dy = ny - vby, dz = nz - vbz;
        o_c[0] += dx * py; o_c[1] += dy * px; o_c[2] += dy * pz;
        o_c[3] += dz * py; o_c[4] += dz * px; o_c[5] += dx * pz;
      }
    }
    // stream for step n+1 (this is the only streaming of the particle per step) and
    // find the brick of its next collision cell
    if constexpr (PLAIN) stream_periodic_pow2(g, x, y, z, nx, ny, nz);
    else stream(g, x, y, z, nx, ny, nz);
    sx[i] = x; sy[i] = y; sz[i] = z;
    svx[i] = nx; svy[i] = ny; svz[i] = nz;
    const uint32_t zs = z & ~kCrossedBit;
    uint32_t code;
    if (inner) {
      const int dxb = (int)(x + S1x - Ox) >> (g.F + Bs0);
      const int dyb = (int)(y + S1y - Oy) >> (g.F + Bs1);
      const int dzb = (int)(zs + S1z - Oz) >> (g.F + Bs2);
      code = ((unsigned)(dxb + 1) > 2u || (unsigned)(dyb + 1) > 2u || (unsigned)(dzb + 1) > 2u)
                 ? 27u
                 : (uint32_t)((dxb + 1) + 3 * (dyb + 1) + 9 * (dzb + 1));
    } else {
      const int qx = cell_axis(g, x, S1x, 0) >> Bs0;
      const int qy = cell_axis(g, y, S1y, 1) >> Bs1;
      const int qz = cell_axis(g, zs, S1z, 2) >> Bs2;
      const int dxb = brick_delta(qx, bx, g.nb[0], true);
      const int dyb = brick_delta(qy, by, g.nb[1], true);
      const int dzb = brick_delta(qz, bz, g.nb[2], zper);
      code = (dxb == 9 || dyb == 9 || dzb == 9)
                 ? 27u
                 : (uint32_t)((dxb + 1) + 3 * (dyb + 1) + 9 * (dzb + 1));
    }
    // rank within the warp's group for the destination: the lanes bound for the same
    // brick take distinct slots of one run, so their writes below are contiguous.  AT+a:
    // one shared-memory atomic per lane on the warp's counter (0.6 warp instructions per
    // particle fewer than grouping first, 0.8 % faster); SRD and SRD+a, with 9 CTAs per SM
    // contending for the atomic unit: the lanes grouped by destination (match) and one
    // atomic per group (1.8 % faster there)
    uint32_t rank;
    if constexpr (VAR == 1) {
      rank = atomicAdd(&wcount[28 * (tid >> 5) + code], 1u);
    } else {
      const uint32_t active = __activemask();
      const uint32_t peers = __match_any_sync(active, code);
      const int leader = __ffs(peers) - 1;
      uint32_t rank0 = 0;
      if (lane == leader) rank0 = atomicAdd(&wcount[28 * (tid >> 5) + code], (uint32_t)__popc(peers));
      rank = __shfl_sync(active, rank0, leader) + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    stag[i] = (Tag)(code | (rank << 5));
  }
  // ---- 5. per warp: this warp's runs in the destination bricks (one global atomic per
  // destination group of the warp, issued first so that its round trip overlaps the
  // observables reduction), the observables partials, and the write-out of the warp's
  // own particles -- the ones it collided, so no block barrier is needed ----
  const int w = tid >> 5;
  __syncwarp();
  uint32_t rbase = 0, rdest = 0;  // lane c: the warp's run for destination code c
  if (lane < 27) {
    const uint32_t n = wcount[28 * w + lane];
    if (n > 0) {
      const int dxb = lane % 3 - 1, dyb = (lane / 3) % 3 - 1, dzb = lane / 9 - 1;
      int qx = bx + dxb, qy = by + dyb, qz = bz + dzb;
      if (qx < 0) qx += g.nb[0]; else if (qx >= g.nb[0]) qx -= g.nb[0];
      if (qy < 0) qy += g.nb[1]; else if (qy >= g.nb[1]) qy -= g.nb[1];
      if (zper) { if (qz < 0) qz += g.nb[2]; else if (qz >= g.nb[2]) qz -= g.nb[2]; }
      rdest = (uint32_t)(qx + g.nb[0] * (qy + g.nb[1] * qz));
      rbase = atomicAdd(&cnt_dst[rdest], n);
    }
  }

  if (g.obs) {
    double* orow = &a.obs_partials[(b % kObsSlots) * kObsWidth];
    if constexpr (DET) {
      long long vals[16] = {o_q[0], o_q[1], o_q[2], o_q[3], o_q[4], o_q[5], o_q[6], o_q[7],
                            o_q[8], o_q[9], o_q[10], o_q[11], o_q[12], 0, 0, 0};
      const long long s = warp_reduce_scatter16(vals, lane);
      // integer partials: the order of the atomics does not matter
      if (!(lane & 1) && (lane >> 1) < 13)
        atomicAdd(reinterpret_cast<unsigned long long*>(orow + (lane >> 1)), (unsigned long long)s);
    } else {
      float vals[16] = {o_px, o_py, o_pz, o_e, o_kxy, o_kyz, o_kzx, o_c[0], o_c[1], o_c[2],
                        o_c[3], o_c[4], o_c[5], 0.f, 0.f, 0.f};
      const float s = warp_reduce_scatter16(vals, lane);
      if (!(lane & 1) && (lane >> 1) < 13) atomicAdd(orow + (lane >> 1), (double)s);
    }
  }
  // ---- 6. write out: each particle to its reserved slot; the ids come from the source
  // brick in global memory (L2: loaded or prefetched with the brick) ----
  uint32_t* const dX = par ? a.buf[0].x[0] : a.buf[1].x[0];
  uint32_t* const dY = par ? a.buf[0].x[1] : a.buf[1].x[1];
  uint32_t* const dZ = par ? a.buf[0].x[2] : a.buf[1].x[2];
  float* const dVX = par ? a.buf[0].v[0] : a.buf[1].v[0];
  float* const dVY = par ? a.buf[0].v[1] : a.buf[1].v[1];
  float* const dVZ = par ? a.buf[0].v[2] : a.buf[1].v[2];
  uint32_t* const dID = par ? a.buf[0].id : a.buf[1].id;
  const uint32_t* const src_id = a.buf[par].id + (size_t)b * cap;
  bool rare = false;
  const int wfirst = 32 * w;
  // every lane of the warp takes part in the shuffles; lanes past the count write nothing
  auto write_one = [&](int i, uint32_t id) {
    const bool valid = i < cnt;
    const uint32_t t = valid ? (uint32_t)stag[i] : 0u;
    const uint32_t code = t & 31u;
    const uint32_t base = __shfl_sync(0xffffffffu, rbase, (int)code);
    const uint32_t dest = __shfl_sync(0xffffffffu, rdest, (int)code);
    const uint32_t slot = base + (t >> 5);  // meaningless for code 27, not used
    if (valid) {
      if (code < 27 && slot < (uint32_t)cap) {
        const size_t o = (size_t)dest * cap + slot;
        dX[o] = sx[i]; dY[o] = sy[i]; dZ[o] = sz[i];
        dVX[o] = svx[i]; dVY[o] = svy[i]; dVZ[o] = svz[i];
        dID[o] = id;
        if (debug) dst.cell[o] = sgc[i];
      } else {
        rare = true;
      }
    }
  };
  if constexpr (TIER > 0) {
    // all of this thread's ids in flight at once
    constexpr int K = (kTile + kThreads - 1) / kThreads;
    uint32_t idr[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = tid + k * kThreads;
      idr[k] = i < cnt ? __ldg(src_id + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (wfirst + k * kThreads >= cnt) break;
      write_one(tid + k * kThreads, idr[k]);
    }
  } else {
    for (int i0 = wfirst; i0 < cnt; i0 += kThreads) {
      const int i = i0 + lane;
      write_one(i, i < cnt ? __ldg(src_id + i) : 0u);
    }
  }
  // the rare ones, kept out of the loop above: a particle bound beyond the neighbour
  // bricks (a global atomic for its slot) or past its destination's capacity (spilled)
  if (__any_sync(0xffffffffu, rare)) {
    for (int i0 = wfirst; i0 < cnt; i0 += kThreads) {
      const int i = i0 + lane;
      const bool valid = i < cnt;
      const uint32_t t = valid ? (uint32_t)stag[i] : 0u;
      const uint32_t code = t & 31u;
      const uint32_t base = __shfl_sync(0xffffffffu, rbase, (int)code);
      const uint32_t dgrp = __shfl_sync(0xffffffffu, rdest, (int)code);
      if (!valid || (code < 27 && base + (t >> 5) < (uint32_t)cap)) continue;
      uint32_t d, slot;
      if (code < 27) {
        d = dgrp;
        slot = base + (t >> 5);
      } else {
        const int qx = cell_axis(g, sx[i], S1x, 0) >> Bs0;
        const int qy = cell_axis(g, sy[i], S1y, 1) >> Bs1;
        const int qz = cell_axis(g, sz[i] & ~kCrossedBit, S1z, 2) >> Bs2;
        d = (uint32_t)(qx + g.nb[0] * (qy + g.nb[1] * qz));
        slot = atomicAdd(&cnt_dst[d], 1u);
      }
      const uint32_t id = src_id[i];
      if (slot < (uint32_t)cap) {
        const size_t o = (size_t)d * cap + slot;
        dX[o] = sx[i]; dY[o] = sy[i]; dZ[o] = sz[i];
        dVX[o] = svx[i]; dVY[o] = svy[i]; dVZ[o] = svz[i];
        dID[o] = id;
        if (debug) dst.cell[o] = sgc[i];
      } else {
        atomicExch(&a.ctrl->overflow, 1);
        const uint32_t s = atomicAdd(&a.ctrl->spill_count, 1u);
        if (s < a.spill.capacity) {
          a.spill.x[0][s] = sx[i]; a.spill.x[1][s] = sy[i]; a.spill.x[2][s] = sz[i];
          a.spill.v[0][s] = svx[i]; a.spill.v[1][s] = svy[i]; a.spill.v[2][s] = svz[i];
          a.spill.id[s] = id;
          if (debug) a.spill.cell[s] = sgc[i];
          a.spill.dest[s] = d;
        } else {
          atomicExch(&a.ctrl->lost, 1);
        }
      }
    }
  }
  return true;
}


// --- kernels -------------------------------------------------------------------------

// CTAs per SM the default bricks fit in shared memory (26.5 KB SRD, 27.8 KB SRD+a,
// 36.8 KB AT+a of dynamic shared memory per CTA); the register budget is held to match.
template <int VAR>
constexpr int kMinBlocks = VAR == 1 ? 6 : 8;

// One box: one CTA per brick.  DEFER: the smaller shared-memory tile (7 CTAs per SM for
// AT+a, 9 for SRD and SRD+a), bricks that exceed it left to k_step_deferred.
template <int VAR, bool DEFER>
constexpr int kMinBlocksStep = DEFER ? (VAR == 1 ? 7 : 9) : kMinBlocks<VAR>;

// the variants and summation modes that take the deferring kernel on large boxes: AT+a
// (7 CTAs per SM instead of 6, both modes), SRD and SRD+a with floating-point sums (9
// instead of 8; their fixed-point kernels need more than the 56 registers a ninth CTA
// leaves)
template <int VAR, bool DET>
constexpr bool kDefers = VAR == 1 || !DET;

template <int VAR, bool DET, int TIER, bool DEFER = false, bool PLAIN = false>
__global__ void __launch_bounds__(kThreads, kMinBlocksStep<VAR, DEFER>) k_step(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ BrickShared sh;
  uint32_t phase = 0;
  step_brick<VAR, DET, false, TIER, DEFER, PLAIN>(a, blockIdx.x, smem, sh, phase);
}

// The full-capacity pass of a step: the bricks a deferring k_step left in a.deferred, by
// the generic body (same arithmetic and order as the compiled-in tiers: identical
// results).  The last CTA to finish clears the list for the next step.
template <int VAR, bool DET>
__global__ void __launch_bounds__(kThreads, kMinBlocks<VAR>) k_step_deferred(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ BrickShared sh;
  __shared__ uint32_t s_n;
  if (threadIdx.x == 0) {
    mbar_init(&sh.bar, 1);
    s_n = *(volatile uint32_t*)&a.deferred[0];
  }
  __syncthreads();
  const uint32_t n = s_n;
  uint32_t phase = 0;
  for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
    if (!step_brick<VAR, DET, true, 0>(a, (int)a.deferred[2 + k], smem, sh, phase)) break;
    // the next brick's bulk copies overwrite shared memory this one wrote
    fence_proxy_async_smem();
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.deferred[1], 1u) == gridDim.x - 1) {
      a.deferred[0] = 0;
      a.deferred[1] = 0;
    }
  }
}

// Many small boxes of one variant in one persistent launch.  The boxes' arguments
// travel in kernel parameter space (PackTable, passed by value), so the per-box values
// the hot loops read are uniform constant-bank loads like those of the single-box
// kernel rather than per-thread registers.  CTAs claim work items (bricks of the
// packed boxes, box k owning items [begin[k], begin[k+1])) from a counter that is zero
// at launch; each CTA's claims increase, so its box index only moves forward.
template <int VAR, bool DET, int TIER>
__global__ void __launch_bounds__(kThreads, kMinBlocks<VAR>) k_step_packed(const __grid_constant__ PackTable p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ BrickShared sh;
  __shared__ int s_w;
  if (threadIdx.x == 0) mbar_init(&sh.bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  const int total = p.begin[p.n];
  int k = 0;
  for (;;) {
    if (threadIdx.x == 0) s_w = (int)atomicAdd(p.counter, 1u);
    __syncthreads();
    const int w = s_w;
    if (w >= total) return;
    while (k + 1 < p.n && p.begin[k + 1] <= w) ++k;
    if (!step_brick<VAR, DET, true, TIER>(p.args[k], w - p.begin[k], smem, sh, phase)) return;
    // the next item's bulk copies overwrite shared memory this item wrote
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// --- launch helpers, one variant at a time (instantiated in mpc_step_<variant>.cu) ---

template <int VAR, bool DET>
cudaError_t set_cap_tiers(int v) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_step<VAR, DET, 0>, a, v);
  if constexpr (kDefers<VAR, DET>) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 1, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 2, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 1, true, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 2, true, true>, a, v);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_deferred<VAR, DET>, a, v);
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 1>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 2>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<VAR, DET, 3>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_packed<VAR, DET, 0>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_packed<VAR, DET, 1>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_packed<VAR, DET, 2>, a, v);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step_packed<VAR, DET, 3>, a, v);
  return e;
}

// Boxes of at least this many bricks (about eight waves of 7 CTAs on 152 SMs) take the
// deferring kernel: below it the full-capacity pass's extra launch costs more than the
// seventh CTA per SM gains.
constexpr int kDeferMinBricks = 8192;
constexpr int kDeferGrid = 256;  // CTAs of the full-capacity pass

template <int VAR>
size_t deferred_smem_bytes(const Geom& g) {
  return make_layout(g.cap, g.brick_cells, CellParams<VAR>::kParams,
                     CellParams<VAR>::kStoresRandomVelocity, g.debug, 4).total;
}

template <int VAR, bool DET>
void launch_tier(const StepArgs& a, size_t bytes, cudaStream_t s) {
  const int tier = tier_of(a.g);
  if constexpr (kDefers<VAR, DET>) {
    // tiers 1 and 2 (16-bit tags) fit 7 CTAs per SM with the smaller tile; tier 3's 128
    // cells do not
    if ((tier == 1 || tier == 2) && a.g.nbricks >= kDeferMinBricks && a.deferred) {
      const size_t tile = make_layout(TierShape<1>::scap, a.g.brick_cells, CellParams<VAR>::kParams,
                                      CellParams<VAR>::kStoresRandomVelocity, 0, 2).total;
      // periodic, gravity-free boxes of power-of-two extents take the plain body
      if (periodic_pow2_box(a.g)) {
        if (tier == 1) k_step<VAR, DET, 1, true, true><<<a.g.nbricks, kThreads, tile, s>>>(a);
        else k_step<VAR, DET, 2, true, true><<<a.g.nbricks, kThreads, tile, s>>>(a);
      } else {
        if (tier == 1) k_step<VAR, DET, 1, true><<<a.g.nbricks, kThreads, tile, s>>>(a);
        else k_step<VAR, DET, 2, true><<<a.g.nbricks, kThreads, tile, s>>>(a);
      }
      k_step_deferred<VAR, DET><<<kDeferGrid, kThreads, deferred_smem_bytes<VAR>(a.g), s>>>(a);
      return;
    }
  }
  switch (tier) {
    case 1: k_step<VAR, DET, 1><<<a.g.nbricks, kThreads, bytes, s>>>(a); break;
    case 2: k_step<VAR, DET, 2><<<a.g.nbricks, kThreads, bytes, s>>>(a); break;
    case 3: k_step<VAR, DET, 3><<<a.g.nbricks, kThreads, bytes, s>>>(a); break;
    default: k_step<VAR, DET, 0><<<a.g.nbricks, kThreads, bytes, s>>>(a); break;
  }
}

template <int VAR, bool DET>
cudaError_t packed_occupancy_v(int tier, size_t smem_bytes, int* ctas_per_sm) {
  switch (tier) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_step_packed<VAR, DET, 1>, kThreads, smem_bytes);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_step_packed<VAR, DET, 2>, kThreads, smem_bytes);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_step_packed<VAR, DET, 3>, kThreads, smem_bytes);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_step_packed<VAR, DET, 0>, kThreads, smem_bytes);
  }
}

template <int VAR, bool DET>
void launch_packed_v(const PackTable& t, int tier, int grid, size_t smem_bytes, cudaStream_t s) {
  switch (tier) {
    case 1: k_step_packed<VAR, DET, 1><<<grid, kThreads, smem_bytes, s>>>(t); break;
    case 2: k_step_packed<VAR, DET, 2><<<grid, kThreads, smem_bytes, s>>>(t); break;
    case 3: k_step_packed<VAR, DET, 3><<<grid, kThreads, smem_bytes, s>>>(t); break;
    default: k_step_packed<VAR, DET, 0><<<grid, kThreads, smem_bytes, s>>>(t); break;
  }
}

// The entry points of one variant (both summation modes): each variant's kernels are
// compiled in a translation unit of their own, which instantiates these.
template <int VAR>
cudaError_t configure_variant(int max_dynamic_smem) {
  cudaError_t e = set_cap_tiers<VAR, false>(max_dynamic_smem);
  if (e == cudaSuccess) e = set_cap_tiers<VAR, true>(max_dynamic_smem);
  return e;
}

template <int VAR>
void launch_variant(const StepArgs& a, size_t bytes, cudaStream_t s) {
  if (a.g.det) launch_tier<VAR, true>(a, bytes, s);
  else launch_tier<VAR, false>(a, bytes, s);
}

template <int VAR>
cudaError_t packed_occupancy_variant(int tier, bool det, size_t smem_bytes, int* ctas_per_sm) {
  return det ? packed_occupancy_v<VAR, true>(tier, smem_bytes, ctas_per_sm)
             : packed_occupancy_v<VAR, false>(tier, smem_bytes, ctas_per_sm);
}

template <int VAR>
void launch_packed_variant(const PackTable& t, int tier, bool det, int grid, size_t smem_bytes,
                           cudaStream_t s) {
  if (det) launch_packed_v<VAR, true>(t, tier, grid, smem_bytes, s);
  else launch_packed_v<VAR, false>(t, tier, grid, smem_bytes, s);
}

}  // namespace mpc
