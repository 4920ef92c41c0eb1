// Device building blocks of the MPC step: counter-based random numbers, samplers,
// the fixed-point streaming contract and the shifted-lattice cell assignment.
//
// Everything here follows the written state contract of include/mpc.h; the float32
// expressions whose result decides an integer (the gamma sampler's accept/reject, the
// displacement rounding) use explicitly rounded intrinsics so the compiler cannot
// contract them into FMAs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mpc_internal.h"

namespace mpc {

// Philox counter word 2 = (tag << 24) | sub-draw index.  Tag values are part of the
// keying contract.
enum : uint32_t {
  kTagShift = 1, kTagAxis = 2, kTagMbs = 3, kTagPhantom = 4, kTagPhGamma = 5,
  kTagAtVel = 6, kTagInitX = 7, kTagInitV = 8, kTagPhPart = 9
};

// Philox4x32-10 (Salmon et al., SC'11): per round, the two multiplier words give
// 64-bit products whose high halves are mixed into the other pair of words with the
// round key; the key advances by the Weyl increments after every round.  The ten round
// keys depend on the seed alone, so the host computes them once (round_keys) and every
// round xors a kernel-parameter word instead of adding the increments per draw.
__device__ __forceinline__ uint4 philox4x32(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const uint32_t (&rk)[20]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
    c0 = hi_b ^ c1 ^ rk[2 * r];
    c1 = lo_b;
    c2 = hi_a ^ c3 ^ rk[2 * r + 1];
    c3 = lo_a;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 draw(const Geom& g, uint32_t index, uint32_t step, uint32_t tag,
                                      uint32_t sub) {
  return philox4x32(index, step, (tag << 24) | sub, g.box, g.rk);
}

// (k + 1/2) 2^-23 from the top 23 bits: k 2^-23 + 2^-24 in one fused operation, exact in
// float32 (k < 2^23)
__device__ __forceinline__ float u01(uint32_t r) {
  return __fmaf_rn((float)(r >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
}

// 2 u01(r) - 1 = (k + 1/2) 2^-22 - 1, exact in float32
__device__ __forceinline__ float u11(uint32_t r) {
  return __fmaf_rn((float)(r >> 9), 2.384185791015625e-7f, -0.99999988079071044921875f);
}

// The hardware approximations (PTX *.approx.ftz): every argument they get here is a
// normal float32, where they agree with the non-ftz forms without those forms' subnormal
// handling
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_approx(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_approx(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Box-Muller pair of standard normals
__device__ __forceinline__ float2 normal2(uint32_t ra, uint32_t rb) {
  const float R = sqrtf(-2.0f * logf(u01(ra)));
  float s, c;
  sincospif(2.0f * u01(rb), &s, &c);
  return make_float2(R * c, R * s);
}

// -2 ln u for u = (k + 1/2) 2^-23 in (0, 1).  With t = 1 - u (exact): for t >= 2^-7 the
// hardware log2 (absolute error below 2^-22 on [0.5, 2), 2 ulp below 0.5), else the
// series 2 (t + t^2/2 + t^3/3), whose truncation is below t^3/4 relative.  Absolute error
// below 3.4e-7 + 2.5e-7 |result|.
__device__ __forceinline__ float minus_2_log_u01(float u) {
  const float t = 1.0f - u;
  const float series = 2.0f * t * (1.0f + t * (0.5f + t * (1.0f / 3.0f)));
  const float hw = -1.3862943611198906f * lg2_approx(u);  // -2 ln 2 log2(u)
  return t < 0.0078125f ? series : hw;
}

// The three AT+a random-velocity normals from one Philox draw, times sigma: the
// Box-Muller pair of (r.x, r.y) and the cosine normal of (r.z, r.w).  The radius is
// sqrt(-2 ln u) as y rsqrt(y) (y > 0: u < 1), scaled by sigma once, the angle -cos / -sin
// of pi (2u - 1) in [-pi, pi) by the hardware approximations (absolute error below
// 6e-7).  A normal is off by less than 6e-6 in the worst case (radius 5.8, u = 2^-24)
// and ~1e-6 typically.  These values decide no integer.
__device__ __forceinline__ float3 normal3_at(uint4 r, float sigma) {
  constexpr float kPi = 3.14159265358979f;
  const float y0 = minus_2_log_u01(u01(r.x)), y1 = minus_2_log_u01(u01(r.z));
  const float R0 = sigma * (y0 * rsqrt_approx(y0)), R1 = sigma * (y1 * rsqrt_approx(y1));
  const float a0 = kPi * u11(r.y);
  const float c = cos_approx(a0), s = sin_approx(a0);
  const float c1 = cos_approx(kPi * u11(r.w));
  return make_float3(-R0 * c, -R0 * s, -R1 * c1);
}

// Gamma(shape a >= 1, scale 1), Marsaglia & Tsang (ACM TOMS 26, 2000); attempt k uses
// Philox(index, step, tag, k).  Float32 decisions in a fixed evaluation order.
__device__ __forceinline__ float gamma_mt(const Geom& g, uint32_t index, uint32_t step, uint32_t tag,
                                          float a) {
  const float d = __fsub_rn(a, 1.0f / 3.0f);
  const float c = __fdiv_rn(1.0f, __fsqrt_rn(__fmul_rn(9.0f, d)));
  for (uint32_t k = 0; k < 32; ++k) {
    const uint4 r = draw(g, index, step, tag, k);
    const float x = normal2(r.x, r.y).x;
    const float u = u01(r.z);
    const float v1 = __fmaf_rn(c, x, 1.0f);
    if (v1 <= 0.0f) continue;
    const float v3 = __fmul_rn(__fmul_rn(v1, v1), v1);
    const float x2 = __fmul_rn(x, x);
    const float x4 = __fmul_rn(x2, x2);
    const float squeeze = __fsub_rn(1.0f, __fmul_rn(0.0331f, x4));
    if (u < squeeze) return d * v3;
    const float rhs =
        __fadd_rn(__fmul_rn(0.5f, x2), __fmul_rn(d, __fadd_rn(__fsub_rn(1.0f, v3), logf(v3))));
    if (logf(u) < rhs) return d * v3;
  }
  return d;
}

// Poisson(lambda) by sequential CDF inversion in float64 (wall cells only)
__device__ __forceinline__ int poisson_inv(double u, double lambda) {
  int k = 0;
  double prob = exp(-lambda);
  double cdf = prob;
  while (u > cdf && k < 100000) {
    ++k;
    prob *= lambda / (double)k;
    cdf += prob;
  }
  return k;
}

// Phantom particle j of the wall-cut collision cell cg (the angular-momentum-conserving
// variants at no-slip walls, Sec. II "Boundary conditions"; the oracle draws the same
// particles from the same counters): its position relative to the cell centre on the
// fixed-point grid (integers, units 2^-F) -- x and y uniform over the cell, z uniform over
// the part beyond the wall (local coordinate below the shift Sz at the bottom wall, from Sz
// up at the top) --, its velocity u_wall x + sigma (n0, n1, n2) and random velocity
// sigma (n3, n4, n5), from Philox(cg, step, kTagPhPart, 3j + q), q = 0, 1, 2.
struct PhantomParticle {
  int ix, iy, iz;
  float vx, vy, vz, ux, uy, uz;
};

__device__ __forceinline__ PhantomParticle phantom_particle(const Geom& g, uint32_t cg, uint32_t step,
                                                            int j, uint32_t Sz, int wall) {
  const uint4 a = draw(g, cg, step, kTagPhPart, 3u * (uint32_t)j);
  const uint4 b = draw(g, cg, step, kTagPhPart, 3u * (uint32_t)j + 1u);
  const uint4 c = draw(g, cg, step, kTagPhPart, 3u * (uint32_t)j + 2u);
  const uint32_t one = 1u << g.F, half = one >> 1;
  const uint32_t ix = a.x >> (32 - g.F), iy = a.y >> (32 - g.F);
  const uint32_t iz = wall == 0 ? (uint32_t)(((uint64_t)a.z * Sz) >> 32)
                                : Sz + (uint32_t)(((uint64_t)a.z * (uint64_t)(one - Sz)) >> 32);
  const float2 n01 = normal2(b.x, b.y), n23 = normal2(b.z, b.w), n45 = normal2(c.x, c.y);
  PhantomParticle q;
  q.ix = (int)ix - (int)half;
  q.iy = (int)iy - (int)half;
  q.iz = (int)iz - (int)half;
  q.vx = g.wall_u[wall] + g.sigma * n01.x;
  q.vy = g.sigma * n01.y;
  q.vz = g.sigma * n23.x;
  q.ux = g.sigma * n23.y;
  q.uy = g.sigma * n45.x;
  q.uz = g.sigma * n45.y;
  return q;
}

__device__ __forceinline__ uint3 lattice_shift(const Geom& g, uint32_t step) {
  const uint4 r = draw(g, 0u, step, kTagShift, 0u);
  const int sh = 32 - g.F;
  return make_uint3(r.x >> sh, r.y >> sh, r.z >> sh);
}

// float32 product v * (h 2^F) rounded half-to-even, saturated (NaN -> 0), clamped
__device__ __forceinline__ int displacement(float v, float hs, uint32_t P) {
  int d = __float2int_rn(__fmul_rn(v, hs));
  const int lim = (int)(P - 1u);
  return max(-lim, min(lim, d));
}

// (x + d) mod P for x in [0, P), |d| <= P - 1, P <= 2^31, in 32-bit arithmetic
__device__ __forceinline__ uint32_t add_wrap(uint32_t x, int d, uint32_t P) {
  uint32_t t = x + (uint32_t)d;
  if (t >= P) t = (d < 0) ? t + P : t - P;
  return t;
}

// round(num / den) to nearest, ties to even, exact integers (den != 0)
__device__ __forceinline__ int64_t rdiv_half_even(int64_t num, int64_t den) {
  if (den < 0) { num = -num; den = -den; }
  int64_t q = num / den;
  int64_t r = num - q * den;  // sign of num
  const int64_t twice = 2 * (r < 0 ? -r : r);
  if (twice > den || (twice == den && (q & 1))) q += (num < 0) ? -1 : 1;
  return q;
}

// Stored positions carry, in bit 31 of z (positions are below 2^31), whether the
// streaming that produced them crossed a wall.
constexpr uint32_t kCrossedBit = 0x80000000u;

// Lateral displacement along x or y of a particle that bounced back from a no-slip wall
// moving with displacement U per step along that axis (Sec. II, Boundary conditions):
// with the walls at w = -1/2 and P - 1/2 and tau the fraction of the step before the
// hit, d (2 tau - 1) + 2 U (1 - tau) = (d (Z' - Z) + U (2 z_n - 2w)) / dz exactly,
// rounded half to even (Z' the mirrored, z_n the free end position).
__device__ __forceinline__ int bounce_lateral(int d, int U, int64_t Z, int64_t zn, int64_t Znew,
                                              int dz, int64_t two_w) {
  return (int)rdiv_half_even((int64_t)d * (Znew - Z) + (int64_t)U * (2 * zn - two_w), (int64_t)dz);
}

// Eq. (1) with gravity kick and boundary conditions.  In: position x and velocity v
// before the step.  Out: the streamed position (z with kCrossedBit set after a wall
// hit).  The velocity entering the collision is v + g h, reflected at a wall hit as
// collision_velocity() says.
__device__ __forceinline__ void stream(const Geom& g, uint32_t& x, uint32_t& y, uint32_t& z,
                                       float vx, float vy, float vz) {
  vx = __fadd_rn(vx, g.gh[0]);
  vy = __fadd_rn(vy, g.gh[1]);
  vz = __fadd_rn(vz, g.gh[2]);
  int dx = displacement(vx, g.hs, g.P[0]);
  int dy = displacement(vy, g.hs, g.P[1]);
  const int dz = displacement(vz, g.hs, g.P[2]);
  if (g.walls) {
    const int64_t Z = z;
    const int64_t zn = Z + dz;
    const int64_t Pz = g.P[2];
    if (zn >= Pz || zn < 0) {
      const bool top = zn >= Pz;
      const int64_t Znew = top ? (2 * Pz - 1 - zn) : (-1 - zn);
      if (g.walls == 1) {  // no-slip: bounce-back in the frame of the (moving) wall
        const int64_t two_w = top ? 2 * Pz - 1 : -1;
        dx = bounce_lateral(dx, displacement(g.wall_u[top], g.hs, g.P[0]), Z, zn, Znew, dz, two_w);
        dy = bounce_lateral(dy, 0, Z, zn, Znew, dz, two_w);
      }  // slip: specular reflection, the tangential motion continues
      z = (uint32_t)Znew | kCrossedBit;
    } else {
      z = (uint32_t)zn;
    }
  } else {
    z = add_wrap(z, dz, g.P[2]);
  }
  x = add_wrap(x, dx, g.P[0]);
  y = add_wrap(y, dy, g.P[1]);
}

// stream() for a periodic box without gravity whose extents P are powers of two (the
// displacement clamped to +-(P - 1) as there; (x + d) mod P is then a mask): the same
// result in fewer instructions.
__device__ __forceinline__ void stream_periodic_pow2(const Geom& g, uint32_t& x, uint32_t& y, uint32_t& z,
                                                     float vx, float vy, float vz) {
  x = (x + (uint32_t)displacement(vx, g.hs, g.P[0])) & (g.P[0] - 1u);
  y = (y + (uint32_t)displacement(vy, g.hs, g.P[1])) & (g.P[1] - 1u);
  z = (z + (uint32_t)displacement(vz, g.hs, g.P[2])) & (g.P[2] - 1u);
}

// the boxes stream_periodic_pow2 serves
__host__ __device__ inline bool periodic_pow2_box(const Geom& g) {
  bool ok = g.walls == 0 && g.gh[0] == 0.0f && g.gh[1] == 0.0f && g.gh[2] == 0.0f;
  for (int ax = 0; ax < 3; ++ax) ok = ok && (g.P[ax] & (g.P[ax] - 1u)) == 0u;
  return ok;
}

// The exact inverse of stream(): from a stored (streamed) position and the velocity v it
// was streamed with (before the kick), the position before the step.
__device__ __forceinline__ void unstream(const Geom& g, uint32_t& x, uint32_t& y, uint32_t& z,
                                         float vx, float vy, float vz) {
  vx = __fadd_rn(vx, g.gh[0]);
  vy = __fadd_rn(vy, g.gh[1]);
  vz = __fadd_rn(vz, g.gh[2]);
  int dx = displacement(vx, g.hs, g.P[0]);
  int dy = displacement(vy, g.hs, g.P[1]);
  const int dz = displacement(vz, g.hs, g.P[2]);
  const bool crossed = (z & kCrossedBit) != 0;
  const uint32_t zs = z & ~kCrossedBit;
  if (g.walls) {
    if (crossed) {
      const int64_t Pz = g.P[2];
      const bool top = dz > 0;
      const int64_t zn = top ? (2 * Pz - 1 - (int64_t)zs) : (-1 - (int64_t)zs);
      const int64_t Z = zn - dz;
      if (g.walls == 1) {
        const int64_t two_w = top ? 2 * Pz - 1 : -1;
        dx = bounce_lateral(dx, displacement(g.wall_u[top], g.hs, g.P[0]), Z, zn, (int64_t)zs, dz, two_w);
        dy = bounce_lateral(dy, 0, Z, zn, (int64_t)zs, dz, two_w);
      }
      z = (uint32_t)Z;
    } else {
      z = zs - (uint32_t)dz;
    }
  } else {
    z = add_wrap(zs, -dz, g.P[2]);
  }
  x = add_wrap(x, -dx, g.P[0]);
  y = add_wrap(y, -dy, g.P[1]);
}

// velocity entering the collision for a particle stored as (streamed x, pre-kick v): the
// kicked velocity, after a wall hit reflected -- specularly (slip: v_z flips) or in the
// frame of the wall it hit (no-slip: v -> 2 u_wall - v)
__device__ __forceinline__ void collision_velocity(const Geom& g, uint32_t zraw, float& vx, float& vy,
                                                   float& vz) {
  vx = __fadd_rn(vx, g.gh[0]);
  vy = __fadd_rn(vy, g.gh[1]);
  vz = __fadd_rn(vz, g.gh[2]);
  if (zraw & kCrossedBit) {
    if (g.walls == 2) {
      vz = -vz;
    } else {
      const bool top = vz > 0.0f;  // moving up before the hit: the wall at z = Lz
      vx = 2.0f * g.wall_u[top] - vx;
      vy = -vy;
      vz = -vz;
    }
  }
}

// cell of the shifted lattice, per axis; periodic axes wrap index L to 0
__device__ __forceinline__ int cell_axis(const Geom& g, uint32_t x, uint32_t s, int ax) {
  int c = (int)((x + s) >> g.F);
  if (c >= g.L[ax] && (ax < 2 || !g.walls)) c -= g.L[ax];
  return c;
}

// position relative to the cell centre, in units of a
__device__ __forceinline__ float rho_axis(const Geom& g, uint32_t x, uint32_t s) {
  const int u = (int)((x + s) & g.mask) - (int)(1u << (g.F - 1));
  return __fmul_rn((float)u, g.inv2F);
}

}  // namespace mpc
