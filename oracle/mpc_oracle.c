/*
 * Oracle for one MPC step -- TEST INFRASTRUCTURE ONLY (see mpc_oracle.h).
 *
 * Plain single-threaded C, FP64 throughout except where the written state contract
 * fixes a float32 operation (the displacement product of the fixed-point streaming,
 * and the accept/reject decisions of the gamma sampler, which are taken in the same
 * float32 precision as the GPU kernel takes them).  No blocking, no fusion: every step
 * follows the paper's order -- stream (Eq. 1), shift the lattice, sort into cells,
 * collide (Eq. 2 / Eqs. 3-4 / AT+a), thermostat (Eqs. 5-7).
 *
 * Parity pins (tests/test_oracle_*.py): Philox against cuRAND's host generator; the
 * rotation against scipy's Rotation; cell assignment against exact rational
 * enumeration; streaming and wall reflections against their closed forms; conservation
 * laws; sampler distributions against scipy.stats; equipartition; Poiseuille flow
 * against its closed form; the angular-momentum solve against numpy's solve / pinv and
 * its float32 sensitivity against float32 evaluations; the ill-conditioning flag against
 * LAPACK eigenvalues; phantom particles (counts, aggregate momentum and energy, one-by-one
 * positions and velocities) against their distributions and an independent numpy
 * collision; the stress observables against the momentum flux through planes, and their
 * Green-Kubo viscosity against the SRD closed form.  Every function here has a pin.
 */
#include "mpc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Philox counter word 2 carries (tag << 24) | sub-draw index.  The tag values are a
 * keying contract shared (by value, not by code) with the CUDA implementation. */
#define TAG_SHIFT 1u
#define TAG_AXIS 2u
#define TAG_MBS 3u
#define TAG_PHANTOM 4u
#define TAG_PHGAMMA 5u
#define TAG_ATV 6u
#define TAG_INITX 7u
#define TAG_INITV 8u
#define TAG_PHPART 9u
#define TAG_TEST 15u

#define GAMMA_MAX_ATTEMPTS 32
#define POISSON_MAX_K 100000

/* ------------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications whose halves are
 * xor-ed with the other two words and the round key; the key is bumped by the two
 * Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod1;
    uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(const orc_params* p, uint32_t c0, uint32_t c1, uint32_t tag, uint32_t sub,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, (tag << 24) | sub, p->box};
  uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* uniform in (0,1): the top 23 random bits plus half of their ulp, (2k+1) / 2^24 with
 * k < 2^23 -- a 24-bit odd numerator, so the value is exact in float and double */
static double uniform01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller: two uniforms -> two independent standard normals */
static void box_muller(double u0, double u1, double* z0, double* z1) {
  double R = sqrt(-2.0 * log(u0));
  double phi = 2.0 * M_PI * u1;
  *z0 = R * cos(phi);
  *z1 = R * sin(phi);
}

static int near(double a, double b, double rel) {
  double s = fabs(a) + fabs(b);
  return fabs(a - b) <= rel * (s > 1.0 ? s : 1.0);
}

/* Gamma(shape a >= 1, scale 1) by Marsaglia & Tsang (ACM TOMS 26, 2000): d = a - 1/3,
 * c = 1/sqrt(9d); propose v = (1 + c x)^3 from a standard normal x and accept with the
 * squeeze u < 1 - 0.0331 x^4 or the exact test ln u < x^2/2 + d(1 - v + ln v).
 * Attempt k draws Philox(c0, c1, tag, k).  The decisions are taken in float32 with
 * the same expressions as the GPU kernel; the returned value is FP64. */
static double gamma_mt(const orc_params* p, uint32_t c0, uint32_t c1, uint32_t tag, double a,
                       int* near_tie) {
  float a_f = (float)a;
  float d_f = a_f - (1.0f / 3.0f);
  float c_f = 1.0f / sqrtf(9.0f * d_f);
  for (uint32_t k = 0; k < GAMMA_MAX_ATTEMPTS; ++k) {
    uint32_t r[4];
    draw(p, c0, c1, tag, k, r);
    double z0, z1;
    box_muller(uniform01(r[0]), uniform01(r[1]), &z0, &z1);
    (void)z1;
    double x_d = z0;
    float x = (float)x_d;
    float u = (float)uniform01(r[2]);
    float v1 = fmaf(c_f, x, 1.0f);
    if (near_tie && near((double)v1, 0.0, 1e-5)) *near_tie = 1;
    if (v1 <= 0.0f) continue;
    float v3 = (v1 * v1) * v1;
    float x2 = x * x;
    float x4 = x2 * x2;
    float squeeze = 1.0f - 0.0331f * x4;
    if (near_tie && near((double)u, (double)squeeze, 1e-5)) *near_tie = 1;
    double vd = 1.0 + (double)c_f * x_d;
    double value = (double)d_f * vd * vd * vd;
    if (u < squeeze) return value;
    float lhs = logf(u);
    float rhs = 0.5f * x2 + d_f * (1.0f - v3 + logf(v3));
    if (near_tie && near((double)lhs, (double)rhs, 1e-5)) *near_tie = 1;
    if (lhs < rhs) return value;
  }
  return (double)d_f;
}

/* Poisson(lambda) by sequential inversion of the CDF with one uniform, FP64 */
static int32_t poisson_inv(double u, double lambda, int* near_tie) {
  int32_t k = 0;
  double prob = exp(-lambda);
  double cdf = prob;
  while (u > cdf && k < POISSON_MAX_K) {
    if (near_tie && fabs(u - cdf) < 1e-12) *near_tie = 1;
    k += 1;
    prob *= lambda / (double)k;
    cdf += prob;
  }
  if (near_tie && fabs(u - cdf) < 1e-12) *near_tie = 1;
  return k;
}

/* ------------------------------------------------------------------------------ */
/* fixed-point position contract: F fractional bits per cell, P = L * 2^F < 2^32     */

static int ceil_log2(int32_t v) {
  int k = 0;
  while ((1LL << k) < (int64_t)v) ++k;
  return k;
}

int orc_fixed_bits(const orc_params* p) {
  int32_t lmax = p->L[0];
  if (p->L[1] > lmax) lmax = p->L[1];
  if (p->L[2] > lmax) lmax = p->L[2];
  return 31 - ceil_log2(lmax);
}

int64_t orc_num_particles(const orc_params* p) {
  double vol = (double)p->L[0] * (double)p->L[1] * (double)p->L[2];
  return (int64_t)llround(vol * p->n_c);
}

int64_t orc_num_cells(const orc_params* p) {
  return (int64_t)p->L[0] * p->L[1] * (p->L[2] + (p->walls_z ? 1 : 0));
}

void orc_shift(const orc_params* p, int64_t step, uint32_t S[3]) {
  int F = orc_fixed_bits(p);
  uint32_t r[4];
  draw(p, 0u, (uint32_t)step, TAG_SHIFT, 0u, r);
  for (int ax = 0; ax < 3; ++ax) S[ax] = r[ax] >> (32 - F);
}

/* displacement of one axis: the float32 product v * (h 2^F), rounded half-to-even to an
 * integer, saturated to the int32 range (NaN -> 0), then clamped to +-(P-1) */
static int64_t displacement(double v, float hs, uint32_t P) {
  float vf = (float)v;
  float prod = vf * hs;
  int64_t d;
  if (isnan(prod)) d = 0;
  else if (prod >= 2147483648.0f) d = 2147483647LL;
  else if (prod <= -2147483648.0f) d = -2147483648LL;
  else d = (int64_t)nearbyintf(prod);
  int64_t lim = (int64_t)P - 1;
  if (d > lim) d = lim;
  if (d < -lim) d = -lim;
  return d;
}

/* exact rational num/den rounded to the nearest integer, ties to even (den != 0) */
static int64_t div_round_half_even(int64_t num, int64_t den) {
  int64_t q = num / den;
  int64_t r = num % den;
  if (r == 0) return q;
  int64_t sgn = ((num < 0) != (den < 0)) ? -1 : 1;
  int64_t twice = 2 * (r < 0 ? -r : r);
  int64_t aden = den < 0 ? -den : den;
  if (twice > aden || (twice == aden && (q & 1))) q += sgn;
  return q;
}

static uint32_t wrap_periodic(int64_t t, uint32_t P) {
  int64_t PP = (int64_t)P;
  if (t < 0) t += PP;
  else if (t >= PP) t -= PP;
  return (uint32_t)t;
}

typedef struct {
  int F;
  uint32_t P[3];
  float hs;       /* float32(h * 2^F) */
  float gh[3];    /* float32(g * h) */
  double inv2F;
} geom_t;

static geom_t make_geom(const orc_params* p) {
  geom_t g;
  g.F = orc_fixed_bits(p);
  for (int ax = 0; ax < 3; ++ax) g.P[ax] = (uint32_t)p->L[ax] << g.F;
  g.hs = (float)ldexp(p->h, g.F);
  for (int ax = 0; ax < 3; ++ax) g.gh[ax] = (float)(p->g[ax] * p->h);
  g.inv2F = ldexp(1.0, -g.F);
  return g;
}

/* Streaming, Eq. (1): kick by gravity ("External fields"), move ballistically, and
 * apply the boundary conditions ("Boundary conditions"): periodic wrap; or, at the z
 * walls, no-slip bounce-back -- the particle is reflected back into the box for the
 * remainder of the step and its velocity relative to the wall is reversed (a wall
 * moving with u along x: v -> 2u - v) -- or slip (specular reflection: only v_z flips,
 * the tangential motion continues).  x: fixed-point position (in/out); v: velocity (in:
 * pre-kick; out: the velocity that enters the collision).
 *
 * Bounce-back positions in fixed point: the walls sit at w = -1/2 and P - 1/2, the z
 * position is mirrored about the wall, and with tau the fraction of the step before the
 * hit the lateral displacement is dx (2 tau - 1) + 2 U (1 - tau), U the wall's own
 * displacement over a step; with 2 tau - 1 = (Z' - Z)/dz and 2(1 - tau) = (2 z_n - 2w)/dz
 * this is the exact rational (dx (Z' - Z) + U (2 z_n - 2w)) / dz, rounded half to even. */
static void stream_particle(const orc_params* p, const geom_t* g, uint32_t x[3], double v[3]) {
  double vk[3];
  int64_t d[3];
  for (int ax = 0; ax < 3; ++ax) {
    vk[ax] = v[ax] + (double)g->gh[ax];
    d[ax] = displacement(vk[ax], g->hs, g->P[ax]);
  }
  int crossed = 0, top = 0;
  if (p->walls_z) {
    int64_t Z = (int64_t)x[2];
    int64_t zn = Z + d[2];
    int64_t Pz = (int64_t)g->P[2];
    int64_t Znew = zn;
    if (zn >= Pz) { Znew = 2 * Pz - 1 - zn; crossed = 1; top = 1; }
    else if (zn < 0) { Znew = -1 - zn; crossed = 1; }
    if (crossed && p->walls_z == 1) {
      const int64_t U = displacement(p->wall_u[top], g->hs, g->P[0]);
      const int64_t two_w = top ? 2 * Pz - 1 : -1;
      d[0] = div_round_half_even(d[0] * (Znew - Z) + U * (2 * zn - two_w), d[2]);
      d[1] = div_round_half_even(d[1] * (Znew - Z), d[2]);
    }
    x[2] = (uint32_t)Znew;
  } else {
    x[2] = wrap_periodic((int64_t)x[2] + d[2], g->P[2]);
  }
  x[0] = wrap_periodic((int64_t)x[0] + d[0], g->P[0]);
  x[1] = wrap_periodic((int64_t)x[1] + d[1], g->P[1]);
  for (int ax = 0; ax < 3; ++ax) v[ax] = vk[ax];
  if (crossed && p->walls_z == 2) {
    v[2] = -vk[2];
  } else if (crossed) {
    v[0] = 2.0 * p->wall_u[top] - vk[0];
    v[1] = -vk[1];
    v[2] = -vk[2];
  }
}

void orc_stream_one(const orc_params* p, uint32_t x[3], double v[3]) {
  geom_t g = make_geom(p);
  stream_particle(p, &g, x, v);
}

/* collision cell of a position on the lattice shifted by S (Sec. II: the whole lattice
 * is shifted by a random vector before every collision); rho = position relative to the
 * cell centre in units of a */
int orc_cell_of(const orc_params* p, const uint32_t x[3], const uint32_t S[3], uint32_t* cell,
                double rho[3]) {
  geom_t g = make_geom(p);
  uint32_t mask = (1u << g.F) - 1u;
  uint32_t c[3];
  for (int ax = 0; ax < 3; ++ax) {
    uint32_t t = x[ax] + S[ax];
    c[ax] = t >> g.F;
    int periodic = (ax < 2) || !p->walls_z;
    if (periodic && c[ax] >= (uint32_t)p->L[ax]) c[ax] -= (uint32_t)p->L[ax];
    int64_t u = (int64_t)(t & mask) - (int64_t)(1u << (g.F - 1));
    rho[ax] = (double)u * g.inv2F;
  }
  *cell = c[0] + (uint32_t)p->L[0] * (c[1] + (uint32_t)p->L[1] * c[2]);
  return 0;
}

void orc_srd_axis(const orc_params* p, int64_t step, uint32_t cell, double axis[3]) {
  uint32_t r[4];
  draw(p, cell, (uint32_t)step, TAG_AXIS, 0u, r);
  double cos_t = 2.0 * uniform01(r[0]) - 1.0;
  double phi = 2.0 * M_PI * uniform01(r[1]);
  double sin_t = sqrt(fmax(0.0, 1.0 - cos_t * cos_t));
  axis[0] = sin_t * cos(phi);
  axis[1] = sin_t * sin(phi);
  axis[2] = cos_t;
}

/* rotation by alpha about a unit axis (Rodrigues): D v = v cos a + (n x v) sin a
 * + n (n.v)(1 - cos a) */
void orc_rotate(const double n[3], double alpha, const double v[3], double out[3]) {
  double ca = cos(alpha), sa = sin(alpha);
  double nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
  double cx = n[1] * v[2] - n[2] * v[1];
  double cy = n[2] * v[0] - n[0] * v[2];
  double cz = n[0] * v[1] - n[1] * v[0];
  out[0] = v[0] * ca + cx * sa + n[0] * nv * (1.0 - ca);
  out[1] = v[1] * ca + cy * sa + n[1] * nv * (1.0 - ca);
  out[2] = v[2] * ca + cz * sa + n[2] * nv * (1.0 - ca);
}

static void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* smallest and largest eigenvalue of a symmetric 3x3 matrix, closed form of O. K. Smith,
 * "Eigenvalues of a symmetric 3x3 matrix", CACM 4 (1961): with q = tr(A)/3 and
 * B = (A - q 1)/p, the eigenvalues are q + 2 p cos(phi + 2 pi k/3), phi = acos(det(B)/2)/3 */
static void eigen_extremes_sym3(const double A[3][3], double* lmin, double* lmax) {
  double p1 = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
  double q = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
  if (p1 == 0.0) {
    double lo = A[0][0], hi = A[0][0];
    for (int a = 1; a < 3; ++a) {
      if (A[a][a] < lo) lo = A[a][a];
      if (A[a][a] > hi) hi = A[a][a];
    }
    *lmin = lo;
    *lmax = hi;
    return;
  }
  double p2 = (A[0][0] - q) * (A[0][0] - q) + (A[1][1] - q) * (A[1][1] - q) +
              (A[2][2] - q) * (A[2][2] - q) + 2.0 * p1;
  double pp = sqrt(p2 / 6.0);
  double B[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) B[a][b] = (A[a][b] - (a == b ? q : 0.0)) / pp;
  double detB = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  double r = detB / 2.0;
  if (r < -1.0) r = -1.0;
  if (r > 1.0) r = 1.0;
  double phi = acos(r) / 3.0;
  *lmax = q + 2.0 * pp * cos(phi);
  *lmin = q + 2.0 * pp * cos(phi + 2.0 * M_PI / 3.0);
}

static double min_eigenvalue_sym3(const double A[3][3]) {
  double lo, hi;
  eigen_extremes_sym3(A, &lo, &hi);
  return lo;
}

/* First-order sensitivity of the new velocities to float32 rounding in the cell's
 * angular-momentum solve (test diagnostics, in units of the rounding unit u): relative
 * rounding of every product and of the centre-of-mass positions (|rho| <= 1) perturbs
 * L = sum r_j x w_j by ~ sum |r_j||w_j| + sum |w_j| and J by ~ 2 sum |r_j|; omega = J^-1 L
 * then moves by 1/lambda_min times (dL + |omega| dJ), and omega x r_i by that times |r_i|,
 * plus |omega| times the rounding of r_i itself.  Returns the factor multiplying |r_i|
 * (per cell); the caller adds the direct 2|omega| term. */
static double omega_sensitivity(int64_t n, const double J[3][3], const double pair_axis[3],
                                double sum_rw, double sum_w, double sum_r, double omega_norm) {
  if (n <= 1) return 0.0;
  double lam;
  if (n == 2) {
    double d2 = pair_axis[0] * pair_axis[0] + pair_axis[1] * pair_axis[1] +
                pair_axis[2] * pair_axis[2];
    lam = 0.5 * d2;
  } else {
    lam = min_eigenvalue_sym3(J);
  }
  return lam > 0.0 ? (sum_rw + sum_w + 2.0 * omega_norm * sum_r) / lam : INFINITY;
}

/* omega = J^{-1} Lr for the geometric moment-of-inertia tensor J of a cell
 * (n >= 3: inverse; n == 2: pseudo-inverse on the plane normal to the pair axis;
 * otherwise zero).  Returns flags. */
static int solve_inertia(int64_t n, const double J[3][3], const double Lr[3],
                         const double pair_axis[3], double omega[3]) {
  omega[0] = omega[1] = omega[2] = 0.0;
  if (n <= 1) return 0;
  /* members within ORC_TIGHT_RMS of their centre of mass: see ORC_FLAG_ILL_CONDITIONED */
  const double trM = 0.5 * (J[0][0] + J[1][1] + J[2][2]);
  const int tight = trM < ORC_TIGHT_RMS * ORC_TIGHT_RMS * (double)n ? ORC_FLAG_ILL_CONDITIONED : 0;
  if (n == 2) {
    double d2 = pair_axis[0] * pair_axis[0] + pair_axis[1] * pair_axis[1] +
                pair_axis[2] * pair_axis[2];
    if (d2 <= 0.0) return ORC_FLAG_DEGENERATE;
    double dl = (pair_axis[0] * Lr[0] + pair_axis[1] * Lr[1] + pair_axis[2] * Lr[2]) / d2;
    for (int a = 0; a < 3; ++a) omega[a] = (2.0 / d2) * (Lr[a] - pair_axis[a] * dl);
    return tight;
  }
  double A[3][3];
  A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  double det = J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
  if (!(det > 0.0)) return ORC_FLAG_DEGENERATE;
  /* ill-conditioned for a float32 solve: see ORC_FLAG_ILL_CONDITIONED */
  double lo, hi;
  eigen_extremes_sym3(J, &lo, &hi);
  int flags = (!(lo > 0.0) || hi > ORC_COND_FLOAT32 * lo) ? ORC_FLAG_ILL_CONDITIONED : tight;
  for (int a = 0; a < 3; ++a)
    omega[a] = (A[a][0] * Lr[0] + A[a][1] * Lr[1] + A[a][2] * Lr[2]) / det;
  return flags;
}

/* The angular-momentum restoring rotation of one cell (Eqs. 3-4 for SRD+a; the same
 * construction for AT+a): with r_j = rho_j - rho_cm the positions relative to the cell's
 * centre of mass (unit masses), J = sum_j (|r_j|^2 1 - r_j r_j^T) the moment-of-inertia
 * tensor and L = sum_j r_j x w_j the angular momentum the collision would otherwise
 * change, omega = J^{-1} L.  rho, w: 3n values (particle-major); sens (n values or NULL):
 * the float32 rounding sensitivity of each particle's new velocity (omega_sensitivity
 * times |r_i|, plus 2|omega| for the rounding of r_i itself).  Returns cell flags. */
int orc_cell_omega(int64_t n, const double* rho, const double* w, double omega[3],
                   double rcm[3], double* sens) {
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double Lr[3] = {0, 0, 0};
  double pair_axis[3] = {0, 0, 0};
  double sum_rw = 0.0, sum_w = 0.0, sum_r = 0.0;
  rcm[0] = rcm[1] = rcm[2] = 0.0;
  omega[0] = omega[1] = omega[2] = 0.0;
  if (n <= 0) return 0;
  for (int64_t k = 0; k < n; ++k)
    for (int a = 0; a < 3; ++a) rcm[a] += rho[3 * k + a];
  for (int a = 0; a < 3; ++a) rcm[a] /= (double)n;
  if (n == 2)
    for (int a = 0; a < 3; ++a) pair_axis[a] = rho[a] - rho[3 + a];
  for (int64_t k = 0; k < n; ++k) {
    double r[3], rxw[3];
    for (int a = 0; a < 3; ++a) r[a] = rho[3 * k + a] - rcm[a];
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) J[a][b] += (a == b ? r2 : 0.0) - r[a] * r[b];
    cross3(r, w + 3 * k, rxw);
    for (int a = 0; a < 3; ++a) Lr[a] += rxw[a];
    const double* wv = w + 3 * k;
    double wn = sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
    sum_rw += sqrt(r2) * wn;
    sum_w += wn;
    sum_r += sqrt(r2);
  }
  int flags = solve_inertia(n, J, Lr, pair_axis, omega);
  if (sens) {
    double on = sqrt(omega[0] * omega[0] + omega[1] * omega[1] + omega[2] * omega[2]);
    double sc = omega_sensitivity(n, J, pair_axis, sum_rw, sum_w, sum_r, on);
    for (int64_t k = 0; k < n; ++k) {
      double r[3];
      for (int a = 0; a < 3; ++a) r[a] = rho[3 * k + a] - rcm[a];
      sens[k] = sc * sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) + 2.0 * on;
    }
  }
  return flags;
}

/* Phantom particles of a wall-cut cell (Sec. II, "Boundary conditions"): the part of the
 * cell inside the wall (volume fraction phi) is filled with virtual particles at the mean
 * density, with Maxwell-Boltzmann velocities about the wall's own velocity.  Only their
 * aggregates enter an SRD collision, so they are drawn as aggregates: the count
 * k ~ Poisson(N_c phi); the total momentum, per component m k u_wall + N(0, k m kT); and
 * Kint = sum m |v - <v>|^2 about their own mean velocity (twice their internal kinetic
 * energy), kT chi^2(3(k - 1)), i.e. 2 kT times a Gamma(3(k - 1)/2) draw -- exact in
 * distribution for k Gaussian velocities.  wall: 0 the
 * wall at z = 0, 1 the wall at z = Lz.  Returns cell flags (near-tie decisions). */
int orc_phantoms(const orc_params* p, int64_t step, uint32_t cell, double phi, int wall,
                 double* nph, double P[3], double* Kint) {
  const double m = p->m;
  int flags = 0;
  uint32_t r[4], r1[4];
  draw(p, cell, (uint32_t)step, TAG_PHANTOM, 0u, r);
  draw(p, cell, (uint32_t)step, TAG_PHANTOM, 1u, r1);
  int tie = 0;
  int32_t k = poisson_inv(uniform01(r[0]), p->n_c * phi, &tie);
  if (tie) flags |= ORC_FLAG_POISSON_NEAR_TIE;
  *nph = (double)k;
  double zx, zy, zz, zdummy;
  box_muller(uniform01(r[1]), uniform01(r[2]), &zx, &zy);
  box_muller(uniform01(r1[0]), uniform01(r1[1]), &zz, &zdummy);
  double sp = m * sqrt((double)k * p->kT / m);
  /* phantoms move with their wall on average */
  P[0] = sp * zx + m * (double)k * p->wall_u[wall];
  P[1] = sp * zy;
  P[2] = sp * zz;
  *Kint = 0.0;
  if (k >= 2) {
    int t2 = 0;
    *Kint = p->kT * 2.0 * gamma_mt(p, cell, (uint32_t)step, TAG_PHGAMMA, 1.5 * (double)(k - 1), &t2);
    if (t2) flags |= ORC_FLAG_MBS_NEAR_TIE;
  }
  return flags;
}

/* Phantom particles of a wall-cut cell one by one, for the angular-momentum-conserving
 * variants, whose collision needs every member's position (Sec. II, "Boundary
 * conditions"; positions drawn uniformly in the wall part of the cell).  The count k is
 * orc_phantoms' count for the same cell and step.  Phantom j draws Philox(cell, step,
 * TAG_PHPART, 3j + q): q = 0 its position on the fixed-point grid of the cell -- x and y
 * uniform over the cell, z uniform over the part beyond the wall (local coordinate below
 * the lattice shift Sz at the bottom wall, at or above it at the top wall) --, q = 1, 2 six
 * standard normals by Box-Muller: its velocity u_wall x + sqrt(kT/m) (n0, n1, n2) and its
 * random velocity sqrt(kT/m) (n3, n4, n5).  rho (3k): positions relative to the cell
 * centre; v, vran (3k).  wall: 0 bottom (z = 0), 1 top (z = Lz). */
void orc_phantom_particles(const orc_params* p, int64_t step, uint32_t cell, uint32_t Sz, int wall,
                           int32_t k, double* rho, double* v, double* vran) {
  const int F = orc_fixed_bits(p);
  const uint64_t one = (uint64_t)1 << F;
  const double inv2F = ldexp(1.0, -F), sigma = sqrt(p->kT / p->m);
  for (int32_t j = 0; j < k; ++j) {
    uint32_t a[4], b[4], c[4];
    draw(p, cell, (uint32_t)step, TAG_PHPART, 3u * (uint32_t)j, a);
    draw(p, cell, (uint32_t)step, TAG_PHPART, 3u * (uint32_t)j + 1u, b);
    draw(p, cell, (uint32_t)step, TAG_PHPART, 3u * (uint32_t)j + 2u, c);
    const uint64_t ix = a[0] >> (32 - F), iy = a[1] >> (32 - F);
    const uint64_t iz = wall == 0 ? (((uint64_t)a[2] * (uint64_t)Sz) >> 32)
                                  : (uint64_t)Sz + (((uint64_t)a[2] * (one - (uint64_t)Sz)) >> 32);
    const double half = (double)(one >> 1);
    rho[3 * j + 0] = ((double)ix - half) * inv2F;
    rho[3 * j + 1] = ((double)iy - half) * inv2F;
    rho[3 * j + 2] = ((double)iz - half) * inv2F;
    double n0, n1, n2, n3, n4, n5;
    box_muller(uniform01(b[0]), uniform01(b[1]), &n0, &n1);
    box_muller(uniform01(b[2]), uniform01(b[3]), &n2, &n3);
    box_muller(uniform01(c[0]), uniform01(c[1]), &n4, &n5);
    v[3 * j + 0] = p->wall_u[wall] + sigma * n0;
    v[3 * j + 1] = sigma * n1;
    v[3 * j + 2] = sigma * n2;
    vran[3 * j + 0] = sigma * n3;
    vran[3 * j + 1] = sigma * n4;
    vran[3 * j + 2] = sigma * n5;
  }
}

/* ------------------------------------------------------------------------------ */

int orc_init(const orc_params* p, int64_t N, uint32_t* X, double* V, uint32_t* id) {
  geom_t g = make_geom(p);
  double sigma = sqrt(p->kT / p->m);
  double mean[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < N; ++i) {
    uint32_t r[4];
    draw(p, (uint32_t)i, 0u, TAG_INITX, 0u, r);
    for (int ax = 0; ax < 3; ++ax)
      X[ax * N + i] = (uint32_t)(((uint64_t)r[ax] * (uint64_t)g.P[ax]) >> 32);
    draw(p, (uint32_t)i, 0u, TAG_INITV, 0u, r);
    double z0, z1, z2, z3;
    box_muller(uniform01(r[0]), uniform01(r[1]), &z0, &z1);
    box_muller(uniform01(r[2]), uniform01(r[3]), &z2, &z3);
    V[0 * N + i] = sigma * z0;
    V[1 * N + i] = sigma * z1;
    V[2 * N + i] = sigma * z2;
    for (int ax = 0; ax < 3; ++ax) mean[ax] += V[ax * N + i];
    id[i] = (uint32_t)i;
  }
  for (int ax = 0; ax < 3; ++ax) mean[ax] /= (double)(N > 0 ? N : 1);
  for (int64_t i = 0; i < N; ++i)
    for (int ax = 0; ax < 3; ++ax) V[ax * N + i] -= mean[ax];
  return 0;
}

/* One MPC step (step index `step`) applied to the state (X, V, id) in place. */
int orc_step(const orc_params* p, int64_t N, uint32_t* X, double* V, const uint32_t* id,
             int64_t step, uint32_t* cell_out, uint32_t* count_out, double* vpre_out,
             double* obs_out, uint8_t* cell_flags, double* sens_out) {
  geom_t g = make_geom(p);
  const int64_t C = orc_num_cells(p);
  const double m = p->m;
  const double alpha = p->alpha_deg * M_PI / 180.0;
  const double sigma = sqrt(p->kT / p->m);

  uint32_t* cell = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1));
  double* rho = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
  double* vb = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
  int64_t* start = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
  int64_t* members = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  int64_t* fill = (int64_t*)calloc((size_t)C + 1, sizeof(int64_t));
  if (!cell || !rho || !vb || !start || !members || !fill) return -1;
  if (cell_flags) memset(cell_flags, 0, (size_t)C);

  /* 1. random shift of the collision lattice, one vector per step */
  uint32_t S[3];
  orc_shift(p, step, S);

  /* 2. streaming with boundary conditions, Eq. (1) */
  for (int64_t i = 0; i < N; ++i) {
    uint32_t x[3] = {X[i], X[N + i], X[2 * N + i]};
    double v[3] = {V[i], V[N + i], V[2 * N + i]};
    stream_particle(p, &g, x, v);
    for (int ax = 0; ax < 3; ++ax) {
      X[ax * N + i] = x[ax];
      vb[3 * i + ax] = v[ax];
    }
    /* 3. sort into the cells of the shifted lattice */
    orc_cell_of(p, x, S, &cell[i], &rho[3 * i]);
  }

  /* member lists per cell (plain counting sort) */
  for (int64_t i = 0; i < N; ++i) start[cell[i] + 1] += 1;
  for (int64_t c = 0; c < C; ++c) start[c + 1] += start[c];
  for (int64_t i = 0; i < N; ++i) {
    int64_t c = cell[i];
    members[start[c] + fill[c]] = i;
    fill[c] += 1;
  }

  double* vnew = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
  if (!vnew) return -1;
  const double fluid_volume = (double)p->L[0] * p->L[1] * p->L[2];

  /* 4. collision per cell */
  for (int64_t c = 0; c < C; ++c) {
    int64_t n = start[c + 1] - start[c];
    if (count_out) count_out[c] = (uint32_t)n;
    if (n == 0) continue;
    const int64_t* mem = members + start[c];
    int flags = 0;
    double sumv[3] = {0, 0, 0};
    for (int64_t k = 0; k < n; ++k)
      for (int a = 0; a < 3; ++a) sumv[a] += vb[3 * mem[k] + a];

    if (p->variant == ORC_SRD) {
      /* phantom particles in the wall part of cut cells (Sec. II, Boundary conditions) */
      double nph = 0.0, Pph[3] = {0, 0, 0}, Kint = 0.0;
      if (p->walls_z == 1) {
        int64_t cz = c / ((int64_t)p->L[0] * p->L[1]);
        double s = (double)S[2] * g.inv2F;
        double phi = -1.0;
        if (cz == 0) phi = s;
        else if (cz == p->L[2]) phi = 1.0 - s;
        if (phi >= 0.0)
          flags |= orc_phantoms(p, step, (uint32_t)c, phi, cz == 0 ? 0 : 1, &nph, Pph, &Kint);
      }
      double ntot = (double)n + nph;
      double vcm[3];
      for (int a = 0; a < 3; ++a) vcm[a] = (m * sumv[a] + Pph[a]) / (m * ntot);
      double axis[3];
      orc_srd_axis(p, step, (uint32_t)c, axis);
      double kappa = 1.0;
      if (p->thermostat && ntot >= 2.0) {
        /* MBS, Eqs. (5)-(7): kappa = sqrt(2 E_k / sum m v_ic^2), E_k ~ Gamma(f/2, kT) */
        double Krel = 0.0;
        for (int64_t k = 0; k < n; ++k)
          for (int a = 0; a < 3; ++a) {
            double dv = vb[3 * mem[k] + a] - vcm[a];
            Krel += m * dv * dv;
          }
        if (nph > 0.0) {
          Krel += Kint;
          for (int a = 0; a < 3; ++a) {
            double dv = Pph[a] / (m * nph) - vcm[a];
            Krel += nph * m * dv * dv;
          }
        }
        int tie = 0;
        double Ek = p->kT * gamma_mt(p, (uint32_t)c, (uint32_t)step, TAG_MBS,
                                     1.5 * (ntot - 1.0), &tie);
        if (tie) flags |= ORC_FLAG_MBS_NEAR_TIE;
        if (Krel > 0.0) kappa = sqrt(2.0 * Ek / Krel);
      }
      /* SRD, Eq. (2): v_i <- v_cm + D(alpha) (v_i - v_cm), scaled by kappa */
      for (int64_t k = 0; k < n; ++k) {
        int64_t i = mem[k];
        double rel[3], rot[3];
        for (int a = 0; a < 3; ++a) rel[a] = vb[3 * i + a] - vcm[a];
        orc_rotate(axis, alpha, rel, rot);
        for (int a = 0; a < 3; ++a) vnew[3 * i + a] = vcm[a] + kappa * rot[a];
        if (sens_out) sens_out[i] = 0.0;
      }
    } else {
      /* angular-momentum-conserving variants: centre-of-mass frame of the cell.  In a
       * cell cut by a no-slip wall the members are the fluid particles and the phantom
       * particles of the wall part (orc_phantom_particles); only the fluid ones are
       * updated. */
      int32_t kph = 0;
      uint32_t Sz = S[2];
      int wall = 0;
      if (p->walls_z == 1) {
        int64_t cz = c / ((int64_t)p->L[0] * p->L[1]);
        double s_frac = (double)S[2] * g.inv2F;
        double phi = -1.0;
        if (cz == 0) phi = s_frac;
        else if (cz == p->L[2]) { phi = 1.0 - s_frac; wall = 1; }
        if (phi >= 0.0) {
          double nph, Pph[3], Kint;
          flags |= orc_phantoms(p, step, (uint32_t)c, phi, wall, &nph, Pph, &Kint);
          kph = (int32_t)nph;
        }
      }
      const int64_t nt = n + kph;  /* all members */
      double* rk = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
      double* vk = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
      double* ran = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
      double* wk = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
      double* dv = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
      double* sk = (double*)malloc(sizeof(double) * (size_t)nt);
      if (!rk || !vk || !ran || !wk || !dv || !sk) return -1;
      for (int64_t k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
          rk[3 * k + a] = rho[3 * mem[k] + a];
          vk[3 * k + a] = vb[3 * mem[k] + a];
        }
      if (kph > 0)
        orc_phantom_particles(p, step, (uint32_t)c, Sz, wall, kph, rk + 3 * n, vk + 3 * n, ran + 3 * n);
      double vcm[3] = {0, 0, 0};
      for (int64_t k = 0; k < nt; ++k)
        for (int a = 0; a < 3; ++a) vcm[a] += vk[3 * k + a];
      for (int a = 0; a < 3; ++a) vcm[a] /= (double)nt;
      double vrm[3] = {0, 0, 0};
      if (p->variant == ORC_AT_A) {
        /* MPC-AT+a: v_i' = v_cm + v_i^ran - <v^ran> + omega x r_ic, with
         * omega = J^{-1} sum_j r_jc x (v_j - v_j^ran), v^ran ~ N(0, kT/m) per component
         * (fluid particles keyed by their id) */
        for (int64_t k = 0; k < n; ++k) {
          uint32_t r[4];
          draw(p, id[mem[k]], (uint32_t)step, TAG_ATV, 0u, r);
          double z0, z1, z2, z3;
          box_muller(uniform01(r[0]), uniform01(r[1]), &z0, &z1);
          box_muller(uniform01(r[2]), uniform01(r[3]), &z2, &z3);
          ran[3 * k + 0] = sigma * z0;
          ran[3 * k + 1] = sigma * z1;
          ran[3 * k + 2] = sigma * z2;
        }
        for (int64_t k = 0; k < nt; ++k)
          for (int a = 0; a < 3; ++a) {
            vrm[a] += ran[3 * k + a];
            wk[3 * k + a] = vk[3 * k + a] - ran[3 * k + a];
            dv[3 * k + a] = ran[3 * k + a];
          }
        for (int a = 0; a < 3; ++a) vrm[a] /= (double)nt;
      } else {
        /* MPC-SRD+a, Eqs. (3)-(4): v_i' = v_cm + D v_ic + omega x r_ic with
         * omega = m I^{-1} sum_i r_ic x (v_ic - D v_ic); dv holds D v_ic */
        double axis[3];
        orc_srd_axis(p, step, (uint32_t)c, axis);
        for (int64_t k = 0; k < nt; ++k) {
          double vic[3], rot[3];
          for (int a = 0; a < 3; ++a) vic[a] = vk[3 * k + a] - vcm[a];
          orc_rotate(axis, alpha, vic, rot);
          for (int a = 0; a < 3; ++a) {
            dv[3 * k + a] = rot[a];
            wk[3 * k + a] = vic[a] - rot[a];
          }
        }
      }
      double omega[3], rcm[3];
      flags |= orc_cell_omega(nt, rk, wk, omega, rcm, sens_out ? sk : NULL);
      for (int64_t k = 0; k < n; ++k) {
        int64_t i = mem[k];
        double r[3], wxr[3];
        for (int a = 0; a < 3; ++a) r[a] = rk[3 * k + a] - rcm[a];
        cross3(omega, r, wxr);
        for (int a = 0; a < 3; ++a) {
          if (p->variant == ORC_AT_A)
            vnew[3 * i + a] = vcm[a] + dv[3 * k + a] - vrm[a] + wxr[a];
          else
            vnew[3 * i + a] = vcm[a] + dv[3 * k + a] + wxr[a];
        }
        if (sens_out) sens_out[i] = sk[k];
      }
      free(rk); free(vk); free(ran); free(wk); free(dv); free(sk);
    }
    if (cell_flags) cell_flags[c] = (uint8_t)flags;
  }

  /* 5. write back, observables */
  double P[3] = {0, 0, 0}, sumsq = 0.0, skin[3] = {0, 0, 0}, scol[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    const double* v = vnew + 3 * i;
    const double* u = vb + 3 * i;
    const double* r = rho + 3 * i;
    for (int a = 0; a < 3; ++a) {
      V[a * N + i] = v[a];
      P[a] += m * v[a];
    }
    sumsq += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    skin[0] += u[0] * u[1];
    skin[1] += u[1] * u[2];
    skin[2] += u[2] * u[0];
    double dvx = v[0] - u[0], dvy = v[1] - u[1], dvz = v[2] - u[2];
    scol[0] += dvx * r[1];  /* xy */
    scol[1] += dvy * r[0];  /* yx */
    scol[2] += dvy * r[2];  /* yz */
    scol[3] += dvz * r[1];  /* zy */
    scol[4] += dvz * r[0];  /* zx */
    scol[5] += dvx * r[2];  /* xz */
    if (cell_out) cell_out[i] = cell[i];
    if (vpre_out)
      for (int a = 0; a < 3; ++a) vpre_out[a * N + i] = u[a];
  }
  if (obs_out) {
    for (int k = 0; k < ORC_OBS_COUNT; ++k) obs_out[k] = 0.0;
    for (int a = 0; a < 3; ++a) obs_out[ORC_OBS_PX + a] = P[a];
    obs_out[ORC_OBS_EKIN] = 0.5 * m * sumsq;
    double mean2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double mv = (N > 0) ? P[a] / (m * (double)N) : 0.0;
      mean2 += mv * mv;
    }
    obs_out[ORC_OBS_TEMP] =
        (N > 1) ? m * (sumsq - (double)N * mean2) / (3.0 * (double)(N - 1)) : 0.0;
    for (int k = 0; k < 3; ++k) obs_out[ORC_OBS_SKIN_XY + k] = -m * skin[k] / fluid_volume;
    for (int k = 0; k < 6; ++k) obs_out[ORC_OBS_SCOL_XY + k] = -m * scol[k] / (fluid_volume * p->h);
  }

  free(cell); free(rho); free(vb); free(start); free(members); free(fill); free(vnew);
  return 0;
}

double orc_min_eigenvalue_sym3(const double A[9]) {
  double M[3][3] = {{A[0], A[1], A[2]}, {A[3], A[4], A[5]}, {A[6], A[7], A[8]}};
  return min_eigenvalue_sym3(M);
}

double orc_max_eigenvalue_sym3(const double A[9]) {
  double M[3][3] = {{A[0], A[1], A[2]}, {A[3], A[4], A[5]}, {A[6], A[7], A[8]}};
  double lo, hi;
  eigen_extremes_sym3(M, &lo, &hi);
  return hi;
}

/* ------------------------------------------------------------------------------ */
/* sampler access for distribution pins */

void orc_sample_normal(uint64_t seed, int64_t n, double* out) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.seed = seed;
  for (int64_t i = 0; i < n; i += 2) {
    uint32_t r[4];
    draw(&p, (uint32_t)(i / 2), 0u, TAG_TEST, 0u, r);
    double z0, z1;
    box_muller(uniform01(r[0]), uniform01(r[1]), &z0, &z1);
    out[i] = z0;
    if (i + 1 < n) out[i + 1] = z1;
  }
}

void orc_sample_gamma(uint64_t seed, double shape, int64_t n, double* out) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.seed = seed;
  for (int64_t i = 0; i < n; ++i) out[i] = gamma_mt(&p, (uint32_t)i, 1u, TAG_TEST, shape, NULL);
}

void orc_sample_poisson(uint64_t seed, double lambda, int64_t n, int32_t* out) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.seed = seed;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t r[4];
    draw(&p, (uint32_t)i, 2u, TAG_TEST, 0u, r);
    out[i] = poisson_inv(uniform01(r[0]), lambda, NULL);
  }
}
