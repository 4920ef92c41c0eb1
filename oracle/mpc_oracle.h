/*
 * Oracle for one multiparticle-collision-dynamics (MPC) step: plain, single-threaded,
 * FP64 C.  TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library; the product path never does.
 * It shares no code with the CUDA implementation: both follow the same written
 * contract (fixed-point positions, Philox keying), each in its own code.
 *
 * Paper: Westphal, Goh, Winkler, Gompper, "HTMPC", arXiv 2406.15236,
 *   Sec. II Eq. (1)  streaming,            Eq. (2) SRD collision,
 *   Sec. II Eqs.(3)-(4) SRD+a (angular-momentum conservation),
 *   Sec. II Eqs.(5)-(7) Maxwell-Boltzmann-scaling thermostat,
 *   Sec. II "Boundary conditions" (bounce-back walls, phantom particles),
 *   Sec. II "External fields" (gravity), Sec. III.A.3 permanent reorder.
 * MPC-AT+a follows the reference the paper cites for angular-momentum-conserving
 * MPC (Noguchi, Kikuchi, Gompper 2007).
 */
#ifndef MPC_ORACLE_H
#define MPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SRD = 0, ORC_AT_A = 1, ORC_SRD_A = 2 };

typedef struct {
  int32_t L[3];          /* box edge in collision cells (a = 1) */
  double n_c;            /* mean particles per cell */
  double h;              /* time step */
  double alpha_deg;      /* SRD rotation angle */
  double kT;             /* thermal energy */
  double m;              /* particle mass */
  int32_t variant;       /* ORC_SRD / ORC_AT_A / ORC_SRD_A */
  int32_t thermostat;    /* 1: MBS after SRD */
  int32_t walls_z;       /* walls at z = 0 and z = Lz: 0 none (periodic), 1 no-slip
                            (bounce-back + phantom particles), 2 slip (specular) */
  double g[3];           /* body-force acceleration */
  uint64_t seed;
  uint32_t box;          /* fourth Philox counter word */
  double wall_u[2];      /* x velocity of the no-slip wall at z = 0 and at z = Lz */
} orc_params;

/* per-cell flags written by orc_step */
enum {
  ORC_FLAG_MBS_NEAR_TIE = 1,   /* a Marsaglia-Tsang decision was within 1e-5 of its threshold */
  ORC_FLAG_POISSON_NEAR_TIE = 2,
  /* angular-momentum solve that float32 arithmetic cannot take to the 1e-5 velocity bar;
   * there the float32 result is good only to its first-order sensitivity (sens_out):
   * (a) n >= 3 and cond(J) = lambda_max / lambda_min > ORC_COND_FLOAT32.  A float32 solve
   *     rounds the entries of J by a relative u = 2^-24; that moves omega by ~u cond
   *     |omega|, and where L points along the weak axis omega itself grows like cond, so
   *     a member's velocity error grows like u cond^2 |L| |r| / lambda_max (about
   *     1e-7 cond^2 / sqrt(n) in unit-temperature cells): near 1e-5 at cond = 20 (a
   *     float32 kernel measured 1.2e-5 in a cell of cond 19.3), a quarter of that at the
   *     threshold 10.  About 0.5 % of the cells at N_c = 10.
   * (b) n >= 2 members within ORC_TIGHT_RMS (rms) of their centre of mass.  Positions
   *     relative to the cell hold an absolute precision of u a; a cluster of radius
   *     0.05 a is resolved only to 20 u, which omega (growing like 1/radius) carries
   *     past 1e-5.  Never seen in a fluid at N_c >= 1; crafted states only. */
  ORC_FLAG_ILL_CONDITIONED = 4,
  ORC_FLAG_DEGENERATE = 8       /* n >= 3 but det(J) <= 0: omega set to zero */
};

#define ORC_COND_FLOAT32 10.0
#define ORC_TIGHT_RMS 0.05

/* observables slots (orc_step obs_out, 16 doubles) */
enum {
  ORC_OBS_PX = 0, ORC_OBS_PY, ORC_OBS_PZ, ORC_OBS_EKIN, ORC_OBS_TEMP,
  ORC_OBS_SKIN_XY, ORC_OBS_SKIN_YZ, ORC_OBS_SKIN_ZX,
  ORC_OBS_SCOL_XY, ORC_OBS_SCOL_YX, ORC_OBS_SCOL_YZ, ORC_OBS_SCOL_ZY,
  ORC_OBS_SCOL_ZX, ORC_OBS_SCOL_XZ, ORC_OBS_COUNT = 16
};

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int orc_fixed_bits(const orc_params* p);
int64_t orc_num_particles(const orc_params* p);
int64_t orc_num_cells(const orc_params* p);
void orc_shift(const orc_params* p, int64_t step, uint32_t S[3]);

int orc_init(const orc_params* p, int64_t N, uint32_t* X, double* V, uint32_t* id);

int orc_step(const orc_params* p, int64_t N, uint32_t* X, double* V, const uint32_t* id,
             int64_t step, uint32_t* cell_out, uint32_t* count_out, double* vpre_out,
             double* obs_out, uint8_t* cell_flags, double* sens_out);

/* building blocks exposed for the pin tests */
int orc_cell_of(const orc_params* p, const uint32_t x[3], const uint32_t S[3],
                uint32_t* cell, double rho[3]);
void orc_srd_axis(const orc_params* p, int64_t step, uint32_t cell, double axis[3]);
void orc_rotate(const double axis[3], double alpha_rad, const double v[3], double out[3]);
void orc_stream_one(const orc_params* p, uint32_t x[3], double v[3]);
double orc_min_eigenvalue_sym3(const double A[9]);
double orc_max_eigenvalue_sym3(const double A[9]);
int orc_cell_omega(int64_t n, const double* rho, const double* w, double omega[3],
                   double rcm[3], double* sens);
int orc_phantoms(const orc_params* p, int64_t step, uint32_t cell, double phi, int wall,
                 double* nph, double P[3], double* Kint);
void orc_phantom_particles(const orc_params* p, int64_t step, uint32_t cell, uint32_t Sz, int wall,
                           int32_t k, double* rho, double* v, double* vran);
void orc_sample_normal(uint64_t seed, int64_t n, double* out);
void orc_sample_gamma(uint64_t seed, double shape, int64_t n, double* out);
void orc_sample_poisson(uint64_t seed, double lambda, int64_t n, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
