/*
 * Plain FP64 CPU oracle for the D2Q9 MRT pseudopotential lattice Boltzmann
 * step with fluid-solid interaction (Li, Luo, Kang & Chen, "Contact angles
 * in the pseudopotential lattice Boltzmann modeling of wetting").
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source, header, table or helper with
 * the CUDA library; its parameter structure below is its own.
 *
 * Arithmetic: IEEE FP64, built with -ffp-contract=off (no FMA contraction),
 * populations summed in the order alpha = 0..8, every node updated by the
 * same code whether the row loop runs on one thread or many.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_lbm oracle_lbm;

/* Fluid-solid interaction: Eq. (10), Eq. (11), Eq. (14). */
enum { ORC_FSI_DENSITY = 0, ORC_FSI_PSI = 1, ORC_FSI_MODIFIED = 2 };
/* Wall treatment: the on-node scheme of Sec. III.A, or halfway bounce-back. */
enum { ORC_WALL_NEQ = 0, ORC_WALL_BB = 1 };
/* Pseudopotential assigned to solid nodes when Eq. (7) is applied at walls;
   SKIP: Eq. (7) not applied at fluid nodes with a solid neighbour. */
enum { ORC_GHOST_COPY = 0, ORC_GHOST_MIRROR = 1, ORC_GHOST_ZERO = 2, ORC_GHOST_SKIP = 3,
       ORC_GHOST_MEAN = 4 };
/* Weights omega_alpha of the fluid-solid force, Eqs. (10), (11), (14).
   ORC_OMEGA_W: omega_alpha = w_alpha of Eq. (7) (1/3, 1/12); the G_w values
   printed with Figs. 2-4 give the printed angles under this choice.
   ORC_OMEGA_CS2W: omega_alpha = cs^2 w_alpha (1/9, 1/36), the sentence
   after Eq. (10) read literally. */
enum { ORC_OMEGA_W = 0, ORC_OMEGA_CS2W = 1 };
/* Equation of state: the piecewise-linear EOS of Eq. (15), or Carnahan-
   Starling, p = rho R T (1 + e + e^2 - e^3) / (1 - e)^3 - a rho^2 with
   e = b rho / 4 (an option: the paper uses Eq. (15) only). */
enum { ORC_EOS_PL = 0, ORC_EOS_CS = 1 };
/* tau_nu between the phases when tau_nu_L != tau_nu_V (Sec. III.C gives the
   two end values only).  ORC_VISC_TAU: tau_nu linear in rho (equivalently
   the kinematic viscosity nu = (tau_nu - 1/2) cs^2 linear in rho).
   ORC_VISC_MU: the dynamic viscosity mu = rho nu linear in rho,
   tau_nu = 1/2 + 3 mu(rho) / rho.  Both clamped to the two end values. */
enum { ORC_VISC_TAU = 0, ORC_VISC_MU = 1 };

typedef struct {
  /* Eq. (15): theta_V, theta_M, theta_L in units of cs^2, spinodal rho_1, rho_2 */
  double kV, kM, kL, rho_1, rho_2;
  double G;          /* interaction strength of Eq. (7) */
  double sigma;      /* Eq. (9) mechanical-stability parameter */
  /* relaxation times of Eq. (2): tau_rho, tau_e, tau_zeta, tau_j, tau_q */
  double tau_rho, tau_e, tau_zeta, tau_j, tau_q;
  /* tau_nu in the liquid and vapour phase; interpolated between rho_V and
     rho_L (clamped) when they differ, as `visc` says */
  double tau_nu_L, tau_nu_V, rho_L, rho_V;
  int wall, ghost, omega;
  int eos;                     /* ORC_EOS_* */
  double cs_a, cs_b, cs_R, cs_T; /* Carnahan-Starling constants */
  int visc;                    /* ORC_VISC_* */
} oracle_params;

typedef struct {
  long step;
  double mass, rho_max, rho_min, u_max;
  double theta_deg, fit_rms, xc, yc, radius;
  int n_contour;
  int status; /* 0 ok, 1 non-finite or non-positive density, 2 too few contour points */
} oracle_diag;

oracle_lbm* oracle_create(int nx, int ny, const oracle_params* p, const uint8_t* solid,
                          int fsi, const double* gw_field, double gw_uniform);
void oracle_destroy(oracle_lbm* o);
void oracle_set_threads(int n);
/* f_alpha = w_alpha rho (fluid at rest) from a density field [ny][nx] */
int oracle_set_density(oracle_lbm* o, const double* rho);
/* Sec. III.A initial droplet with a tanh interface of the given width */
int oracle_init_droplet(oracle_lbm* o, double x0, double y0, double R, double width);
void oracle_step(oracle_lbm* o, long n);
long oracle_time(const oracle_lbm* o);
/* rho, velocity of Eq. (6), total force F = F_m + F_ads [ny][nx] each; NULL skips */
void oracle_get_fields(oracle_lbm* o, double* rho, double* ux, double* uy, double* Fx,
                       double* Fy, double* psi);
/* populations f_alpha(x, t) after streaming and the wall rule, layout [9][ny][nx] */
void oracle_get_populations(const oracle_lbm* o, double* f);
void oracle_set_populations(oracle_lbm* o, const double* f, const double* F_prev_x,
                            const double* F_prev_y);
/* contact-angle measurement level (rho_L + rho_V)/2, wall height y_w, unwrap
   reference x_ref, points closer than d_min to the wall discarded */
int oracle_diagnostics(oracle_lbm* o, double y_w, double x_ref, double d_min, oracle_diag* d);
/* circle fit on an explicit density field (used by the adjoint loss) */
/* spreading (contact) radius along node row `row`, Sec. III.A / Fig. 7 */
double oracle_contact_radius(int nx, int ny, const double* rho, const uint8_t* solid, int row,
                             double level, double x_ref);
int oracle_contact_angle(int nx, int ny, const double* rho, const uint8_t* solid, double level,
                         double y_w, double x_ref, double d_min, oracle_diag* d);
/* the 9x9 transformation matrix M and its inverse, row-major */
void oracle_mrt_matrices(double* M, double* Minv);
/* Eq. (15) pressure and the pseudopotential psi of Sec. II.B */
double oracle_p_eos(const oracle_params* p, double rho);
double oracle_psi(const oracle_params* p, double rho);

#ifdef __cplusplus
}
#endif
#endif
