/*
 * Plain FP64 CPU oracle of the D2Q9 MRT pseudopotential LBM with fluid-solid
 * interaction (Li, Luo, Kang & Chen, "Contact angles in the pseudopotential
 * lattice Boltzmann modeling of wetting", Sec. II and Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the CUDA library.
 *
 * One time step, in the paper's order:
 *   1. rho = sum_alpha f_alpha                              Eq. (6)
 *   2. psi = sqrt(2 (p_EOS - rho cs^2) / (G c^2))            Sec. II.B, Eq. (15)
 *   3. psi on solid nodes next to fluid (ghost layer)        Sec. III.A
 *   4. F_m = -G psi(x) sum_alpha w_alpha psi(x+e_alpha) e    Eq. (7)
 *   5. F_ads (density / psi / modified psi based)            Eqs. (10), (11), (14)
 *   6. F = F_m + F_ads,  rho v = sum_alpha e f + F/2         Eq. (6)
 *   7. m = M f, m_eq, S, m* = m - Lambda (m - m_eq) + (I - Lambda/2) S,
 *      f* = M^-1 m*                                          Eqs. (2)-(4), (9)
 *   8. f_alpha(x + e_alpha, t + 1) = f*_alpha(x, t)          Eq. (5)
 *   9. unknown populations at wall nodes                     Sec. III.A
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   - lattice numbering: e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 *     e6=(-1,1) e7=(-1,-1) e8=(1,-1); it is the numbering under which the
 *     wall rule of Sec. III.A gives zero momentum at the wall node.
 *   - the lattice is periodic in x and y; walls are rows of solid nodes.
 *   - omega_alpha of Eqs. (10), (11), (14): the text gives cs^2 w_alpha,
 *     but the G_w -> theta pairs printed with Figs. 2 and 4 are reproduced
 *     with omega_alpha = w_alpha (3x stronger); both are selectable.
 *   - G_w may vary from solid node to solid node; F_ads then reads G_w at
 *     the solid neighbour x + e_alpha.  A uniform G_w is Eqs. (10)/(11)/(14).
 *   - the wall rule uses F(x, t), the force of the same node's collision in
 *     the same step; the top wall uses the rule mirrored in y.
 *   - ghost psi: COPY takes psi of the fluid node next to the solid node
 *     along the wall normal, MIRROR the node two rows away, ZERO uses 0;
 *     SKIP does not apply Eq. (7) at fluid nodes touching solid (Sec. III.B:
 *     rough surfaces without a ghost layer); MEAN takes the mean psi of the
 *     fluid nodes next to the solid node along the axes, COPY extended to
 *     walls of any shape (a ghost layer below rough surfaces, Sec. III.B).
 *   - tau_nu varies linearly with rho between rho_V and rho_L (clamped)
 *     when the liquid and vapour values differ (Sec. III.C); the option
 *     ORC_VISC_MU makes the dynamic viscosity rho nu linear in rho instead.
 *   - M is the orthogonal D2Q9 basis whose rows give the equilibria of
 *     Eq. (3): 1, -4+3|e|^2, 4-21|e|^2/2+9|e|^4/2, e_x, (3|e|^2-5)e_x,
 *     e_y, (3|e|^2-5)e_y, e_x^2-e_y^2, e_x e_y.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

static const int ex[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int opp[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* weights of the equilibrium (D2Q9 lattice) */
static const double w_eq[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double cs2 = 1.0 / 3.0;

struct oracle_lbm {
  int nx, ny, fsi;
  oracle_params p;
  uint8_t* s;  /* switch function s(x): 1 solid, 0 fluid */
  double* gw;  /* G_w on solid nodes */
  double *f, *fnew, *fstar;
  double *rho, *psi, *Fmx, *Fmy, *Fx, *Fy, *vx, *vy;
  double M[Q * Q], Minv[Q * Q];
  long t;
};

static int g_threads = 1;
void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }

static inline int wrap(int a, int n) { return ((a % n) + n) % n; }
static inline size_t nid(const oracle_lbm* o, int x, int y) {
  return (size_t)wrap(y, o->ny) * o->nx + wrap(x, o->nx);
}
static inline double* fa(double* f, const oracle_lbm* o, int a) {
  return f + (size_t)a * o->nx * o->ny;
}

/* ---------------- Eq. (15) and the pseudopotential ---------------- */
double oracle_p_eos(const oracle_params* p, double rho) {
  if (p->eos == ORC_EOS_CS) {
    /* Carnahan-Starling: hard-sphere repulsion and van der Waals attraction */
    const double e = p->cs_b * rho / 4.0;
    return rho * p->cs_R * p->cs_T * (1.0 + e + e * e - e * e * e) / ((1.0 - e) * (1.0 - e) * (1.0 - e)) -
           p->cs_a * rho * rho;
  }
  const double thV = p->kV * cs2, thM = p->kM * cs2, thL = p->kL * cs2;
  if (rho <= p->rho_1) return rho * thV;
  if (rho <= p->rho_2) return p->rho_1 * thV + (rho - p->rho_1) * thM;
  return p->rho_1 * thV + (p->rho_2 - p->rho_1) * thM + (rho - p->rho_2) * thL;
}

double oracle_psi(const oracle_params* p, double rho) {
  const double c = 1.0;
  return sqrt(2.0 * (oracle_p_eos(p, rho) - rho * cs2) / (p->G * c * c));
}

/* ---------------- transformation matrix ---------------- */
static void invert9(const double* A, double* Ainv) {
  double a[Q][2 * Q];
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < 2 * Q; ++j) a[i][j] = j < Q ? A[i * Q + j] : (j - Q == i ? 1.0 : 0.0);
  for (int c = 0; c < Q; ++c) {
    int piv = c;
    for (int r = c + 1; r < Q; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 2 * Q; ++j) {
        double tmp = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = tmp;
      }
    double d = a[c][c];
    for (int j = 0; j < 2 * Q; ++j) a[c][j] /= d;
    for (int r = 0; r < Q; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      if (m == 0.0) continue;
      for (int j = 0; j < 2 * Q; ++j) a[r][j] -= m * a[c][j];
    }
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) Ainv[i * Q + j] = a[i][j + Q];
}

void oracle_mrt_matrices(double* M, double* Minv) {
  for (int a = 0; a < Q; ++a) {
    double e2 = (double)(ex[a] * ex[a] + ey[a] * ey[a]);
    double row[Q] = {1.0,
                     -4.0 + 3.0 * e2,
                     4.0 - 10.5 * e2 + 4.5 * e2 * e2,
                     (double)ex[a],
                     (3.0 * e2 - 5.0) * ex[a],
                     (double)ey[a],
                     (3.0 * e2 - 5.0) * ey[a],
                     (double)(ex[a] * ex[a] - ey[a] * ey[a]),
                     (double)(ex[a] * ey[a])};
    for (int k = 0; k < Q; ++k) M[k * Q + a] = row[k];
  }
  invert9(M, Minv);
}

/* ---------------- creation ---------------- */
static int mask_rows_flat(int nx, int ny, const uint8_t* s) {
  for (int y = 0; y < ny; ++y)
    for (int x = 1; x < nx; ++x)
      if ((s[(size_t)y * nx + x] != 0) != (s[(size_t)y * nx] != 0)) return 0;
  return 1;
}

oracle_lbm* oracle_create(int nx, int ny, const oracle_params* p, const uint8_t* solid, int fsi,
                          const double* gw_field, double gw_uniform) {
  if (nx < 1 || ny < 3 || !p || fsi < 0 || fsi > 2) return NULL;
  const int flat = p->wall == ORC_WALL_NEQ || p->ghost == ORC_GHOST_COPY ||
                   p->ghost == ORC_GHOST_MIRROR;
  if (flat) {
    /* the wall rule of Sec. III.A and the ghost layer are defined for flat walls */
    if (solid && !mask_rows_flat(nx, ny, solid)) return NULL;
  }
  oracle_lbm* o = (oracle_lbm*)calloc(1, sizeof(oracle_lbm));
  size_t N = (size_t)nx * ny;
  o->nx = nx;
  o->ny = ny;
  o->fsi = fsi;
  o->p = *p;
  o->s = (uint8_t*)calloc(N, 1);
  o->gw = (double*)calloc(N, sizeof(double));
  o->f = (double*)calloc(Q * N, sizeof(double));
  o->fnew = (double*)calloc(Q * N, sizeof(double));
  o->fstar = (double*)calloc(Q * N, sizeof(double));
  double** fields[] = {&o->rho, &o->psi, &o->Fmx, &o->Fmy, &o->Fx, &o->Fy, &o->vx, &o->vy};
  for (int i = 0; i < 8; ++i) *fields[i] = (double*)calloc(N, sizeof(double));
  for (size_t i = 0; i < N; ++i) {
    o->s[i] = solid ? (solid[i] != 0) : 0;
    o->gw[i] = o->s[i] ? (gw_field ? gw_field[i] : gw_uniform) : 0.0;
  }
  if (flat) {
    /* a fluid node may not have solid both directly above and below */
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        if (!o->s[nid(o, x, y)] && o->s[nid(o, x, y - 1)] && o->s[nid(o, x, y + 1)]) {
          oracle_destroy(o);
          return NULL;
        }
  }
  oracle_mrt_matrices(o->M, o->Minv);
  o->t = 0;
  return o;
}

void oracle_destroy(oracle_lbm* o) {
  if (!o) return;
  free(o->s);
  free(o->gw);
  free(o->f);
  free(o->fnew);
  free(o->fstar);
  free(o->rho);
  free(o->psi);
  free(o->Fmx);
  free(o->Fmy);
  free(o->Fx);
  free(o->Fy);
  free(o->vx);
  free(o->vy);
  free(o);
}

long oracle_time(const oracle_lbm* o) { return o->t; }

int oracle_set_density(oracle_lbm* o, const double* rho) {
  for (int a = 0; a < Q; ++a)
    for (int y = 0; y < o->ny; ++y)
      for (int x = 0; x < o->nx; ++x) {
        size_t i = nid(o, x, y);
        fa(o->f, o, a)[i] = o->s[i] ? 0.0 : w_eq[a] * rho[i];
      }
  o->t = 0;
  return 0;
}

int oracle_init_droplet(oracle_lbm* o, double x0, double y0, double R, double width) {
  const double rl = o->p.rho_L, rv = o->p.rho_V;
  size_t N = (size_t)o->nx * o->ny;
  double* rho = (double*)malloc(N * sizeof(double));
  for (int y = 0; y < o->ny; ++y)
    for (int x = 0; x < o->nx; ++x) {
      double dx = (double)x - x0;
      /* minimum image in the periodic x direction */
      dx -= o->nx * floor(dx / o->nx + 0.5);
      double dy = (double)y - y0;
      double r = sqrt(dx * dx + dy * dy);
      rho[(size_t)y * o->nx + x] = rv + 0.5 * (rl - rv) * (1.0 - tanh(2.0 * (r - R) / width));
    }
  oracle_set_density(o, rho);
  free(rho);
  return 0;
}

/* ---------------- steps 1-6: macroscopic quantities and forces ---------------- */
static void macroscopic(oracle_lbm* o) {
  const int nx = o->nx, ny = o->ny;
  const oracle_params* p = &o->p;
  /* 1-2: density and pseudopotential on fluid nodes */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (o->s[i]) {
        o->rho[i] = 0.0;
        continue;
      }
      double r = 0.0;
      for (int a = 0; a < Q; ++a) r += fa(o->f, o, a)[i];
      o->rho[i] = r;
      o->psi[i] = oracle_psi(p, r);
    }
  /* 3: ghost pseudopotential on solid nodes */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (!o->s[i]) continue;
      double g = 0.0;
      int up = !o->s[nid(o, x, y + 1)], dn = !o->s[nid(o, x, y - 1)];
      if (p->ghost == ORC_GHOST_COPY) {
        if (up) g = o->psi[nid(o, x, y + 1)];
        else if (dn) g = o->psi[nid(o, x, y - 1)];
      } else if (p->ghost == ORC_GHOST_MIRROR) {
        if (up) g = o->psi[nid(o, x, y + 2)];
        else if (dn) g = o->psi[nid(o, x, y - 2)];
      } else if (p->ghost == ORC_GHOST_MEAN) {
        /* any wall shape: the mean psi of the fluid nodes next to the solid
           node along the axes (up, down, right, left); on a flat wall this
           is COPY */
        const int gx[4] = {0, 0, 1, -1}, gy[4] = {1, -1, 0, 0};
        double sum = 0.0;
        int n = 0;
        for (int k = 0; k < 4; ++k) {
          size_t j = nid(o, x + gx[k], y + gy[k]);
          if (!o->s[j]) {
            sum += o->psi[j];
            ++n;
          }
        }
        if (n > 0) g = sum / n;
      }
      o->psi[i] = g;
    }
  /* 4-6: F_m (Eq. 7), F_ads (Eqs. 10, 11, 14), F and v (Eq. 6) */
  const double wF[Q] = {0.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0,
                        1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (o->s[i]) {
        o->Fmx[i] = o->Fmy[i] = o->Fx[i] = o->Fy[i] = o->vx[i] = o->vy[i] = 0.0;
        continue;
      }
      double sx = 0.0, sy = 0.0, ax = 0.0, ay = 0.0;
      for (int a = 1; a < Q; ++a) {
        size_t j = nid(o, x + ex[a], y + ey[a]);
        sx += wF[a] * o->psi[j] * ex[a];
        sy += wF[a] * o->psi[j] * ey[a];
        /* omega_alpha (see ORC_OMEGA_*); s(x + e_alpha) switches the solid on */
        double omega = (p->omega == ORC_OMEGA_CS2W ? cs2 : 1.0) * wF[a];
        ax += omega * o->gw[j] * (double)o->s[j] * ex[a];
        ay += omega * o->gw[j] * (double)o->s[j] * ey[a];
      }
      double Fmx = -p->G * o->psi[i] * sx;
      double Fmy = -p->G * o->psi[i] * sy;
      if (p->ghost == ORC_GHOST_SKIP) {
        /* Eq. (7) not applied next to the wall (Sec. III.B) */
        int touches = 0;
        for (int a = 1; a < Q; ++a) touches |= o->s[nid(o, x + ex[a], y + ey[a])];
        if (touches) Fmx = Fmy = 0.0;
      }
      double X;
      if (o->fsi == ORC_FSI_DENSITY) X = o->rho[i];                       /* Eq. (10) */
      else if (o->fsi == ORC_FSI_PSI) X = o->psi[i];                      /* Eq. (11) */
      else X = o->psi[i] * o->psi[i]; /* Eq. (14), phi(x) = psi(x) */
      double Fadsx = -X * ax, Fadsy = -X * ay;
      double Fx = Fmx + Fadsx, Fy = Fmy + Fadsy;
      double jx = 0.0, jy = 0.0;
      for (int a = 0; a < Q; ++a) {
        jx += ex[a] * fa(o->f, o, a)[i];
        jy += ey[a] * fa(o->f, o, a)[i];
      }
      o->Fmx[i] = Fmx;
      o->Fmy[i] = Fmy;
      o->Fx[i] = Fx;
      o->Fy[i] = Fy;
      o->vx[i] = (jx + 0.5 * Fx) / o->rho[i];
      o->vy[i] = (jy + 0.5 * Fy) / o->rho[i];
    }
}

static double tau_nu_of(const oracle_params* p, double rho) {
  if (p->tau_nu_L == p->tau_nu_V) return p->tau_nu_L;
  const double frac = (rho - p->rho_V) / (p->rho_L - p->rho_V);
  double t;
  if (p->visc == ORC_VISC_MU) {
    /* mu = rho nu linear in rho, nu = (tau - 1/2) cs^2 */
    const double muV = p->rho_V * (p->tau_nu_V - 0.5) * cs2;
    const double muL = p->rho_L * (p->tau_nu_L - 0.5) * cs2;
    t = 0.5 + (muV + frac * (muL - muV)) / rho / cs2;
  } else {
    t = p->tau_nu_V + frac * (p->tau_nu_L - p->tau_nu_V);
  }
  double lo = p->tau_nu_L < p->tau_nu_V ? p->tau_nu_L : p->tau_nu_V;
  double hi = p->tau_nu_L < p->tau_nu_V ? p->tau_nu_V : p->tau_nu_L;
  return t < lo ? lo : (t > hi ? hi : t);
}

/* ---------------- step 7: MRT collision with the forcing of Eq. (9) ---------------- */
static void collide(oracle_lbm* o) {
  const int nx = o->nx, ny = o->ny;
  const oracle_params* p = &o->p;
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (o->s[i]) continue;
      double f[Q], m[Q], meq[Q], S[Q], L[Q], ms[Q];
      for (int a = 0; a < Q; ++a) f[a] = fa(o->f, o, a)[i];
      for (int k = 0; k < Q; ++k) {
        m[k] = 0.0;
        for (int a = 0; a < Q; ++a) m[k] += o->M[k * Q + a] * f[a];
      }
      const double rho = o->rho[i], vx = o->vx[i], vy = o->vy[i];
      const double Fx = o->Fx[i], Fy = o->Fy[i];
      const double v2 = vx * vx + vy * vy;
      /* Eq. (3) */
      meq[0] = rho;
      meq[1] = rho * (-2.0 + 3.0 * v2);
      meq[2] = rho * (1.0 - 3.0 * v2);
      meq[3] = rho * vx;
      meq[4] = -rho * vx;
      meq[5] = rho * vy;
      meq[6] = -rho * vy;
      meq[7] = rho * (vx * vx - vy * vy);
      meq[8] = rho * vx * vy;
      /* Eq. (2) */
      const double tau_nu = tau_nu_of(p, rho);
      L[0] = 1.0 / p->tau_rho;
      L[1] = 1.0 / p->tau_e;
      L[2] = 1.0 / p->tau_zeta;
      L[3] = 1.0 / p->tau_j;
      L[4] = 1.0 / p->tau_q;
      L[5] = 1.0 / p->tau_j;
      L[6] = 1.0 / p->tau_q;
      L[7] = 1.0 / tau_nu;
      L[8] = 1.0 / tau_nu;
      /* Eq. (9), delta_t = 1 */
      const double Fm2 = o->Fmx[i] * o->Fmx[i] + o->Fmy[i] * o->Fmy[i];
      const double psi2 = o->psi[i] * o->psi[i];
      const double vF = vx * Fx + vy * Fy;
      S[0] = 0.0;
      S[1] = 6.0 * vF + 12.0 * p->sigma * Fm2 / (psi2 * (p->tau_e - 0.5));
      S[2] = -6.0 * vF - 12.0 * p->sigma * Fm2 / (psi2 * (p->tau_zeta - 0.5));
      S[3] = Fx;
      S[4] = -Fx;
      S[5] = Fy;
      S[6] = -Fy;
      S[7] = 2.0 * (vx * Fx - vy * Fy);
      S[8] = vx * Fy + vy * Fx;
      /* Eq. (4) */
      for (int k = 0; k < Q; ++k) ms[k] = m[k] - L[k] * (m[k] - meq[k]) + (1.0 - 0.5 * L[k]) * S[k];
      /* f* = M^-1 m* */
      for (int a = 0; a < Q; ++a) {
        double v = 0.0;
        for (int k = 0; k < Q; ++k) v += o->Minv[a * Q + k] * ms[k];
        fa(o->fstar, o, a)[i] = v;
      }
    }
}

/* ---------------- steps 8-9: streaming (Eq. 5) and the walls ---------------- */
static void stream_and_walls(oracle_lbm* o) {
  const int nx = o->nx, ny = o->ny;
  const size_t N = (size_t)nx * ny;
  for (size_t k = 0; k < Q * N; ++k) o->fnew[k] = 0.0;
  for (int a = 0; a < Q; ++a)
    for (size_t i = 0; i < N; ++i)
      if (!o->s[i]) fa(o->fnew, o, a)[i] = NAN; /* every fluid entry must be written */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (o->s[i]) continue;
      for (int a = 0; a < Q; ++a) {
        size_t j = nid(o, x + ex[a], y + ey[a]);
        if (!o->s[j]) fa(o->fnew, o, a)[j] = fa(o->fstar, o, a)[i];
        else if (o->p.wall == ORC_WALL_BB) fa(o->fnew, o, opp[a])[i] = fa(o->fstar, o, a)[i];
      }
    }
  if (o->p.wall == ORC_WALL_NEQ) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t i = (size_t)y * nx + x;
        if (o->s[i]) continue;
        double* g[Q];
        for (int a = 0; a < Q; ++a) g[a] = fa(o->fnew, o, a) + i;
        const double Fx = o->Fx[i], Fy = o->Fy[i];
        if (o->s[nid(o, x, y - 1)]) { /* solid below: the rule of Sec. III.A */
          *g[2] = *g[4];
          *g[5] = *g[7] - 0.5 * (*g[1] - *g[3]) - 0.25 * (Fx + Fy);
          *g[6] = *g[8] + 0.5 * (*g[1] - *g[3]) + 0.25 * (Fx - Fy);
        } else if (o->s[nid(o, x, y + 1)]) { /* solid above: the same rule mirrored in y */
          *g[4] = *g[2];
          *g[8] = *g[6] - 0.5 * (*g[1] - *g[3]) - 0.25 * (Fx - Fy);
          *g[7] = *g[5] + 0.5 * (*g[1] - *g[3]) + 0.25 * (Fx + Fy);
        }
      }
  }
  double* tmp = o->f;
  o->f = o->fnew;
  o->fnew = tmp;
}

void oracle_step(oracle_lbm* o, long n) {
  for (long k = 0; k < n; ++k) {
    macroscopic(o);
    collide(o);
    stream_and_walls(o);
    o->t += 1;
  }
}

void oracle_get_fields(oracle_lbm* o, double* rho, double* ux, double* uy, double* Fx, double* Fy,
                       double* psi) {
  macroscopic(o);
  size_t N = (size_t)o->nx * o->ny;
  for (size_t i = 0; i < N; ++i) {
    if (rho) rho[i] = o->rho[i];
    if (ux) ux[i] = o->vx[i];
    if (uy) uy[i] = o->vy[i];
    if (Fx) Fx[i] = o->Fx[i];
    if (Fy) Fy[i] = o->Fy[i];
    if (psi) psi[i] = o->psi[i];
  }
}

void oracle_get_populations(const oracle_lbm* o, double* f) {
  memcpy(f, o->f, sizeof(double) * Q * o->nx * o->ny);
}

void oracle_set_populations(oracle_lbm* o, const double* f, const double* unused_x,
                            const double* unused_y) {
  (void)unused_x;
  (void)unused_y;
  memcpy(o->f, f, sizeof(double) * Q * o->nx * o->ny);
}

/* ---------------- diagnostics and the contact angle ---------------- */
/* Spreading radius of a droplet on a wall (dynamic wetting, Sec. III.A and
 * Fig. 7): on node row `row`, starting at the column nearest x_ref, the
 * first node on the right and on the left whose density is below `level`
 * (solid nodes count as 0); the level crossing lies between it and the
 * previous node, by linear interpolation.  The radius is half the distance
 * between the two crossings; 0 if the start node is below the level, nx/2 if
 * no node of the row is. */
double oracle_contact_radius(int nx, int ny, const double* rho, const uint8_t* solid, int row,
                             double level, double x_ref) {
  (void)ny;
  const double* r = rho + (size_t)row * nx;
  const uint8_t* s = solid ? solid + (size_t)row * nx : NULL;
  int x0 = (int)floor(x_ref + 0.5);
  x0 = ((x0 % nx) + nx) % nx;
#define RHO_AT(x) ((s && s[x]) ? 0.0 : r[x])
  if (!(RHO_AT(x0) >= level)) return 0.0;
  double right = -1.0, left = -1.0;
  for (int d = 1; d <= nx && right < 0.0; ++d) {
    const int xb = (x0 + d) % nx, xa = (x0 + d - 1) % nx;
    if (RHO_AT(xb) < level) right = (d - 1) + (level - RHO_AT(xa)) / (RHO_AT(xb) - RHO_AT(xa));
  }
  for (int d = 1; d <= nx && left < 0.0; ++d) {
    const int xb = ((x0 - d) % nx + nx) % nx, xa = ((x0 - d + 1) % nx + nx) % nx;
    if (RHO_AT(xb) < level) left = (d - 1) + (level - RHO_AT(xa)) / (RHO_AT(xb) - RHO_AT(xa));
  }
#undef RHO_AT
  if (right < 0.0 || left < 0.0) return 0.5 * nx;
  return 0.5 * (right + left);
}

/* Level-set points of rho = level on grid edges between fluid nodes, linear
 * interpolation; x unwrapped about x_ref; points closer than d_min to the wall
 * height y_w dropped; Kasa circle fit x^2 + y^2 + D x + E y + F = 0 by least
 * squares (3x3 normal equations); theta = 90 deg + asin((y_c - y_w) / R). */
int oracle_contact_angle(int nx, int ny, const double* rho, const uint8_t* s, double level,
                         double y_w, double x_ref, double d_min, oracle_diag* d) {
  double A[3][3] = {{0}}, b[3] = {0};
  int n = 0;
  double* px = (double*)malloc(sizeof(double) * 2 * (size_t)nx * ny + 1);
  double* py = (double*)malloc(sizeof(double) * 2 * (size_t)nx * ny + 1);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t i = (size_t)y * nx + x;
      if (s && s[i]) continue;
      for (int dir = 0; dir < 2; ++dir) {
        int x2 = dir == 0 ? x + 1 : x, y2 = dir == 0 ? y : y + 1;
        if (dir == 1 && y2 >= ny) continue; /* no vertical crossing through the y seam */
        size_t j = (size_t)y2 * nx + (x2 % nx);
        if (s && s[j]) continue;
        double ra = rho[i], rb = rho[j];
        if ((ra >= level) == (rb >= level)) continue;
        double t = (level - ra) / (rb - ra);
        double X = (double)x + t * (double)(x2 - x) - x_ref;
        X -= nx * floor(X / nx + 0.5);
        double Y = (double)y + t * (double)(y2 - y) - y_w;
        if (Y < d_min) continue;
        px[n] = X;
        py[n] = Y;
        ++n;
      }
    }
  for (int k = 0; k < n; ++k) {
    double X = px[k], Y = py[k], r2 = X * X + Y * Y;
    double row[3] = {X, Y, 1.0};
    for (int a = 0; a < 3; ++a) {
      for (int c = 0; c < 3; ++c) A[a][c] += row[a] * row[c];
      b[a] -= row[a] * r2;
    }
  }
  d->n_contour = n;
  if (n < 3) {
    d->theta_deg = NAN;
    d->fit_rms = NAN;
    d->xc = d->yc = d->radius = NAN;
    free(px);
    free(py);
    return 2;
  }
  /* solve the 3x3 normal equations by Cramer's rule */
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  double sol[3];
  for (int c = 0; c < 3; ++c) {
    double B[3][3];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) B[r][k] = (k == c) ? b[r] : A[r][k];
    sol[c] = (B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
              B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
              B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0])) /
             det;
  }
  double xc = -0.5 * sol[0], yc = -0.5 * sol[1];
  double R = sqrt(xc * xc + yc * yc - sol[2]);
  double ratio = yc / R;
  if (ratio > 1.0) ratio = 1.0;
  if (ratio < -1.0) ratio = -1.0;
  d->theta_deg = 90.0 + asin(ratio) * 180.0 / M_PI;
  double ss = 0.0;
  for (int k = 0; k < n; ++k) {
    double dr = sqrt((px[k] - xc) * (px[k] - xc) + (py[k] - yc) * (py[k] - yc)) - R;
    ss += dr * dr;
  }
  d->fit_rms = sqrt(ss / n);
  d->xc = xc + x_ref;
  d->yc = yc + y_w;
  d->radius = R;
  free(px);
  free(py);
  return 0;
}

int oracle_diagnostics(oracle_lbm* o, double y_w, double x_ref, double d_min, oracle_diag* d) {
  macroscopic(o);
  size_t N = (size_t)o->nx * o->ny;
  double mass = 0.0, rmax = -INFINITY, rmin = INFINITY, umax = 0.0;
  int bad = 0;
  for (size_t i = 0; i < N; ++i) {
    if (o->s[i]) continue;
    double r = o->rho[i];
    if (!isfinite(r) || r <= 0.0) bad = 1;
    mass += r;
    if (r > rmax) rmax = r;
    if (r < rmin) rmin = r;
    double u = sqrt(o->vx[i] * o->vx[i] + o->vy[i] * o->vy[i]);
    if (!isfinite(u)) bad = 1;
    if (u > umax) umax = u;
  }
  d->step = o->t;
  d->mass = mass;
  d->rho_max = rmax;
  d->rho_min = rmin;
  d->u_max = umax;
  int st = oracle_contact_angle(o->nx, o->ny, o->rho, o->s, 0.5 * (o->p.rho_L + o->p.rho_V), y_w,
                                x_ref, d_min, d);
  d->status = bad ? 1 : st;
  return d->status;
}
