// C ABI of liblbm: context management, validation, host-side set-up of the
// per-node wall data, stepping and field read-back (declared in lbm.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <functional>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_diag.cuh"
#include "lbm_internal.cuh"

using namespace lbm;

static thread_local std::string g_err;

static lbm_status fail(lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,        \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

extern "C" const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm::set_error(lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

namespace {

struct Inst {
  int nx = 0, ny = 0;
  lbm_params p{};
  lbm_fsi fsi = LBM_FSI_MODIFIED;
  std::vector<uint8_t> solid;
  std::vector<double> gw;
  std::vector<uint16_t> flags;
  std::vector<uint8_t> row_plain;
  // device
  void* f[2] = {nullptr, nullptr};
  void* Fw[2] = {nullptr, nullptr};
  uint16_t* d_flags = nullptr;
  uint8_t* d_row_plain = nullptr;
  double2* d_A = nullptr;
  InstDesc desc{};
};

}  // namespace

struct lbm_ctx {
  int prec = LBM_FP64;
  cudaStream_t stream = nullptr;
  std::vector<Inst> inst;
  InstDesc* d_desc = nullptr;
  WorkItem* d_items = nullptr;
  int n_items = 0;
  // parameter classes: instances whose PhysDesc agree byte for byte; the
  // items of class j are [cls_beg[j], cls_beg[j] + cls_n[j]) and go out in
  // one launch with cls[j] as its kernel parameter
  std::vector<PhysDesc> cls;
  std::vector<int> cls_beg, cls_n, cls_tall;  // cls_tall: items before the short segments
  bool alt_items = false;  // d_items holds a second, reversed list for odd steps
  // node offsets of the instances in concatenated batch fields: instance k
  // holds [offs[k], offs[k+1]); d_offs is the device copy
  std::vector<long long> offs;
  long long* d_offs = nullptr;
  int* d_err = nullptr;       // [0] latched error bits
  unsigned* d_barrier = nullptr;  // [0] arrival counter, [1] error word of the persistent kernel
  // persistent warp strips: the items each item waits for (CSR) and the
  // per-item count of finished steps
  int *d_nbr_off = nullptr, *d_nbr = nullptr;
  unsigned* d_done = nullptr;
  // host copies of the items and of those lists (lbm_get_work_items)
  std::vector<WorkItem> h_items;
  std::vector<int> h_nbr_off, h_nbr;
  int parity = 0;
  long t = 0;
  int bx = 0, h = 0, persistent = 0, use_graph = 0, stages = 0;
  int bx_used = 0, stages_used = 0;
  // CUDA graphs of n launches, keyed by (n, parity)
  std::map<std::pair<long, int>, cudaGraphExec_t> graphs;
  // scratch for field read-back and diagnostics
  size_t scratch_n = 0;
  double *d_rho = nullptr, *d_psi = nullptr, *d_ux = nullptr, *d_uy = nullptr;
  DiagScratch diag{};
  // host transfers of the batch calls, on streams of their own so that they
  // overlap the steps: xs_in copies host densities into d_in, xs_out copies
  // the scratch fields to the host.  ev_in_free: the last initialisation
  // has read d_in; ev_out_free: the last read-back has left the scratch.
  cudaStream_t xs_in = nullptr, xs_out = nullptr;
  cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr;
  cudaEvent_t ev_out_ready = nullptr, ev_out_free = nullptr;
  double* d_in = nullptr;
  size_t in_n = 0;
};

static size_t tsize(int prec) { return prec == LBM_FP64 ? sizeof(double) : sizeof(float); }

// NVTX range over an entry point (a no-op unless a profiler is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

extern "C" lbm_status lbm_default_params(lbm_params* p) {
  if (!p) return fail(LBM_ERR_ARG, "lbm_default_params: NULL");
  memset(p, 0, sizeof *p);
  p->eos = LBM_EOS_PIECEWISE_LINEAR;
  p->eos_p[0] = 0.64;
  p->eos_p[1] = -0.04;
  p->eos_p[2] = 1.0;
  p->eos_p[3] = 1.36;
  p->eos_p[4] = 481.04;
  p->G = -1.0;
  p->sigma = 0.084;
  p->tau_rho = 1.0;
  p->tau_e = 1.0 / 0.8;
  p->tau_zeta = 1.0 / 0.8;
  p->tau_j = 1.0;
  p->tau_q = 1.0 / 1.1;
  p->tau_nu_L = 1.1;
  p->tau_nu_V = 1.1;
  p->rho_L = 500.0;
  p->rho_V = 1.0;
  p->wall = LBM_WALL_NEQ_ONNODE;
  p->ghost = LBM_GHOST_COPY;
  p->omega = LBM_OMEGA_W;
  p->prec = LBM_FP64;
  p->rho_ref = 1.0;
  return LBM_OK;
}

static lbm_status validate_params(const lbm_params* p) {
  if (!p) return fail(LBM_ERR_ARG, "params is NULL");
  if (p->eos != LBM_EOS_PIECEWISE_LINEAR && p->eos != LBM_EOS_CARNAHAN_STARLING)
    return fail(LBM_ERR_ARG, "unknown EOS %d", (int)p->eos);
  if (!(p->G < 0.0)) return fail(LBM_ERR_ARG, "G must be negative for a real psi (got %g)", p->G);
  if (p->eos == LBM_EOS_PIECEWISE_LINEAR && !(p->eos_p[3] > 0.0 && p->eos_p[4] > p->eos_p[3]))
    return fail(LBM_ERR_ARG, "need 0 < rho_1 < rho_2");
  if (p->eos == LBM_EOS_CARNAHAN_STARLING &&
      !(p->eos_p[0] > 0.0 && p->eos_p[1] > 0.0 && p->eos_p[2] > 0.0 && p->eos_p[3] > 0.0))
    return fail(LBM_ERR_ARG, "Carnahan-Starling needs a, b, R, T > 0");
  const double taus[] = {p->tau_rho, p->tau_e, p->tau_zeta, p->tau_j, p->tau_q, p->tau_nu_L,
                         p->tau_nu_V};
  for (double t : taus)
    if (!(t > 0.5) || !isfinite(t)) return fail(LBM_ERR_ARG, "relaxation times must exceed 1/2");
  if (!(p->sigma >= 0.0)) return fail(LBM_ERR_ARG, "sigma must be >= 0");
  if (!(p->rho_L > p->rho_V && p->rho_V > 0.0)) return fail(LBM_ERR_ARG, "need rho_L > rho_V > 0");
  if ((int)p->wall < 0 || (int)p->wall > 1) return fail(LBM_ERR_ARG, "unknown wall %d", (int)p->wall);
  if ((int)p->ghost < 0 || (int)p->ghost > 4) return fail(LBM_ERR_ARG, "unknown ghost %d", (int)p->ghost);
  if ((int)p->omega < 0 || (int)p->omega > 1) return fail(LBM_ERR_ARG, "unknown omega %d", (int)p->omega);
  if ((int)p->prec < 0 || (int)p->prec > 2) return fail(LBM_ERR_ARG, "unknown precision %d", (int)p->prec);
  if ((int)p->visc < 0 || (int)p->visc > 1)
    return fail(LBM_ERR_ARG, "unknown viscosity interpolation %d", (int)p->visc);
  if (!isfinite(p->rho_ref)) return fail(LBM_ERR_ARG, "rho_ref must be finite");
  return LBM_OK;
}

static inline int wrap(int a, int n) { return ((a % n) + n) % n; }

static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// node flags and plain-row table from the solid mask
static lbm_status build_flags(Inst& I) {
  const int nx = I.nx, ny = I.ny;
  const bool flat_needed = I.p.wall == LBM_WALL_NEQ_ONNODE || I.p.ghost == LBM_GHOST_COPY ||
                           I.p.ghost == LBM_GHOST_MIRROR;
  auto S = [&](int x, int y) { return I.solid[(size_t)wrap(y, ny) * nx + wrap(x, nx)] != 0; };
  if (flat_needed) {
    for (int y = 0; y < ny; ++y)
      for (int x = 1; x < nx; ++x)
        if (S(x, y) != S(0, y))
          return fail(LBM_ERR_ARG,
                      "row %d is partly solid: the NEQ wall rule and COPY/MIRROR ghosts need "
                      "walls made of whole solid rows (use LBM_WALL_HALFWAY_BB + LBM_GHOST_ZERO)",
                      y);
  }
  I.flags.assign((size_t)nx * ny, 0);
  I.row_plain.assign(ny, 1);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      uint16_t fl = 0;
      if (S(x, y)) {
        fl |= NF_SELF_SOLID;
        if (I.p.ghost == LBM_GHOST_MEAN) {
          // every axis neighbour that is fluid contributes to the mean
          if (!S(x, y + 1)) fl |= NF_GHOST_UP;
          if (!S(x, y - 1)) fl |= NF_GHOST_DOWN;
          if (!S(x + 1, y)) fl |= NF_GHOST_RIGHT;
          if (!S(x - 1, y)) fl |= NF_GHOST_LEFT;
        } else if (!S(x, y + 1)) {
          fl |= NF_GHOST_UP;
        } else if (!S(x, y - 1)) {
          fl |= NF_GHOST_DOWN;
        }
        if (I.p.ghost == LBM_GHOST_MIRROR) {
          if ((fl & NF_GHOST_UP) && S(x, y + 2))
            return fail(LBM_ERR_ARG, "MIRROR ghost needs two fluid rows above solid row %d", y);
          if ((fl & NF_GHOST_DOWN) && S(x, y - 2))
            return fail(LBM_ERR_ARG, "MIRROR ghost needs two fluid rows below solid row %d", y);
        }
        if ((fl & NF_GHOST_UP) && flat_needed && I.p.ghost != LBM_GHOST_ZERO &&
            I.p.ghost != LBM_GHOST_SKIP && !S(x, y - 1))
          return fail(LBM_ERR_ARG, "solid row %d has fluid on both sides; COPY/MIRROR ghosts "
                                   "need walls at least two rows thick", y);
      } else {
        for (int a = 1; a < Q; ++a)
          if (S(x - EX[a], y - EY[a])) fl |= (uint16_t)(1u << a);
        if (S(x, y - 1) && S(x, y + 1))
          return fail(LBM_ERR_ARG, "fluid node (%d,%d) has solid directly above and below", x, y);
        if (I.p.wall == LBM_WALL_NEQ_ONNODE) {
          if (S(x, y - 1)) fl |= NF_NEQ_BOTTOM;
          else if (S(x, y + 1)) fl |= NF_NEQ_TOP;
        }
      }
      I.flags[(size_t)y * nx + x] = fl;
      if (fl) I.row_plain[y] = 0;
    }
  return LBM_OK;
}

// A(x) = sum_a omega_a G_w(x+e_a) s(x+e_a) e_a on fluid nodes (Eqs. 10, 11, 14)
static void build_A(const Inst& I, std::vector<double2>& A) {
  const int nx = I.nx, ny = I.ny;
  const double cs2 = 1.0 / 3.0;
  const double scale = I.p.omega == LBM_OMEGA_CS2W ? cs2 : 1.0;
  A.assign((size_t)nx * ny, make_double2(0.0, 0.0));
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t i = (size_t)y * nx + x;
      if (I.solid[i]) continue;
      double ax = 0.0, ay = 0.0;
      for (int a = 1; a < Q; ++a) {
        const size_t j = (size_t)wrap(y + EY[a], ny) * nx + wrap(x + EX[a], nx);
        if (!I.solid[j]) continue;
        const double w = (a <= 4 ? 1.0 / 3.0 : 1.0 / 12.0) * scale;
        ax += w * I.gw[j] * EX[a];
        ay += w * I.gw[j] * EY[a];
      }
      A[i] = make_double2(ax, ay);
    }
}

template <typename T>
static void fill_consts(Consts<T>& K, const lbm_params& p, double rho_ref) {
  const double s_e = 1.0 / p.tau_e, s_z = 1.0 / p.tau_zeta, s_q = 1.0 / p.tau_q;
  const double G2 = p.G * p.G;
  K.G = (T)p.G;
  K.s_e = (T)s_e;
  K.s_z = (T)s_z;
  K.s_q = (T)s_q;
  K.h_e = (T)(1.0 - 0.5 * s_e);
  K.h_z = (T)(1.0 - 0.5 * s_z);
  K.h_q = (T)(1.0 - 0.5 * s_q);
  K.c_e = (T)((1.0 - 0.5 * s_e) * 12.0 * p.sigma * G2 / (p.tau_e - 0.5));
  K.c_z = (T)((1.0 - 0.5 * s_z) * 12.0 * p.sigma * G2 / (p.tau_zeta - 0.5));
  K.s_nu = (T)(1.0 / p.tau_nu_L);
  K.h_nu = (T)(1.0 - 0.5 / p.tau_nu_L);
  K.rho_ref = (T)rho_ref;
  const double h_e = 1.0 - 0.5 * s_e, h_z = 1.0 - 0.5 * s_z, h_q = 1.0 - 0.5 * s_q;
  const double c_e = h_e * 12.0 * p.sigma * G2 / (p.tau_e - 0.5);
  const double c_z = h_z * 12.0 * p.sigma * G2 / (p.tau_zeta - 0.5);
  K.ke_v = (T)(h_e / 6.0);
  K.ke_g = (T)(c_e / 36.0);
  K.ke_n = (T)(s_e / 36.0);
  K.kz_v = (T)(h_z / 6.0);
  K.kz_g = (T)(c_z / 36.0);
  K.kz_n = (T)(s_z / 36.0);
  K.kq = (T)(s_q / 12.0);
  K.kq_F = (T)(h_q / 12.0);
}

template <typename T>
static void fill_visc(Visc<T>& V, const lbm_params& p) {
  const double s_nu = 1.0 / p.tau_nu_L, h_nu = 1.0 - 0.5 * s_nu;
  V.knu = (T)(s_nu / 4.0);
  V.hnu2 = (T)(h_nu / 2.0);
  V.hnu4 = (T)(h_nu / 4.0);
  V.tauV = (T)p.tau_nu_V;
  V.dtau = (T)((p.tau_nu_L - p.tau_nu_V) / (p.rho_L - p.rho_V));
  V.tau_lo = (T)std::min(p.tau_nu_L, p.tau_nu_V);
  V.tau_hi = (T)std::max(p.tau_nu_L, p.tau_nu_V);
  V.rho_V = (T)p.rho_V;
  // dynamic viscosity mu = rho (tau - 1/2) cs^2 at the two ends, times 3
  const double muV3 = p.rho_V * (p.tau_nu_V - 0.5), muL3 = p.rho_L * (p.tau_nu_L - 0.5);
  V.muV3 = (T)muV3;
  V.dmu3 = (T)((muL3 - muV3) / (p.rho_L - p.rho_V));
}

// The part of PhysDesc that the step kernels read: the viscosity (s_nu,
// h_nu) is per instance (Visc in the descriptor head), so instances that
// differ only in viscosity share a launch.
static PhysDesc class_key(PhysDesc ph) {
  ph.cd.s_nu = ph.cd.h_nu = 0.0;
  ph.cf.s_nu = ph.cf.h_nu = 0.f;
  return ph;
}

static void fill_desc(Inst& I, int prec, int* d_err) {
  InstDesc& d = I.desc;
  PhysDesc& ph = d.ph;
  const lbm_params& p = I.p;
  memset(&ph, 0, sizeof ph);  // padding too: classes compare the bytes
  d.nx = I.nx;
  d.ny = I.ny;
  d.fsi = (int)I.fsi;
  ph.wall = (int)p.wall;
  ph.ghost = (int)p.ghost;
  d.var_nu = p.tau_nu_L == p.tau_nu_V ? 0 : (p.visc == LBM_VISC_MU_LINEAR ? 2 : 1);
  ph.omega_cs2w = p.omega == LBM_OMEGA_CS2W;
  ph.eos = (int)p.eos;
  if (p.eos == LBM_EOS_CARNAHAN_STARLING) {
    ph.cs_a = p.eos_p[0];
    ph.cs_b = p.eos_p[1];
    ph.cs_RT = p.eos_p[2] * p.eos_p[3];
    ph.cs_g = 2.0 / (-p.G);
  }
  d.plane = (long long)I.nx * I.ny;
  d.f[0] = I.f[0];
  d.f[1] = I.f[1];
  d.Fw[0] = I.Fw[0];
  d.Fw[1] = I.Fw[1];
  d.flags = I.d_flags;
  d.row_plain = I.d_row_plain;
  d.A = I.d_A;
  d.err = d_err;
  // Eq. (15) in the form psi^2 = 2 cs^2 / |G| * ((1 - k) rho - c) per branch
  const double cs2 = 1.0 / 3.0, kV = p.eos_p[0], kM = p.eos_p[1], kL = p.eos_p[2];
  const double r1 = p.eos_p[3], r2 = p.eos_p[4];
  const double g = 2.0 * cs2 / (-p.G);
  ph.rho1 = r1;
  ph.rho2 = r2;
  ph.aV = g * (1.0 - kV);
  ph.aM = g * (1.0 - kM);
  ph.bM = -g * (kV - kM) * r1;
  ph.aL = g * (1.0 - kL);
  ph.bL = -g * (kV * r1 + kM * (r2 - r1) - kL * r2);
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  const double ab[3][2] = {{ph.aV, 0.0}, {ph.aM, ph.bM}, {ph.aL, ph.bL}};
  for (int b = 0; b < 3; ++b) {
    split(ab[b][0], ph.eosf[b][0], ph.eosf[b][1]);
    split(ab[b][1], ph.eosf[b][2], ph.eosf[b][3]);
  }
  split(r1, ph.thrf[0], ph.thrf[1]);
  split(r2, ph.thrf[2], ph.thrf[3]);
  // the FP32 storage shift is rounded to FP32 so that it is exact in both precisions
  const double rho_ref = prec == LBM_FP64 ? 0.0 : (double)(float)p.rho_ref;
  fill_consts<double>(ph.cd, p, rho_ref);
  fill_consts<float>(ph.cf, p, rho_ref);
  fill_visc<double>(d.vd, p);
  fill_visc<float>(d.vf, p);
}

static void free_inst(Inst& I) {
  for (int k = 0; k < 2; ++k) {
    cudaFree(I.f[k]);
    cudaFree(I.Fw[k]);
    I.f[k] = I.Fw[k] = nullptr;
  }
  cudaFree(I.d_flags);
  cudaFree(I.d_row_plain);
  cudaFree(I.d_A);
  I.d_flags = nullptr;
  I.d_row_plain = nullptr;
  I.d_A = nullptr;
}

static void free_ctx(lbm_ctx* c) {
  if (!c) return;
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  for (auto& I : c->inst) free_inst(I);
  cudaFree(c->d_desc);
  cudaFree(c->d_items);
  cudaFree(c->d_offs);
  cudaFree(c->d_err);
  cudaFree(c->d_barrier);
  cudaFree(c->d_nbr_off);
  cudaFree(c->d_nbr);
  cudaFree(c->d_done);
  cudaFree(c->d_rho);
  cudaFree(c->d_psi);
  cudaFree(c->d_ux);
  cudaFree(c->d_uy);
  diag_free(c->diag);
  if (c->xs_in) {
    cudaStreamSynchronize(c->xs_in);
    cudaStreamSynchronize(c->xs_out);
    cudaStreamDestroy(c->xs_in);
    cudaStreamDestroy(c->xs_out);
    cudaEventDestroy(c->ev_in_ready);
    cudaEventDestroy(c->ev_in_free);
    cudaEventDestroy(c->ev_out_ready);
    cudaEventDestroy(c->ev_out_free);
  }
  cudaFree(c->d_in);
  delete c;
}

static lbm_status upload_inst(lbm_ctx* c, Inst& I) {
  const size_t N = (size_t)I.nx * I.ny;
  const size_t ts = tsize(c->prec);
  for (int k = 0; k < 2; ++k) {
    CK(cudaMalloc(&I.f[k], Q * N * ts));
    CK(cudaMemsetAsync(I.f[k], 0, Q * N * ts, c->stream));
    CK(cudaMalloc(&I.Fw[k], N * 2 * ts));
    CK(cudaMemsetAsync(I.Fw[k], 0, N * 2 * ts, c->stream));
  }
  CK(cudaMalloc(&I.d_flags, N * sizeof(uint16_t)));
  CK(cudaMemcpy(I.d_flags, I.flags.data(), N * sizeof(uint16_t), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&I.d_row_plain, I.ny));
  CK(cudaMemcpy(I.d_row_plain, I.row_plain.data(), I.ny, cudaMemcpyHostToDevice));
  std::vector<double2> A;
  build_A(I, A);
  CK(cudaMalloc(&I.d_A, N * sizeof(double2)));
  CK(cudaMemcpy(I.d_A, A.data(), N * sizeof(double2), cudaMemcpyHostToDevice));
  return LBM_OK;
}

// Dependencies of the persistent warp strips: item i waits for the items of
// its instance whose nodes lie within STRIP_RADIUS nodes of its own along x
// and along y (periodic); the relation is symmetric and contains i.  Items
// of an instance are its segments (outer) times its cols-wide strips
// (inner), instances in order.  shape holds nx, ny per instance.  CSR out:
// the neighbours of item i are nb[off[i] .. off[i+1]).
constexpr int STRIP_RADIUS = 4;
static void strip_neighbours(const std::vector<WorkItem>& items, const std::vector<int>& shape,
                             int cols, std::vector<int>& off, std::vector<int>& nb) {
  off.assign(1, 0);
  nb.clear();
  auto near = [](int a0, int a1, int b0, int b1, int n) {
    // [a0 - R, a1 + R) meets [b0, b1) modulo n
    const int lo = a0 - STRIP_RADIUS, hi = a1 + STRIP_RADIUS;
    if (hi - lo >= n) return true;
    for (int sh = -n; sh <= n; sh += n)
      if (lo < b1 + sh && b0 + sh < hi) return true;
    return false;
  };
  size_t i0 = 0;
  while (i0 < items.size()) {
    const int k = items[i0].inst;
    const int nx = shape[2 * k], ny = shape[2 * k + 1];
    size_t i1 = i0;
    while (i1 < items.size() && items[i1].inst == k) ++i1;
    const int nstr = (nx + cols - 1) / cols;
    const int nseg = (int)((i1 - i0) / nstr);
    auto x1 = [&](int st) { return std::min(nx, st * cols + cols); };
    std::vector<std::vector<int>> sn(nstr), gn(nseg);
    for (int a = 0; a < nstr; ++a)
      for (int b = 0; b < nstr; ++b)
        if (near(a * cols, x1(a), b * cols, x1(b), nx)) sn[a].push_back(b);
    for (int a = 0; a < nseg; ++a) {
      const WorkItem& ia = items[i0 + (size_t)a * nstr];
      for (int b = 0; b < nseg; ++b) {
        const WorkItem& ib = items[i0 + (size_t)b * nstr];
        if (near(ia.y0, ia.y1, ib.y0, ib.y1, ny)) gn[a].push_back(b);
      }
    }
    for (int a = 0; a < nseg; ++a)
      for (int st = 0; st < nstr; ++st) {
        for (int b : gn[a])
          for (int u : sn[st]) nb.push_back((int)i0 + b * nstr + u);
        off.push_back((int)nb.size());
      }
    i0 = i1;
  }
}

// work items: bx-wide column strips, h-row segments
static lbm_status build_items(lbm_ctx* c) {
  // captured graphs refer to the item buffers rebuilt below
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
  // block rows: a block of bx threads covers bx - 2 columns (its two edge
  // lanes evaluate the halo columns); warp strips: each warp covers 30
  // FP32 storage: strips with two columns per lane where every lattice
  // width is a multiple of 4 (automatic, or stages 4; per-step or
  // persistent), else two rows per lane unless one is asked for (a
  // persistent launch of those takes one row per lane)
  bool cols_ok = c->prec == LBM_FP32_SHIFTED;
  for (auto& I : c->inst) cols_ok = cols_ok && (I.nx % 4 == 0);
  // the block width of block rows: the widest instance decides; whole rows
  // up to 512 threads, else 256-wide strips
  int bx_rows = 0;
  {
    int maxnx = 0;
    for (auto& I : c->inst) maxnx = std::max(maxnx, I.nx);
    bx_rows = maxnx + 2 <= 512 ? ((maxnx + 2 + 31) / 32) * 32 : 256;
  }
  // FP64 with the automatic pipeline: block rows where the batch gives at
  // least 1.5 waves of them (one block per SM), warp strips otherwise.  A
  // block row of up to 510 columns has 2 halo columns, a warp strip 2 of
  // 32: block rows issue ~6% fewer FP64 operations, the bound of the FP64
  // step (sweep 3.61k against 3.45k MLUPS, 8192x4096 4.04k against 3.94k),
  // but a single small lattice leaves most SMs idle in them (256x128: 46
  // against 765 MLUPS).
  int stages = c->stages;
  if (c->prec == LBM_FP64 && stages == 0 && !c->persistent) {
    const int bxr = c->bx > 0 ? std::max(32, std::min(512, ((c->bx + 31) / 32) * 32)) : bx_rows;
    const int colsr = bxr - 2;
    long long nb = 0;
    for (auto& I : c->inst) {
      const int hmax_rows = 64;
      const int hr = c->h > 0 ? c->h : (I.ny + (I.ny + hmax_rows - 1) / hmax_rows - 1) /
                                           ((I.ny + hmax_rows - 1) / hmax_rows);
      nb += (long long)((I.nx + colsr - 1) / colsr) * ((I.ny + hr - 1) / hr);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (2 * nb >= 3LL * std::max(sms, 1)) stages = 1;
  }
  const bool cols_mode = cols_ok && (stages == 0 || stages == 4);
  const bool warp_mode = cols_mode || stages == 0 || stages == 2 || stages == 3 || stages == 4;
  const bool two_rows = warp_mode && !cols_mode && stages != 3 && c->prec == LBM_FP32_SHIFTED;
  int bx = c->bx;
  if (bx <= 0) bx = bx_rows;
  // warp strips: 8 warps per block; 4 for two rows per lane (128 registers
  // a thread: four blocks, 16 warps per SM)
  if (warp_mode && c->bx <= 0) bx = cols_mode ? 64 : (two_rows ? 128 : 256);
  bx = std::max(32, std::min(warp_mode ? 256 : 512, ((bx + 31) / 32) * 32));
  const int cols = cols_mode ? 60 : (warp_mode ? 30 : bx - 2);
  // parameter classes, in order of first appearance
  c->cls.clear();
  c->cls_beg.clear();
  c->cls_n.clear();
  c->cls_tall.clear();
  std::vector<int> inst_cls(c->inst.size());
  for (size_t k = 0; k < c->inst.size(); ++k) {
    const PhysDesc ph = class_key(c->inst[k].desc.ph);
    size_t j = 0;
    while (j < c->cls.size() && memcmp(&c->cls[j], &ph, sizeof ph) != 0) ++j;
    if (j == c->cls.size()) c->cls.push_back(ph);
    inst_cls[k] = (int)j;
  }
  if (c->persistent && c->cls.size() > 1) {
    c->persistent = 0;
    return fail(LBM_ERR_ARG, "a persistent launch needs one parameter set across the batch "
                             "(this batch has %d)", (int)c->cls.size());
  }
  // items of instance k: h-row segments of cols-wide strips; without a
  // height from lbm_set_launch, balanced segments of at most hmax rows
  auto seg_h = [&](const Inst& I, int hmax) {
    if (c->h > 0) return c->h;
    const int nseg = (I.ny + hmax - 1) / hmax;
    int h = (I.ny + nseg - 1) / nseg;
    if (two_rows) h += h & 1;  // whole row pairs
    return h;
  };
  // at most 64 rows (32 for warp strips: more, shorter strips balance the
  // waves better).  Warp strips: while the batch gives fewer than two waves
  // of strips for the resident warps (16 per SM for every warp-strip kernel
  // at its register count), halve the segment height, down to 2 rows.
  // Strips shorter than that cost halo rows but fill the GPU: a single
  // 256x128 lattice in FP64 runs 7x faster with 2-row segments than with
  // one 32-row segment per strip; with two or more waves the height does
  // not matter between 16 and 30 rows.
  int hmax = warp_mode ? 32 : 64;
  if (warp_mode && c->h <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = 16LL * std::max(sms, 1);
    int maxny = 0;
    for (const Inst& I : c->inst) maxny = std::max(maxny, I.ny);
    auto count = [&](int hm) {
      long long n = 0;
      for (const Inst& I : c->inst) {
        const int h = seg_h(I, hm);
        n += (long long)((I.ny + h - 1) / h) * ((I.nx + cols - 1) / cols);
      }
      return n;
    };
    if (c->persistent) {
      // one launch for all steps, strips waiting on their neighbours: as
      // many strips as possible but no more than one per resident warp
      while (hmax < maxny && count(hmax) > slots) hmax *= 2;
      while (hmax > 2 && count(hmax / 2) <= slots) hmax /= 2;
      // then row by row: the lowest height that still fits (64 uneven
      // lattices: 2383 strips instead of 1755 for 2432 warps, +9% MLUPS)
      while (hmax > 2 && count(hmax - 1) <= slots) --hmax;
    } else if (cols_mode) {
      // the tallest segments that still give 3.5 waves of strips.  Fewer
      // waves leave SMs idle at the end of the step; shorter segments spend
      // more on their two halo rows; one wave of long runs of rows per warp
      // touches the whole batch at once and ran at two thirds of the rate
      // (sweep of 72 400x200 lattices: 12-row segments, 3.5 waves, beat 25-
      // to 29-row ones by 8%); a batch too small for that takes 2-row segments
      while (hmax > 2 && 2 * count(hmax) < 7 * slots) --hmax;
    } else {
      while (hmax > 2 && count(hmax) < 2 * slots) hmax = std::max(2, hmax / 2);
    }
  }
  auto add_items = [&](int k, std::vector<WorkItem>& items) {
    const Inst& I = c->inst[k];
    auto strips = [&](int y0, int y1) {
      for (int x0 = 0; x0 < I.nx; x0 += cols) items.push_back({k, x0, y0, y1});
    };
    if (c->h > 0) {
      for (int y0 = 0; y0 < I.ny; y0 += c->h) strips(y0, std::min(I.ny, y0 + c->h));
      return;
    }
    // the automatic height: nseg segments with the rows (whole pairs for
    // two rows per lane) spread evenly, so that no segment is much shorter
    // than the others (200 rows in pairs: 30,30,28,28,28,28,28 rather than
    // six of 30 and one of 20)
    const int g = two_rows ? 2 : 1;
    const int units = (I.ny + g - 1) / g;
    const int nseg = (I.ny + seg_h(I, hmax) - 1) / seg_h(I, hmax);
    int y0 = 0;
    for (int j = 0; j < nseg && y0 < I.ny; ++j) {
      const int u = units / nseg + (j < units % nseg ? 1 : 0);
      const int y1 = std::min(I.ny, y0 + u * g);
      strips(y0, y1);
      y0 = y1;
    }
  };
  // column-pair strips launched per step with the automatic height, on a
  // batch that gives at least 2.5 waves: tall segments of every lattice
  // first, then about one wave of 4-row segments taken off the top of each
  // strip, so that the last wave is short and few SMs wait at its end
  const bool lpt = cols_mode && !c->persistent && c->h <= 0;
  std::vector<WorkItem> items;
  for (int j = 0; j < (int)c->cls.size(); ++j) {
    c->cls_beg.push_back((int)items.size());
    bool split = false;
    int nshort = 0;
    if (lpt) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const long long slots = 16LL * std::max(sms, 1);
      long long strips_n = 0, items_n = 0;
      for (int k = 0; k < (int)c->inst.size(); ++k)
        if (inst_cls[k] == j) {
          const Inst& I = c->inst[k];
          const long long ns = (I.nx + cols - 1) / cols;
          strips_n += ns;
          items_n += ns * ((I.ny + seg_h(I, hmax) - 1) / seg_h(I, hmax));
        }
      nshort = (int)std::max<long long>(1, (slots + strips_n - 1) / std::max(strips_n, 1LL));
      split = strips_n > 0 && 2 * items_n >= 5 * slots;
    }
    if (!split) {
      for (int k = 0; k < (int)c->inst.size(); ++k)
        if (inst_cls[k] == j) add_items(k, items);
    } else {
      // per strip: the rows below ny - 4 nshort in tall segments (the
      // automatic count less nshort, at least one), the rest in 4-row ones
      std::vector<WorkItem> tall, shorts;
      for (int k = 0; k < (int)c->inst.size(); ++k) {
        if (inst_cls[k] != j) continue;
        const Inst& I = c->inst[k];
        const int ns = std::min(nshort, std::max(0, (I.ny - 4) / 4));
        const int ytop = I.ny - 4 * ns;
        const int nseg_auto = (I.ny + seg_h(I, hmax) - 1) / seg_h(I, hmax);
        const int nt = std::max(1, std::min(ytop, nseg_auto - ns));
        int y0 = 0;
        for (int q = 0; q < nt; ++q) {
          const int u = ytop / nt + (q < ytop % nt ? 1 : 0);
          for (int x0 = 0; x0 < I.nx; x0 += cols) tall.push_back({k, x0, y0, y0 + u});
          y0 += u;
        }
        for (int q = 0; q < ns; ++q, y0 += 4)
          for (int x0 = 0; x0 < I.nx; x0 += cols) shorts.push_back({k, x0, y0, y0 + 4});
      }
      items.insert(items.end(), tall.begin(), tall.end());
      items.insert(items.end(), shorts.begin(), shorts.end());
      c->cls_tall.push_back((int)tall.size());
    }
    if ((int)c->cls_tall.size() <= j) c->cls_tall.push_back((int)items.size() - c->cls_beg[j]);
    c->cls_n.push_back((int)items.size() - c->cls_beg[j]);
  }
  cudaFree(c->d_items);
  c->d_items = nullptr;
  // per-step launches of the column strips alternate the order of the
  // lattices from step to step (odd steps take each part of a class's list,
  // tall and short segments, back to front): a step starts on the rows the
  // previous one wrote last, which may still be in L2
  const bool alt = cols_mode && !c->persistent;
  std::vector<WorkItem> rev(items);
  if (alt)
    for (int j = 0; j < (int)c->cls.size(); ++j) {
      const int b0 = c->cls_beg[j], n = c->cls_n[j];
      const int nt = j < (int)c->cls_tall.size() ? c->cls_tall[j] : n;
      std::reverse(rev.begin() + b0, rev.begin() + b0 + nt);
      std::reverse(rev.begin() + b0 + nt, rev.begin() + b0 + n);
    }
  const size_t nb = items.size() * sizeof(WorkItem);
  CK(cudaMalloc(&c->d_items, 2 * nb));
  CK(cudaMemcpy(c->d_items, items.data(), nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->d_items + items.size(), rev.data(), nb, cudaMemcpyHostToDevice));
  c->alt_items = alt;
  c->n_items = (int)items.size();
  c->h_items = items;
  c->h_nbr_off.assign(items.size() + 1, 0);
  c->h_nbr.clear();
  cudaFree(c->d_nbr_off);
  cudaFree(c->d_nbr);
  cudaFree(c->d_done);
  c->d_nbr_off = c->d_nbr = nullptr;
  c->d_done = nullptr;
  if (c->persistent && warp_mode) {
    std::vector<int> shape;
    for (const Inst& I : c->inst) {
      shape.push_back(I.nx);
      shape.push_back(I.ny);
    }
    std::vector<int> off, nb;
    strip_neighbours(items, shape, cols, off, nb);
    c->h_nbr_off = off;
    c->h_nbr = nb;
    CK(cudaMalloc(&c->d_nbr_off, off.size() * sizeof(int)));
    CK(cudaMemcpy(c->d_nbr_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_nbr, std::max<size_t>(nb.size(), 1) * sizeof(int)));
    if (!nb.empty())
      CK(cudaMemcpy(c->d_nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_done, items.size() * sizeof(unsigned)));
  }
  c->bx_used = bx;
  // TMA pipeline: FP32 storage, every lattice width a multiple of 4
  bool tma_ok = c->prec != LBM_FP64;
  for (auto& I : c->inst) tma_ok = tma_ok && (I.nx % 4 == 0);
  int S = stages == 0 ? 8 : stages;
  // the ring must fit the per-block shared-memory limit; the pipeline needs
  // at least 8 stages (rows y-1..y+2 in use while later rows are in flight)
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  while (S >= 8 && tma_smem_bytes(bx, S) > (size_t)optin) S /= 2;
  c->stages_used = cols_mode   ? PIPE_COLS
                   : warp_mode ? (stages == 3 ? PIPE_WARP1 : PIPE_WARP)
                               : ((tma_ok && stages != 1 && S >= 8) ? S : 0);
  return LBM_OK;
}

static lbm_status upload_descs(lbm_ctx* c) {
  std::vector<InstDesc> h(c->inst.size());
  for (size_t k = 0; k < c->inst.size(); ++k) h[k] = c->inst[k].desc;
  if (!c->d_desc) CK(cudaMalloc(&c->d_desc, h.size() * sizeof(InstDesc)));
  CK(cudaMemcpy(c->d_desc, h.data(), h.size() * sizeof(InstDesc), cudaMemcpyHostToDevice));
  return LBM_OK;
}

static lbm_status make_inst(const lbm_instance_desc& d, Inst& I) {
  lbm_status st = validate_params(d.params);
  if (st != LBM_OK) return st;
  if (d.nx < 3 || d.ny < 4) return fail(LBM_ERR_ARG, "lattice must be at least 3 x 4 (got %d x %d)", d.nx, d.ny);
  if ((long long)d.nx * d.ny * Q >= (1LL << 31))
    return fail(LBM_ERR_ARG, "lattice too large: 9 * nx * ny must stay below 2^31");
  if ((int)d.fsi < 0 || (int)d.fsi > 2) return fail(LBM_ERR_ARG, "unknown interaction %d", (int)d.fsi);
  I.nx = d.nx;
  I.ny = d.ny;
  I.p = *d.params;
  I.fsi = d.fsi;
  const size_t N = (size_t)d.nx * d.ny;
  I.solid.assign(N, 0);
  if (d.solid)
    for (size_t i = 0; i < N; ++i) I.solid[i] = d.solid[i] != 0;
  I.gw.assign(N, 0.0);
  for (size_t i = 0; i < N; ++i)
    if (I.solid[i]) {
      I.gw[i] = d.gw_field ? d.gw_field[i] : d.gw_uniform;
      if (!isfinite(I.gw[i])) return fail(LBM_ERR_ARG, "non-finite G_w at node %zu", i);
    }
  return build_flags(I);
}

extern "C" lbm_status lbm_create_batch(int count, const lbm_instance_desc* descs, void* stream,
                                       lbm_ctx** out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count <= 0 || !descs) return fail(LBM_ERR_ARG, "need count > 0 instance descriptors");
  for (int k = 0; k < count; ++k)
    if (!descs[k].params) return fail(LBM_ERR_ARG, "instance %d has no params", k);
  const int prec = (int)descs[0].params->prec;
  for (int k = 1; k < count; ++k)
    if ((int)descs[k].params->prec != prec)
      return fail(LBM_ERR_ARG, "all instances of a batch must share the precision");
  lbm_ctx* c = new lbm_ctx();
  c->prec = prec;
  c->stream = (cudaStream_t)stream;
  c->inst.resize(count);
  for (int k = 0; k < count; ++k) {
    lbm_status st = make_inst(descs[k], c->inst[k]);
    if (st != LBM_OK) {
      free_ctx(c);
      return st;
    }
  }
  lbm_status st = LBM_OK;
  cudaError_t e = cudaMalloc(&c->d_err, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_barrier, sizeof(unsigned) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->d_barrier, 0, sizeof(unsigned) * 4);
  if (e != cudaSuccess) {
    free_ctx(c);
    return fail(LBM_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(e));
  }
  for (auto& I : c->inst) {
    st = upload_inst(c, I);
    if (st != LBM_OK) break;
    fill_desc(I, prec, c->d_err);
  }
  if (st == LBM_OK) st = upload_descs(c);
  if (st == LBM_OK) {
    c->offs.assign(1, 0);
    for (auto& I : c->inst) c->offs.push_back(c->offs.back() + (long long)I.nx * I.ny);
    e = cudaMalloc(&c->d_offs, c->offs.size() * sizeof(long long));
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_offs, c->offs.data(), c->offs.size() * sizeof(long long),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "offset table: %s", cudaGetErrorString(e));
  }
  if (st == LBM_OK) st = build_items(c);
  if (st == LBM_OK) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(LBM_ERR_CUDA, "set-up failed: %s", cudaGetErrorString(e));
  }
  if (st != LBM_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return LBM_OK;
}

extern "C" lbm_status lbm_create(int nx, int ny, const lbm_params* p, const uint8_t* solid,
                                 lbm_fsi fsi, const double* gw_field, double gw_uniform,
                                 void* stream, lbm_ctx** out) {
  lbm_instance_desc d;
  d.nx = nx;
  d.ny = ny;
  d.params = p;
  d.solid = solid;
  d.fsi = fsi;
  d.gw_field = gw_field;
  d.gw_uniform = gw_uniform;
  return lbm_create_batch(1, &d, stream, out);
}

extern "C" void lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

extern "C" lbm_status lbm_instance_size(const lbm_ctx* c, int inst, int* nx, int* ny) {
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (inst < 0 || inst >= (int)c->inst.size())
    return fail(LBM_ERR_ARG, "instance %d out of range [0, %d)", inst, (int)c->inst.size());
  if (nx) *nx = c->inst[inst].nx;
  if (ny) *ny = c->inst[inst].ny;
  return LBM_OK;
}

static lbm_status check_inst(const lbm_ctx* c, int inst) {
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (inst < 0 || inst >= (int)c->inst.size())
    return fail(LBM_ERR_ARG, "instance %d out of range [0, %d)", inst, (int)c->inst.size());
  return LBM_OK;
}

// Every user of the scratch fields enqueues its work on c->stream after the
// last read-back of them (lbm_get_fields_all_async copies from them on xs_out).
static lbm_status ensure_scratch(lbm_ctx* c, size_t N) {
  if (c->xs_out) CK(cudaStreamWaitEvent(c->stream, c->ev_out_free, 0));
  if (c->scratch_n >= N) return LBM_OK;
  if (c->xs_out) CK(cudaStreamSynchronize(c->xs_out));
  cudaFree(c->d_rho);
  cudaFree(c->d_psi);
  cudaFree(c->d_ux);
  cudaFree(c->d_uy);
  c->d_rho = c->d_psi = c->d_ux = c->d_uy = nullptr;
  c->scratch_n = 0;
  CK(cudaMalloc(&c->d_rho, N * sizeof(double)));
  CK(cudaMalloc(&c->d_psi, N * sizeof(double)));
  CK(cudaMalloc(&c->d_ux, N * sizeof(double)));
  CK(cudaMalloc(&c->d_uy, N * sizeof(double)));
  c->scratch_n = N;
  return LBM_OK;
}

static lbm_status set_density_dev(lbm_ctx* c, int inst, const double* d_rho0) {
  Inst& I = c->inst[inst];
  CK(launch_init(c->prec, I.desc, c->d_desc + inst, c->parity, d_rho0, c->stream));
  // every instance shares the parity; initialise the other buffer's force too
  return LBM_OK;
}

// the copy into the scratch field and the initialisation kernel, enqueued;
// a later call reuses the scratch only after these in stream order
static lbm_status enqueue_set_density(lbm_ctx* c, int inst, const double* rho, int src_is_device) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!rho) return fail(LBM_ERR_ARG, "rho is NULL");
  const size_t N = (size_t)c->inst[inst].nx * c->inst[inst].ny;
  st = ensure_scratch(c, N);
  if (st != LBM_OK) return st;
  CK(cudaMemcpyAsync(c->d_rho, rho, N * sizeof(double),
                     src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  st = set_density_dev(c, inst, c->d_rho);
  if (st != LBM_OK) return st;
  c->t = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_density(lbm_ctx* c, int inst, const double* rho, int src_is_device) {
  Range range_("lbm_set_density");
  lbm_status st = enqueue_set_density(c, inst, rho, src_is_device);
  if (st != LBM_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_set_density_async(lbm_ctx* c, int inst, const double* rho,
                                            int src_is_device) {
  return enqueue_set_density(c, inst, rho, src_is_device);
}

extern "C" lbm_status lbm_init_droplet(lbm_ctx* c, int inst, double x0, double y0, double R,
                                       double width) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!(width > 0.0) || !(R >= 0.0)) return fail(LBM_ERR_ARG, "need R >= 0 and width > 0");
  const Inst& I = c->inst[inst];
  std::vector<double> rho((size_t)I.nx * I.ny);
  const double rl = I.p.rho_L, rv = I.p.rho_V;
  for (int y = 0; y < I.ny; ++y)
    for (int x = 0; x < I.nx; ++x) {
      double dx = (double)x - x0;
      dx -= I.nx * floor(dx / I.nx + 0.5);
      const double dy = (double)y - y0;
      const double r = sqrt(dx * dx + dy * dy);
      rho[(size_t)y * I.nx + x] = rv + 0.5 * (rl - rv) * (1.0 - tanh(2.0 * (r - R) / width));
    }
  return lbm_set_density(c, inst, rho.data(), 0);
}

// one time step: one launch per parameter class
static cudaError_t launch_one_step(lbm_ctx* c, int parity, cudaStream_t s) {
  for (size_t j = 0; j < c->cls.size(); ++j) {
    const WorkItem* it = c->d_items + c->cls_beg[j] + (c->alt_items && (parity & 1) ? c->n_items : 0);
    cudaError_t e = launch_step(c->prec, c->cls[j], c->d_desc, it, c->cls_n[j], parity, c->bx_used,
                                c->stages_used, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one cooperative launch for all n steps (one parameter class, checked when
// the items are built): block rows with a grid barrier per step, or warp
// strips one row per lane, each waiting only for its neighbours.  The
// kernel's error word is separate from the context's so that a time-out
// does not hide behind a stale value.
static cudaError_t launch_persistent(lbm_ctx* c, long n, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->d_barrier + 1, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (is_warp_pipe(c->stages_used) || c->stages_used == PIPE_COLS)
    return launch_step_dataflow(c->prec, c->cls[0], c->d_desc, c->d_items, c->d_nbr_off,
                                c->d_nbr, c->n_items, c->parity, n, c->bx_used,
                                c->stages_used, c->d_done,
                                (int*)(c->d_barrier + 1), s);
  return launch_step_persistent(c->prec, c->cls[0], c->d_desc, c->d_items, c->n_items, c->parity,
                                n, c->bx_used, c->stages_used, c->d_barrier, s);
}

static lbm_status enqueue_steps(lbm_ctx* c, long n) {
  if (c->persistent) {
    CK(launch_persistent(c, n, c->stream));
    return LBM_OK;
  }
  for (long k = 0; k < n; ++k) CK(launch_one_step(c, (int)((c->parity + k) & 1), c->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_ctx* c, long n) {
  Range range_("lbm_step");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  if (n == 0) return LBM_OK;
  if (c->use_graph) {
    auto key = std::make_pair(n, c->parity);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      cudaStream_t cap;
      CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaGraph_t g;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        if (c->persistent) {
          e = launch_persistent(c, n, cap);  // one persistent launch for all n steps
        } else {
          for (long k = 0; k < n && e == cudaSuccess; ++k)
            e = launch_one_step(c, (int)((c->parity + k) & 1), cap);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
      }
      cudaGraphExec_t ge = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (e == cudaSuccess) cudaGraphDestroy(g);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
      it = c->graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second, c->stream));
  } else {
    lbm_status st = enqueue_steps(c, n);
    if (st != LBM_OK) return st;
  }
  c->parity = (int)((c->parity + n) & 1);
  c->t += n;
  return LBM_OK;
}

extern "C" long lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

extern "C" lbm_status lbm_sync(lbm_ctx* c) {
  Range range_("lbm_sync");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  CK(cudaStreamSynchronize(c->stream));
  if (c->xs_in) {
    CK(cudaStreamSynchronize(c->xs_in));
    CK(cudaStreamSynchronize(c->xs_out));
  }
  int h[2] = {0, 0};
  CK(cudaMemcpy(&h[0], c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&h[1], c->d_barrier + 1, sizeof(int), cudaMemcpyDeviceToHost));
  const int bits = h[0] | h[1];
  if (bits & ERR_BOUNDS)
    return fail(LBM_ERR_STATE, "an index of a step kernel fell outside its buffer (checked build)");
  if (bits & ERR_TIMEOUT)
    return fail(LBM_ERR_TIMEOUT, "a grid barrier of the persistent step kernel timed out");
  if (bits & ERR_NONFINITE)
    return fail(LBM_ERR_NONFINITE, "non-finite or non-positive density on a fluid node");
  return LBM_OK;
}

// the field kernels and the copies out of the scratch fields, enqueued
static lbm_status enqueue_get_fields(lbm_ctx* c, int inst, double* rho, double* ux, double* uy,
                                     int dst_is_device) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  const Inst& I = c->inst[inst];
  const size_t N = (size_t)I.nx * I.ny;
  st = ensure_scratch(c, N);
  if (st != LBM_OK) return st;
  CK(launch_macro(c->prec, I.desc, c->d_desc + inst, c->parity, c->d_rho, c->d_psi,
                  (ux || uy) ? c->d_ux : nullptr, (ux || uy) ? c->d_uy : nullptr, nullptr,
                  c->stream));
  const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (rho) CK(cudaMemcpyAsync(rho, c->d_rho, N * sizeof(double), k, c->stream));
  if (ux) CK(cudaMemcpyAsync(ux, c->d_ux, N * sizeof(double), k, c->stream));
  if (uy) CK(cudaMemcpyAsync(uy, c->d_uy, N * sizeof(double), k, c->stream));
  return LBM_OK;
}

extern "C" lbm_status lbm_get_fields(lbm_ctx* c, int inst, double* rho, double* ux, double* uy,
                                     int dst_is_device) {
  Range range_("lbm_get_fields");
  lbm_status st = enqueue_get_fields(c, inst, rho, ux, uy, dst_is_device);
  if (st != LBM_OK) return st;
  return lbm_sync(c);
}

extern "C" lbm_status lbm_get_fields_async(lbm_ctx* c, int inst, double* rho, double* ux,
                                           double* uy, int dst_is_device) {
  return enqueue_get_fields(c, inst, rho, ux, uy, dst_is_device);
}

extern "C" lbm_status lbm_contact_radius(lbm_ctx* c, int inst, int row, double level,
                                         double x_ref, double* r_out) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!r_out) return fail(LBM_ERR_ARG, "r_out is NULL");
  const Inst& I = c->inst[inst];
  if (row < 0 || row >= I.ny) return fail(LBM_ERR_ARG, "row %d outside [0, %d)", row, I.ny);
  if (!isfinite(x_ref)) return fail(LBM_ERR_ARG, "x_ref must be finite");
  if (!(level > 0.0)) level = 0.5 * (I.p.rho_L + I.p.rho_V);
  st = ensure_scratch(c, (size_t)I.nx * I.ny);
  if (st != LBM_OK) return st;
  int xi = (int)floor(x_ref + 0.5) % I.nx;
  if (xi < 0) xi += I.nx;
  // row densities in d_rho[0, nx), the radius in d_rho[nx]
  CK(launch_row_rho(c->prec, I.desc, c->d_desc + inst, c->parity, row, c->d_rho, c->stream));
  CK(launch_contact_scan(c->d_rho, I.nx, level, xi, c->d_rho + I.nx, c->stream));
  CK(cudaMemcpyAsync(r_out, c->d_rho + I.nx, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return lbm_sync(c);
}

// the side streams and events of the batch host transfers, made on first use
// (all or nothing: the context keeps none of them if one cannot be made)
static lbm_status ensure_xfer(lbm_ctx* c) {
  if (c->xs_in) return LBM_OK;
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    for (cudaStream_t x : st)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    return fail(LBM_ERR_CUDA, "copy streams: %s", cudaGetErrorString(e));
  }
  c->xs_in = st[0];
  c->xs_out = st[1];
  c->ev_in_ready = ev[0];
  c->ev_in_free = ev[1];
  c->ev_out_ready = ev[2];
  c->ev_out_free = ev[3];
  return LBM_OK;
}

extern "C" lbm_status lbm_set_density_all_async(lbm_ctx* c, const double* rho,
                                                int src_is_device) {
  Range range_("lbm_set_density_all_async");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (!rho) return fail(LBM_ERR_ARG, "rho is NULL");
  const long long total = c->offs.back();
  if (src_is_device) {
    // read in place, in stream order
    CK(launch_init_all(c->prec, c->d_desc, c->d_offs, (int)c->inst.size(), total, c->parity, rho,
                       c->stream));
    c->t = 0;
    return LBM_OK;
  }
  lbm_status st = ensure_xfer(c);
  if (st != LBM_OK) return st;
  if (c->in_n < (size_t)total) {
    CK(cudaStreamSynchronize(c->xs_in));
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_in);
    c->d_in = nullptr;
    c->in_n = 0;
    CK(cudaMalloc(&c->d_in, total * sizeof(double)));
    c->in_n = (size_t)total;
  }
  // the upload starts at once, beside the steps still queued on c->stream,
  // as soon as the previous initialisation has read d_in
  CK(cudaStreamWaitEvent(c->xs_in, c->ev_in_free, 0));
  CK(cudaMemcpyAsync(c->d_in, rho, total * sizeof(double), cudaMemcpyHostToDevice, c->xs_in));
  CK(cudaEventRecord(c->ev_in_ready, c->xs_in));
  CK(cudaStreamWaitEvent(c->stream, c->ev_in_ready, 0));
  CK(launch_init_all(c->prec, c->d_desc, c->d_offs, (int)c->inst.size(), total, c->parity, c->d_in,
                     c->stream));
  CK(cudaEventRecord(c->ev_in_free, c->stream));
  c->t = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_get_fields_all_async(lbm_ctx* c, double* rho, double* ux, double* uy,
                                               int dst_is_device) {
  Range range_("lbm_get_fields_all_async");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  const long long total = c->offs.back();
  lbm_status st = ensure_scratch(c, (size_t)total);
  if (st != LBM_OK) return st;
  // (ensure_scratch has ordered this after the previous read-back)
  if (!dst_is_device) {
    st = ensure_xfer(c);
    if (st != LBM_OK) return st;
  }
  CK(launch_macro_all(c->prec, c->d_desc, c->d_offs, (int)c->inst.size(), total, c->parity,
                      c->d_rho, c->d_psi, (ux || uy) ? c->d_ux : nullptr,
                      (ux || uy) ? c->d_uy : nullptr, c->stream));
  const size_t bytes = total * sizeof(double);
  if (dst_is_device) {
    if (rho) CK(cudaMemcpyAsync(rho, c->d_rho, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (ux) CK(cudaMemcpyAsync(ux, c->d_ux, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (uy) CK(cudaMemcpyAsync(uy, c->d_uy, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return LBM_OK;
  }
  // the copies to the host run on xs_out beside the next steps on c->stream;
  // the next user of the scratch waits for ev_out_free
  CK(cudaEventRecord(c->ev_out_ready, c->stream));
  CK(cudaStreamWaitEvent(c->xs_out, c->ev_out_ready, 0));
  if (rho) CK(cudaMemcpyAsync(rho, c->d_rho, bytes, cudaMemcpyDeviceToHost, c->xs_out));
  if (ux) CK(cudaMemcpyAsync(ux, c->d_ux, bytes, cudaMemcpyDeviceToHost, c->xs_out));
  if (uy) CK(cudaMemcpyAsync(uy, c->d_uy, bytes, cudaMemcpyDeviceToHost, c->xs_out));
  CK(cudaEventRecord(c->ev_out_free, c->xs_out));
  return LBM_OK;
}

extern "C" lbm_status lbm_get_populations(lbm_ctx* c, int inst, double* f, int dst_is_device) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  const Inst& I = c->inst[inst];
  const size_t N = (size_t)I.nx * I.ny;
  st = ensure_scratch(c, N);
  if (st != LBM_OK) return st;
  double* d_f = nullptr;
  if (dst_is_device) {
    d_f = f;
  } else {
    CK(cudaMalloc(&d_f, Q * N * sizeof(double)));
  }
  cudaError_t e = launch_macro(c->prec, I.desc, c->d_desc + inst, c->parity, c->d_rho, c->d_psi,
                               nullptr, nullptr, d_f, c->stream);
  if (e == cudaSuccess && !dst_is_device)
    e = cudaMemcpyAsync(f, d_f, Q * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (!dst_is_device) cudaFree(d_f);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "get_populations: %s", cudaGetErrorString(e));
  return lbm_sync(c);
}

extern "C" lbm_status lbm_set_gw_field(lbm_ctx* c, int inst, const double* gw) {
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!gw) return fail(LBM_ERR_ARG, "gw is NULL");
  Inst& I = c->inst[inst];
  const size_t N = (size_t)I.nx * I.ny;
  for (size_t i = 0; i < N; ++i)
    if (I.solid[i]) {
      if (!isfinite(gw[i])) return fail(LBM_ERR_ARG, "non-finite G_w at node %zu", i);
      I.gw[i] = gw[i];
    }
  std::vector<double2> A;
  build_A(I, A);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(I.d_A, A.data(), N * sizeof(double2), cudaMemcpyHostToDevice));
  return LBM_OK;
}

extern "C" lbm_status lbm_set_launch(lbm_ctx* c, int bx, int h, int persistent, int graph,
                                      int stages) {
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (bx < 0 || bx > 512 || h < 0) return fail(LBM_ERR_ARG, "need 0 <= bx <= 512 and h >= 0");
  if (!(stages >= 0 && stages <= 4) && stages != 8 && stages != 16)
    return fail(LBM_ERR_ARG, "stages must be 0 (automatic), 1 (block rows), 2 (warp strips), "
                             "3 (warp strips, one row per lane), 4 (warp strips, two columns "
                             "per lane), 8 or 16 (TMA ring)");
  CK(cudaStreamSynchronize(c->stream));
  c->bx = bx;
  c->h = h;
  c->persistent = persistent != 0;
  c->use_graph = graph != 0;
  c->stages = stages;
  return build_items(c);
}

extern "C" lbm_status lbm_get_launch(const lbm_ctx* c, int* bx, int* pipeline,
                                      int* persistent) {
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  int code = c->stages_used;
  if (code == PIPE_BLOCK) code = 1;
  else if (code == PIPE_WARP) code = c->prec == LBM_FP32_SHIFTED ? 2 : 3;
  else if (code == PIPE_COLS) code = 4;
  if (c->persistent && is_warp_pipe(c->stages_used)) code = 3;  // one row per lane
  if (bx) *bx = c->bx_used;
  if (pipeline) *pipeline = code;
  if (persistent) *persistent = c->persistent;
  return LBM_OK;
}

extern "C" lbm_status lbm_diagnostics(lbm_ctx* c, int inst, double y_w, double x_ref,
                                      double d_min, lbm_diag* out) {
  Range range_("lbm_diagnostics");
  lbm_status st = check_inst(c, inst);
  if (st != LBM_OK) return st;
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  const Inst& I = c->inst[inst];
  const size_t N = (size_t)I.nx * I.ny;
  st = ensure_scratch(c, N);
  if (st != LBM_OK) return st;
  CK(launch_macro(c->prec, I.desc, c->d_desc + inst, c->parity, c->d_rho, c->d_psi, c->d_ux,
                  c->d_uy, nullptr, c->stream));
  DiagResult r;
  CK(run_diagnostics(c->diag, I.nx, I.ny, c->d_rho, c->d_ux, c->d_uy, I.d_flags,
                     0.5 * (I.p.rho_L + I.p.rho_V), y_w, x_ref, d_min, c->stream, &r));
  st = lbm_sync(c);
  memset(out, 0, sizeof *out);
  out->step = c->t;
  out->mass = r.mass;
  out->rho_max = r.rho_max;
  out->rho_min = r.rho_min;
  out->u_max = r.u_max;
  out->theta_deg = r.theta_deg;
  out->fit_rms = r.fit_rms;
  out->xc = r.xc;
  out->yc = r.yc;
  out->radius = r.radius;
  out->n_contour = r.n;
  out->status = st;
  if (st == LBM_OK && !(isfinite(r.mass) && r.rho_min > 0.0))
    out->status = st = fail(LBM_ERR_NONFINITE, "non-finite or non-positive density");
  return st;
}

extern "C" lbm_status lbm_selftest_wait_timeout(void* stream, double seconds) {
  if (!(seconds > 0.0 && seconds <= 10.0)) return fail(LBM_ERR_ARG, "seconds must be in (0, 10]");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* d = nullptr;
  CK(cudaMalloc(&d, 4 * sizeof(unsigned)));
  cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_barrier_selftest(d, (int*)(d + 1), seconds, s);
  unsigned h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
  if (h[1] & ERR_TIMEOUT) return fail(LBM_ERR_TIMEOUT, "bounded wait gave up as intended");
  return LBM_OK;
}

extern "C" lbm_status lbm_selftest_fp32_math(long n, const float* x, float* out) {
  if (!x || !out || n < 1) return fail(LBM_ERR_ARG, "need x, out and n >= 1");
  float *dx = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&dx, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 4 * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_math_selftest(dx, dout, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, 4 * n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dout);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "math selftest: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" lbm_status lbm_selftest_fp64_math(long n, const double* x, double* out) {
  if (!x || !out || n < 1) return fail(LBM_ERR_ARG, "need x, out and n >= 1");
  double *dx = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&dx, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dout, 2 * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_math_selftest64(dx, dout, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, 2 * n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dout);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "math selftest: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" lbm_status lbm_selftest_fp64_rate(double* ops_per_s) {
  if (!ops_per_s) return fail(LBM_ERR_ARG, "ops_per_s is NULL");
  cudaError_t e = measure_fp64_rate(ops_per_s);
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "fp64 probe: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// lbm_adjoint: loss L = (theta - theta_target)^2 after T steps and dL/dG_w.
// ---------------------------------------------------------------------------
namespace {

struct Crossing {
  long long ia, ib;  // edge end nodes
  double dx, dy;     // edge direction (1,0) or (0,1)
  double X, Y;       // point relative to (x_ref, y_w)
};

// the contact-angle fit of lbm_diagnostics on a host density field, with
// dtheta/drho over the fixed set of crossing edges
static bool fit_with_gradient(int nx, int ny, const std::vector<double>& rho,
                              const std::vector<uint8_t>& solid, double level, double y_w,
                              double x_ref, double d_min, double* theta, std::vector<double>* dth) {
  std::vector<Crossing> pts;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const long long i = (long long)y * nx + x;
      if (solid[i]) continue;
      for (int dir = 0; dir < 2; ++dir) {
        const int x2 = dir == 0 ? x + 1 : x, y2 = dir == 0 ? y : y + 1;
        if (dir == 1 && y2 >= ny) continue;
        const long long j = (long long)y2 * nx + (x2 % nx);
        if (solid[j]) continue;
        const double ra = rho[i], rb = rho[j];
        if ((ra >= level) == (rb >= level)) continue;
        const double t = (level - ra) / (rb - ra);
        double X = (double)x + t * (x2 - x) - x_ref;
        X -= nx * floor(X / nx + 0.5);
        const double Y = (double)y + t * (y2 - y) - y_w;
        if (Y < d_min) continue;
        pts.push_back({i, j, (double)(x2 - x), (double)(y2 - y), X, Y});
      }
    }
  if (pts.size() < 3) return false;
  double M[3][3] = {{0}}, r[3] = {0};
  for (auto& q : pts) {
    const double u[3] = {q.X, q.Y, 1.0}, z = q.X * q.X + q.Y * q.Y;
    for (int a = 0; a < 3; ++a) {
      for (int c = 0; c < 3; ++c) M[a][c] += u[a] * u[c];
      r[a] -= u[a] * z;
    }
  }
  auto det3 = [](const double A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
           A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  };
  auto solve = [&](const double b[3], double x[3]) {
    const double d = det3(M);
    for (int c = 0; c < 3; ++c) {
      double B[3][3];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) B[i][k] = k == c ? b[i] : M[i][k];
      x[c] = det3(B) / d;
    }
  };
  double p[3];
  solve(r, p);
  const double xc = -0.5 * p[0], yc = -0.5 * p[1];
  const double R = sqrt(xc * xc + yc * yc - p[2]);
  double s = yc / R;
  s = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
  *theta = 90.0 + asin(s) * (180.0 / M_PI);
  if (!dth) return true;
  // dtheta/dp for p = (D, E, F), yc = -E/2, R^2 = D^2/4 + E^2/4 - F
  const double dths = (180.0 / M_PI) / sqrt(fmax(1e-300, 1.0 - s * s));
  const double R3 = R * R * R;
  const double g[3] = {dths * (yc * xc) / (2.0 * R3), dths * (-(R * R - yc * yc) / (2.0 * R3)),
                       dths * (yc / (2.0 * R3))};
  double mu[3];
  solve(g, mu);  // M is symmetric
  dth->assign(rho.size(), 0.0);
  for (auto& q : pts) {
    const double u[3] = {q.X, q.Y, 1.0}, z = q.X * q.X + q.Y * q.Y;
    const double mu_u = mu[0] * u[0] + mu[1] * u[1] + mu[2];
    const double u_p = u[0] * p[0] + u[1] * p[1] + p[2];
    // from M p = r: dtheta = mu . (dr - dM p)
    const double dX = -mu[0] * z - 2.0 * q.X * mu_u - mu[0] * u_p - mu_u * p[0];
    const double dY = -mu[1] * z - 2.0 * q.Y * mu_u - mu[1] * u_p - mu_u * p[1];
    const double ra = rho[q.ia], rb = rho[q.ib], den = (rb - ra) * (rb - ra);
    const double dt_a = (level - rb) / den, dt_b = (ra - level) / den;
    const double dpt = dX * q.dx + dY * q.dy;
    (*dth)[q.ia] += dpt * dt_a;
    (*dth)[q.ib] += dpt * dt_b;
  }
  return true;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" lbm_status lbm_adjoint(lbm_ctx* c, long T, double theta_target, double y_w,
                                  double x_ref, double d_min, double* loss_out,
                                  double* theta_out, double* grad_gw) {
  Range range_("lbm_adjoint");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (c->inst.size() != 1) return fail(LBM_ERR_ARG, "lbm_adjoint needs a single-lattice context");
  if (c->prec != LBM_FP64) return fail(LBM_ERR_ARG, "lbm_adjoint needs LBM_FP64");
  if (c->inst[0].p.ghost == LBM_GHOST_MEAN)
    return fail(LBM_ERR_ARG, "lbm_adjoint supports the COPY, MIRROR, ZERO and SKIP ghosts");
  if (c->inst[0].p.eos != LBM_EOS_PIECEWISE_LINEAR)
    return fail(LBM_ERR_ARG, "lbm_adjoint supports the EOS of Eq. (15) only");
  if (T < 1) return fail(LBM_ERR_ARG, "T must be >= 1");
  Inst& I = c->inst[0];
  if (I.p.tau_nu_L != I.p.tau_nu_V)
    return fail(LBM_ERR_ARG, "lbm_adjoint needs tau_nu_L == tau_nu_V");
  const size_t N = (size_t)I.nx * I.ny;
  const size_t fN = Q * N;
  lbm_status st = ensure_scratch(c, N);
  if (st != LBM_OK) return st;
  CK(cudaStreamSynchronize(c->stream));
  const int saved_persistent = c->persistent;
  c->persistent = 0;
  // checkpoints every k steps: the library state (f*, F at walls) and parity
  const long k = (long)ceil(sqrt((double)T));
  const long nck = (T + k - 1) / k;
  DevBuf ck, seg[2], segrp[2], lamA, lamB, grad, scr;
  const size_t ck_one = (fN + 2 * N) * sizeof(double);
  CK(cudaMalloc(&ck.p, nck * ck_one));
  // recomputed forward states of a segment, f(t) and rho(t), psi(t), twice:
  // the reverse sweep of one segment reads one buffer while the next
  // segment is recomputed into the other
  const int nbuf = nck > 1 ? 2 : 1;
  for (int b = 0; b < nbuf; ++b) {
    CK(cudaMalloc(&seg[b].p, (size_t)k * fN * sizeof(double)));
    CK(cudaMalloc(&segrp[b].p, (size_t)k * 2 * N * sizeof(double)));
  }
  CK(cudaMalloc(&lamA.p, fN * sizeof(double)));
  CK(cudaMalloc(&lamB.p, fN * sizeof(double)));
  CK(cudaMalloc(&grad.p, N * sizeof(double)));
  CK(cudaMemsetAsync(grad.p, 0, N * sizeof(double), c->stream));
  // scratch of the reverse step
  const size_t scr_doubles = fN + 2 * N + fN + 2 * N + 2 * N + 2 * N;
  CK(cudaMalloc(&scr.p, scr_doubles * sizeof(double)));
  AdjScratch S;
  {
    double* q = (double*)scr.p;
    S.lamp = q; q += fN;
    S.lamF_bc = (double2*)q; q += 2 * N;
    S.lam_dir = q; q += fN;
    S.lam_g = (double2*)q; q += 2 * N;
    S.lam_A = (double2*)q; q += 2 * N;
    S.lam_psi_loc = q; q += N;
    S.lam_rho_loc = q; q += N;
  }
  const size_t fbytes = fN * sizeof(double), Fbytes = 2 * N * sizeof(double);
  std::vector<int> ck_parity(nck);
  auto save = [&](long ci) -> lbm_status {
    char* dst = (char*)ck.p + ci * ck_one;
    CK(cudaMemcpyAsync(dst, I.f[c->parity], fbytes, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(dst + fbytes, I.Fw[c->parity], Fbytes, cudaMemcpyDeviceToDevice, c->stream));
    ck_parity[ci] = c->parity;
    return LBM_OK;
  };
  auto restore = [&](long ci) -> lbm_status {
    const char* srcp = (const char*)ck.p + ci * ck_one;
    c->parity = ck_parity[ci];
    CK(cudaMemcpyAsync(I.f[c->parity], srcp, fbytes, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(I.Fw[c->parity], srcp + fbytes, Fbytes, cudaMemcpyDeviceToDevice, c->stream));
    return LBM_OK;
  };
  const long t0 = c->t;
  // forward pass with checkpoints (each segment's steps replayed from a
  // CUDA graph of the context)
  const int saved_graph = c->use_graph;
  c->use_graph = 1;
  for (long ci = 0; ci < nck; ++ci) {
    if ((st = save(ci)) == LBM_OK) st = lbm_step(c, std::min(k, T - ci * k));
    if (st != LBM_OK) {
      c->use_graph = saved_graph;
      c->persistent = saved_persistent;
      return st;
    }
  }
  c->use_graph = saved_graph;
  st = lbm_sync(c);
  if (st != LBM_OK) return st;
  const int final_parity = c->parity;
  const long final_t = c->t;
  // loss and its seed dL/df(T) = dL/drho(T) on every population
  std::vector<double> rho(N);
  CK(launch_macro(c->prec, I.desc, c->d_desc, c->parity, c->d_rho, c->d_psi, nullptr, nullptr,
                  nullptr, c->stream));
  CK(cudaMemcpyAsync(rho.data(), c->d_rho, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double theta = 0.0;
  std::vector<double> dth;
  if (!fit_with_gradient(I.nx, I.ny, rho, I.solid, 0.5 * (I.p.rho_L + I.p.rho_V), y_w, x_ref,
                         d_min, &theta, &dth)) {
    c->persistent = saved_persistent;
    return fail(LBM_ERR_STATE, "fewer than 3 contour points: no contact angle");
  }
  const double L = (theta - theta_target) * (theta - theta_target);
  std::vector<double> seed(fN, 0.0);
  for (size_t i = 0; i < N; ++i)
    for (int a = 0; a < Q; ++a) seed[a * N + i] = 2.0 * (theta - theta_target) * dth[i];
  CK(cudaMemcpyAsync(lamA.p, seed.data(), fbytes, cudaMemcpyHostToDevice, c->stream));
  // save the final state, then run the segments backwards
  DevBuf fin;
  CK(cudaMalloc(&fin.p, ck_one));
  CK(cudaMemcpyAsync(fin.p, I.f[final_parity], fbytes, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync((char*)fin.p + fbytes, I.Fw[final_parity], Fbytes, cudaMemcpyDeviceToDevice,
                     c->stream));
  double* lam_next = (double*)lamA.p;
  double* lam_cur = (double*)lamB.p;
  // A segment: the forward states f(t) of its len steps recomputed from the
  // restored checkpoint (context stream), then its len reverse steps (a
  // stream of their own).  The reverse sweep of segment ci runs while
  // segment ci - 1 is recomputed into the other buffer: on a small lattice
  // neither fills the GPU.  Each part is captured once per (len, parity or
  // lam orientation, buffer) and replayed from a CUDA graph: the kernels of
  // a 256 x 128 lattice last a few microseconds each.
  auto enqueue_recompute = [&](long len, int p0, int b, cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    int par = p0;
    for (long q = 0; q < len && e == cudaSuccess; ++q) {
      double* fs = (double*)seg[b].p + q * fN;
      double* rs = (double*)segrp[b].p + q * 2 * N;
      e = launch_macro(c->prec, I.desc, c->d_desc, par, rs, rs + N, nullptr, nullptr, fs, s,
                       false);
      if (e == cudaSuccess) e = launch_one_step(c, par, s);
      par ^= 1;
    }
    return e;
  };
  auto enqueue_reverse = [&](long len, int b, double* ln, double* lc,
                             cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (long q = len - 1; q >= 0 && e == cudaSuccess; --q) {
      const double* fs = (const double*)seg[b].p + q * fN;
      double* rs = (double*)segrp[b].p + q * 2 * N;
      e = launch_adjoint_step(I.desc, c->d_desc, fs, rs, rs + N, ln, lc, (double*)grad.p, S, s);
      std::swap(ln, lc);
    }
    return e;
  };
  std::map<std::tuple<int, long, int, int>, cudaGraphExec_t> graphs;
  cudaStream_t cap = nullptr, rev = nullptr;
  cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&rev, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&ev_rec[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_rev[b], cudaEventDisableTiming);
  }
  auto release = [&]() {
    if (rev) cudaStreamSynchronize(rev);
    cudaStreamSynchronize(c->stream);  // no replay still pending
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (int b = 0; b < 2; ++b) {
      if (ev_rec[b]) cudaEventDestroy(ev_rec[b]);
      if (ev_rev[b]) cudaEventDestroy(ev_rev[b]);
    }
    if (rev) cudaStreamDestroy(rev);
    if (cap) cudaStreamDestroy(cap);
  };
  // replay the graph of `key`, capturing it first with `fill`
  auto replay = [&](const std::tuple<int, long, int, int>& key, cudaStream_t s,
                    const std::function<cudaError_t(cudaStream_t)>& fill) -> cudaError_t {
    auto it = graphs.find(key);
    cudaError_t r = cudaSuccess;
    if (it == graphs.end()) {
      cudaGraph_t g = nullptr;
      r = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (r == cudaSuccess) {
        r = fill(cap);
        cudaError_t r2 = cudaStreamEndCapture(cap, &g);
        if (r == cudaSuccess) r = r2;
      }
      cudaGraphExec_t ge = nullptr;
      if (r == cudaSuccess) r = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (r != cudaSuccess) return r;
      it = graphs.emplace(key, ge).first;
    }
    return cudaGraphLaunch(it->second, s);
  };
  auto seg_len = [&](long ci) { return std::min(k, T - ci * k); };
  // recompute segment ci into buffer ci & 1 on the context stream, once the
  // reverse sweep that last read that buffer is done
  auto recompute = [&](long ci) -> cudaError_t {
    const int b = (int)(ci & 1) % nbuf;
    cudaError_t r = cudaStreamWaitEvent(c->stream, ev_rev[b], 0);
    if (r != cudaSuccess) return r;
    if (restore(ci) != LBM_OK) return cudaErrorUnknown;
    const long len = seg_len(ci);
    const int p0 = c->parity;
    r = replay(std::make_tuple(0, len, p0, b), c->stream,
               [&](cudaStream_t s) { return enqueue_recompute(len, p0, b, s); });
    if (r == cudaSuccess) r = cudaEventRecord(ev_rec[b], c->stream);
    return r;
  };
  if (e == cudaSuccess) e = recompute(nck - 1);
  for (long ci = nck - 1; ci >= 0 && e == cudaSuccess; --ci) {
    const int b = (int)(ci & 1) % nbuf;
    const long len = seg_len(ci);
    e = cudaStreamWaitEvent(rev, ev_rec[b], 0);
    const int orient = lam_next == (double*)lamA.p ? 0 : 1;
    double *ln = lam_next, *lc = lam_cur;
    if (e == cudaSuccess)
      e = replay(std::make_tuple(1, len, orient, b), rev,
                 [&](cudaStream_t s) { return enqueue_reverse(len, b, ln, lc, s); });
    if (e == cudaSuccess) e = cudaEventRecord(ev_rev[b], rev);
    if (len & 1) std::swap(lam_next, lam_cur);
    if (e == cudaSuccess && ci > 0) e = recompute(ci - 1);
  }
  // the context stream goes on after the last reverse step
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    if (ev_rev[b]) e = cudaStreamWaitEvent(c->stream, ev_rev[b], 0);
  if (e != cudaSuccess) {
    release();
    c->persistent = saved_persistent;
    return fail(LBM_ERR_CUDA, "adjoint segment: %s", cudaGetErrorString(e));
  }
  release();
  // back to the state after the forward pass
  c->parity = final_parity;
  CK(cudaMemcpyAsync(I.f[final_parity], fin.p, fbytes, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(I.Fw[final_parity], (char*)fin.p + fbytes, Fbytes, cudaMemcpyDeviceToDevice,
                     c->stream));
  c->t = final_t;
  c->persistent = saved_persistent;
  (void)t0;
  if (grad_gw)
    CK(cudaMemcpyAsync(grad_gw, grad.p, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  st = lbm_sync(c);
  if (st != LBM_OK) return st;
  if (grad_gw)
    for (size_t i = 0; i < N; ++i)
      if (!I.solid[i]) grad_gw[i] = 0.0;
  if (loss_out) *loss_out = L;
  if (theta_out) *theta_out = theta;
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume and the launch-shape autotuner.
// ---------------------------------------------------------------------------
namespace {

// FNV-1a over the bytes that define an instance
static uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

static uint64_t ctx_hash(const lbm_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &c->prec, sizeof c->prec);
  for (const auto& I : c->inst) {
    h = fnv(h, &I.nx, sizeof I.nx);
    h = fnv(h, &I.ny, sizeof I.ny);
    h = fnv(h, &I.fsi, sizeof I.fsi);
    // parameters field by field (no padding bytes)
    const lbm_params& p = I.p;
    const double dv[] = {p.eos_p[0], p.eos_p[1], p.eos_p[2], p.eos_p[3], p.eos_p[4], p.G,
                         p.sigma, p.tau_rho, p.tau_e, p.tau_zeta, p.tau_j, p.tau_q, p.tau_nu_L,
                         p.tau_nu_V, p.rho_L, p.rho_V, p.rho_ref};
    const int iv[] = {(int)p.eos, (int)p.wall, (int)p.ghost, (int)p.omega, (int)p.prec,
                      (int)p.visc};
    h = fnv(h, dv, sizeof dv);
    h = fnv(h, iv, sizeof iv);
    h = fnv(h, I.solid.data(), I.solid.size());
    h = fnv(h, I.gw.data(), I.gw.size() * sizeof(double));
  }
  return h;
}

const char kMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};

}  // namespace

extern "C" lbm_status lbm_save(lbm_ctx* c, const char* path) {
  Range range_("lbm_save");
  if (!c || !path) return fail(LBM_ERR_ARG, "ctx and path are required");
  lbm_status st = lbm_sync(c);
  if (st != LBM_OK) return st;
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(LBM_ERR_ARG, "cannot open %s for writing", path);
  const uint64_t h = ctx_hash(c);
  const int64_t hdr[4] = {(int64_t)c->inst.size(), (int64_t)c->t, (int64_t)c->parity,
                          (int64_t)c->prec};
  bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(&h, sizeof h, 1, fp) == 1 &&
            fwrite(hdr, sizeof hdr, 1, fp) == 1;
  std::vector<char> buf;
  for (auto& I : c->inst) {
    if (!ok) break;
    const size_t N = (size_t)I.nx * I.ny, ts = tsize(c->prec);
    const size_t fb = Q * N * ts, Fb = 2 * N * ts;
    buf.resize(fb + Fb);
    cudaError_t e = cudaMemcpy(buf.data(), I.f[c->parity], fb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + fb, I.Fw[c->parity], Fb, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      fclose(fp);
      return fail(LBM_ERR_CUDA, "lbm_save: %s", cudaGetErrorString(e));
    }
    ok = fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  }
  ok = (fclose(fp) == 0) && ok;
  return ok ? LBM_OK : fail(LBM_ERR_ARG, "lbm_save: write to %s failed", path);
}

extern "C" lbm_status lbm_load(lbm_ctx* c, const char* path) {
  Range range_("lbm_load");
  if (!c || !path) return fail(LBM_ERR_ARG, "ctx and path are required");
  CK(cudaStreamSynchronize(c->stream));
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(LBM_ERR_ARG, "cannot open %s", path);
  char magic[8];
  uint64_t h = 0;
  int64_t hdr[4];
  bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kMagic, 8) == 0 &&
            fread(&h, sizeof h, 1, fp) == 1 && fread(hdr, sizeof hdr, 1, fp) == 1;
  if (!ok || h != ctx_hash(c) || hdr[0] != (int64_t)c->inst.size() || hdr[3] != c->prec ||
      (hdr[2] != 0 && hdr[2] != 1)) {
    fclose(fp);
    return fail(LBM_ERR_ARG, "lbm_load: %s was not saved from a context with these lattices, "
                             "parameters, masks and G_w", path);
  }
  std::vector<char> buf;
  const int parity = (int)hdr[2];
  for (auto& I : c->inst) {
    const size_t N = (size_t)I.nx * I.ny, ts = tsize(c->prec);
    const size_t fb = Q * N * ts, Fb = 2 * N * ts;
    buf.resize(fb + Fb);
    if (fread(buf.data(), 1, buf.size(), fp) != buf.size()) {
      fclose(fp);
      return fail(LBM_ERR_ARG, "lbm_load: %s is truncated", path);
    }
    cudaError_t e = cudaMemcpy(I.f[parity], buf.data(), fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(I.Fw[parity], buf.data() + fb, Fb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      fclose(fp);
      return fail(LBM_ERR_CUDA, "lbm_load: %s", cudaGetErrorString(e));
    }
  }
  fclose(fp);
  c->parity = parity;
  c->t = (long)hdr[1];
  return LBM_OK;
}

extern "C" lbm_status lbm_autotune(lbm_ctx* c, int steps, int* bx_out, int* h_out,
                                   int* stages_out, double* ms_out) {
  Range range_("lbm_autotune");
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (steps < 1) return fail(LBM_ERR_ARG, "steps must be >= 1");
  lbm_status st = lbm_sync(c);
  if (st != LBM_OK) return st;
  // keep the state: every trial starts from it and it is put back at the end
  std::vector<void*> keep;
  auto cleanup = [&]() {
    for (void* p : keep) cudaFree(p);
  };
  for (auto& I : c->inst) {
    const size_t N = (size_t)I.nx * I.ny, ts = tsize(c->prec);
    void *pf = nullptr, *pF = nullptr;
    if (cudaMalloc(&pf, Q * N * ts) != cudaSuccess || cudaMalloc(&pF, 2 * N * ts) != cudaSuccess) {
      cudaFree(pf);
      cleanup();
      return fail(LBM_ERR_OOM, "lbm_autotune: no room for a copy of the state");
    }
    keep.push_back(pf);
    keep.push_back(pF);
    cudaMemcpy(pf, I.f[c->parity], Q * N * ts, cudaMemcpyDeviceToDevice);
    cudaMemcpy(pF, I.Fw[c->parity], 2 * N * ts, cudaMemcpyDeviceToDevice);
  }
  const int parity0 = c->parity;
  const long t0 = c->t;
  auto put_back = [&]() {
    c->parity = parity0;
    c->t = t0;
    for (size_t k = 0; k < c->inst.size(); ++k) {
      auto& I = c->inst[k];
      const size_t N = (size_t)I.nx * I.ny, ts = tsize(c->prec);
      cudaMemcpy(I.f[parity0], keep[2 * k], Q * N * ts, cudaMemcpyDeviceToDevice);
      cudaMemcpy(I.Fw[parity0], keep[2 * k + 1], 2 * N * ts, cudaMemcpyDeviceToDevice);
    }
  };
  struct Cand {
    int bx, h, stages, persistent;
  };
  // FP32 warp strips with two columns per lane, warp strips (two rows per
  // lane with FP32 storage: even h), warp strips one row per lane, block
  // rows, TMA block rows, each launched per step; then the persistent warp
  // strips (one parameter set only)
  std::vector<Cand> cands = {
      {128, 0, 4, 0},  {128, 8, 4, 0},  {128, 16, 4, 0}, {128, 32, 4, 0}, {64, 0, 4, 0},
      {256, 0, 4, 0},  {128, 0, 2, 0},  {128, 4, 2, 0},  {128, 8, 2, 0},  {128, 16, 2, 0},
      {128, 24, 2, 0}, {128, 32, 2, 0}, {64, 32, 2, 0},  {256, 32, 2, 0}, {256, 0, 3, 0},
      {256, 8, 3, 0},  {256, 25, 3, 0}, {256, 32, 3, 0}, {128, 32, 3, 0}, {224, 32, 1, 0},
      {224, 50, 1, 0}, {416, 50, 1, 0}, {224, 50, 8, 0}, {416, 50, 8, 0}, {64, 0, 4, 1},
      {128, 0, 4, 1},  {256, 0, 3, 1}};
  const int saved[5] = {c->bx, c->h, c->persistent, c->use_graph, c->stages};
  c->persistent = 0;
  c->use_graph = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  Cand bestc = cands[0];
  for (const Cand& q : cands) {
    c->bx = q.bx;
    c->h = q.h;
    c->stages = q.stages;
    c->persistent = q.persistent;
    if (build_items(c) != LBM_OK) continue;
    if (q.stages >= 8 && c->stages_used < 8) continue;  // TMA not applicable here
    if (q.stages == 4 && c->stages_used != PIPE_COLS) continue;  // widths not multiples of 4
    put_back();
    if (lbm_step(c, 2) != LBM_OK) continue;
    cudaEventRecord(e0, c->stream);
    if (lbm_step(c, steps) != LBM_OK) continue;
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bestc = q;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  put_back();
  c->bx = bestc.bx;
  c->h = bestc.h;
  c->stages = bestc.stages;
  c->persistent = bestc.persistent;
  c->use_graph = saved[3];
  st = build_items(c);
  cleanup();
  if (st != LBM_OK) return st;
  st = lbm_sync(c);
  if (st != LBM_OK) return st;
  if (bx_out) *bx_out = bestc.bx;
  if (h_out) *h_out = bestc.h;
  if (stages_out) *stages_out = bestc.stages;
  if (ms_out) *ms_out = best / steps;
  return LBM_OK;
}

// The strips of one nx x ny lattice in h-row segments (h > 0) and their
// dependency lists as the persistent warp strips use them, on the host only.
extern "C" lbm_status lbm_get_work_items(const lbm_ctx* c, int* n_items, int* items4, int* off,
                                         int* nbr, int cap, int* n_nbr) {
  if (!c) return fail(LBM_ERR_ARG, "ctx is NULL");
  if (!n_items || !n_nbr) return fail(LBM_ERR_ARG, "n_items and n_nbr must not be NULL");
  *n_items = (int)c->h_items.size();
  *n_nbr = (int)c->h_nbr.size();
  if (!items4 || !off || !nbr) return LBM_OK;  // sizes only
  if ((long long)c->h_items.size() * 4 > cap || (long long)c->h_nbr.size() > cap ||
      (long long)c->h_nbr_off.size() > cap)
    return fail(LBM_ERR_ARG, "cap too small: %d items, %d neighbours", *n_items, *n_nbr);
  for (size_t i = 0; i < c->h_items.size(); ++i) {
    const WorkItem& w = c->h_items[i];
    items4[4 * i] = w.inst;
    items4[4 * i + 1] = w.x0;
    items4[4 * i + 2] = w.y0;
    items4[4 * i + 3] = w.y1;
  }
  for (size_t i = 0; i < c->h_nbr_off.size(); ++i) off[i] = c->h_nbr_off[i];
  for (size_t i = 0; i < c->h_nbr.size(); ++i) nbr[i] = c->h_nbr[i];
  return LBM_OK;
}

extern "C" lbm_status lbm_strip_neighbours(int nx, int ny, int h, int* n_items, int* items3,
                                           int* off, int* nbr, int cap, int* n_nbr) {
  if (nx < 3 || ny < 3 || h < 1) return fail(LBM_ERR_ARG, "need nx, ny >= 3 and h >= 1");
  if (!n_items || !n_nbr) return fail(LBM_ERR_ARG, "n_items and n_nbr must not be NULL");
  const int cols = 30;  // the columns of one warp strip
  std::vector<WorkItem> items;
  for (int y0 = 0; y0 < ny; y0 += h)
    for (int x0 = 0; x0 < nx; x0 += cols) items.push_back({0, x0, y0, std::min(ny, y0 + h)});
  std::vector<int> o, nb;
  strip_neighbours(items, {nx, ny}, cols, o, nb);
  *n_items = (int)items.size();
  *n_nbr = (int)nb.size();
  if (!items3 || !off || !nbr) return LBM_OK;  // sizes only
  if ((long long)items.size() * 3 > cap || (long long)nb.size() > cap ||
      (long long)o.size() > cap)
    return fail(LBM_ERR_ARG, "cap too small: %d items, %d neighbours", (int)items.size(),
                (int)nb.size());
  for (size_t i = 0; i < items.size(); ++i) {
    items3[3 * i] = items[i].x0;
    items3[3 * i + 1] = items[i].y0;
    items3[3 * i + 2] = items[i].y1;
  }
  for (size_t i = 0; i < o.size(); ++i) off[i] = o[i];
  for (size_t i = 0; i < nb.size(); ++i) nbr[i] = nb[i];
  return LBM_OK;
}
