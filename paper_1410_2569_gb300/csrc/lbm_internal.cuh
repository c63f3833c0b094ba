// Internal declarations of liblbm (not part of the C ABI).
//
// Device data of one lattice instance:
//   f[2]      two population lattices, [9][ny][nx] of T (double, or float
//             holding f - w_alpha rho_ref); the step pulls from f[p] and
//             writes post-collision populations f* to f[p^1].
//   flags     per node uint16 (bits below); rows whose flags are all zero
//             are marked plain in row_plain and take the fast path.
//   A         per node wall vector A(x) = sum_alpha omega_alpha G_w(x+e_alpha)
//             s(x+e_alpha) e_alpha (zero away from walls); the fluid-solid
//             force is F_ads = -X(x) A(x) with X = rho, psi or psi^2
//             (Eqs. (10), (11), (14)).
//   Fw[2]     per node force of the last collision, read by the wall rule of
//             Sec. III.A when the next step pulls into a wall node.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

constexpr int Q = 9;

// node flags
enum : uint16_t {
  NF_SRC_SOLID = 0x01FF,  // bit a: the pull source x - e_a is solid
  NF_SELF_SOLID = 1u << 9,
  NF_NEQ_BOTTOM = 1u << 10,  // fluid, solid directly below, NEQ wall rule
  NF_NEQ_TOP = 1u << 11,     // fluid, solid directly above, mirrored rule
  NF_GHOST_UP = 1u << 12,    // solid, fluid directly above (ghost psi source)
  NF_GHOST_DOWN = 1u << 13,  // solid, fluid directly below
  NF_GHOST_RIGHT = 1u << 14, // solid, fluid at x + 1 (MEAN ghost only)
  NF_GHOST_LEFT = 1u << 15,  // solid, fluid at x - 1 (MEAN ghost only)
};

template <typename T>
struct Consts {
  T G;                 // Eq. (7)
  T s_e, s_z, s_q;     // 1/tau_e, 1/tau_zeta, 1/tau_q of Eq. (2)
  T h_e, h_z, h_q;     // 1 - s/2
  T c_e, c_z;          // (1 - s/2) * 12 sigma G^2 / (tau - 1/2), Eq. (9)
  T s_nu, h_nu;        // constant-viscosity rate and 1 - s_nu/2 (adjoint)
  T rho_ref;           // storage shift (0 in FP64)
  // the relaxation of Eq. (4) with the diagonal of M^-1 folded in:
  // E = ke_v vF + ke_g g2 - ke_n ne, P = -(kz_v vF + kz_g g2 + kz_n nz),
  // QX = -kq (qx + mx) - kq_F Fx (the shear rates are in Visc)
  T ke_v, ke_g, ke_n, kz_v, kz_g, kz_n, kq, kq_F;
};

// Shear viscosity of one instance: XX = hnu2 (..) - knu (..), XY = hnu4 (..)
// - knu (..) with knu = s_nu / 4, hnu2 = (1 - s_nu / 2) / 2, hnu4 = hnu2 / 2
// (the diagonal of M^-1 folded in), s_nu = 1 / tau_nu_L; or, with a
// viscosity ratio, tau_nu(rho) = tauV + (rho - rho_V) dtau clamped to
// [tau_lo, tau_hi] and the rates formed per node.
// With the dynamic viscosity linear in rho (LBM_VISC_MU_LINEAR), tau_nu(rho)
// = 1/2 + (muV + (rho - rho_V) dmu) / (rho cs^2), clamped likewise.
template <typename T>
struct Visc {
  T knu, hnu2, hnu4;
  T tauV, dtau, tau_lo, tau_hi, rho_V;
  T muV3, dmu3;  // 3 mu_V and 3 dmu (mu / cs^2 with cs^2 = 1/3)
};

// The part of an instance descriptor fixed by its lbm_params.  The step
// kernels take it by value as a kernel parameter (one launch per distinct
// parameter set of a batch): warp-uniform constants then sit in the constant
// bank and enter the arithmetic as operands, without loads or registers.
struct __align__(16) PhysDesc {
  int wall, ghost;
  int omega_cs2w;  // omega_alpha = cs^2 w_alpha (else w_alpha) in A(x)
  int eos;         // lbm_eos
  // Carnahan-Starling option: p = rho RT (1 + e + e^2 - e^3) / (1 - e)^3 -
  // a rho^2, e = b rho / 4; psi^2 = cs_g (rho / 3 - p) with cs_g = 2 / |G|
  double cs_a, cs_b, cs_RT, cs_g;
  // Eq. (15) as psi^2 = a rho + b per branch (G < 0, c = 1)
  double rho1, rho2, aV, aM, bM, aL, bL;
  // the same as unevaluated FP32 pairs (hi, lo): per branch {a_hi, a_lo,
  // b_hi, b_lo}; thresholds {rho1_hi, rho1_lo, rho2_hi, rho2_lo}
  float eosf[3][4];
  float thrf[4];
  Consts<double> cd;
  Consts<float> cf;
};

struct __align__(16) InstDesc {
  int nx, ny;
  int fsi;
  int var_nu;  // 0: one viscosity; 1: tau_nu linear in rho; 2: mu linear in rho
  long long plane;  // nx * ny
  void* f[2];
  const uint16_t* flags;
  const uint8_t* row_plain;
  const double2* A;
  void* Fw[2];
  int* err;  // latched device error bits
  Visc<double> vd;
  Visc<float> vf;
  PhysDesc ph;  // read by the kernels outside the step (init, fields, adjoint)
};

// bytes of InstDesc in front of ph: all that the step kernels read of it
constexpr size_t INST_HEAD_BYTES = offsetof(InstDesc, ph);
static_assert(INST_HEAD_BYTES % 16 == 0, "the head is copied as 16-byte words");

struct WorkItem {
  int inst, x0, y0, y1;
};

enum : int { ERR_NONFINITE = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

// Index checks of the checked build (compiled with -DLBM_BOUNDS_CHECK into
// liblbm_check.so): every global and shared-memory index of the step
// kernels is tested against its buffer before the access; a bad index
// latches ERR_BOUNDS in *err and the access is skipped (a load gives 0), so
// nothing traps.  In the normal build the test is the constant true.
#ifdef LBM_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(long long i, long long n, int* err) {
  if (i >= 0 && i < n) return true;
  atomicOr(err, ERR_BOUNDS);
  return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, int*) { return true; }
#endif

// step pipelines (launch_step's `stages` argument): block rows with register
// prefetch, warp strips (two rows per lane with FP32 storage, one otherwise),
// warp strips with one row per lane, FP32 warp strips with two columns per
// lane (every lattice width a multiple of 4), or block rows with a TMA ring
// of 8 / 16 stages
enum : int { PIPE_BLOCK = 0, PIPE_WARP = 2, PIPE_WARP1 = 3, PIPE_COLS = 4 };
inline bool is_warp_pipe(int S) { return S == PIPE_WARP || S == PIPE_WARP1; }

// D2Q9 weights of the equilibrium
__host__ __device__ constexpr double w_eq(int a) {
  return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// shared memory of the TMA-pipelined FP32 step for bx threads and S stages
size_t tma_smem_bytes(int bx, int S);

// scratch of one reverse step (lbm_adjoint.cu), FP64, N nodes
struct AdjScratch {
  double* lamp = nullptr;  // [9][N]
  double2* lamF_bc = nullptr;
  double* lam_dir = nullptr;  // [9][N]
  double2 *lam_g = nullptr, *lam_A = nullptr;
  double *lam_psi_loc = nullptr, *lam_rho_loc = nullptr;
};
// one reverse step from the forward state f(t) with its rho and psi on
// fluid nodes, as launch_macro gives them with ghost = false (the step fills
// the ghost psi of the solid nodes in place)
cudaError_t launch_adjoint_step(const InstDesc& h, const InstDesc* d_inst, const double* f,
                                const double* rho, double* psi, const double* lam_next,
                                double* lam_out, double* grad, AdjScratch& s, cudaStream_t st);

// FP64 pipe throughput of the current device, DFMA instructions per second
// (lbm_kernels.cu)
cudaError_t measure_fp64_rate(double* ops_per_s);

// FP32 reciprocal / square root self-test (lbm_kernels.cu)
cudaError_t launch_math_selftest(const float* d_x, float* d_out, long n, cudaStream_t s);
// FP64 reciprocal self-test (lbm_kernels.cu)
cudaError_t launch_math_selftest64(const double* d_x, double* d_out, long n, cudaStream_t s);

// records the calling thread's lbm_last_error() message and returns s
lbm_status set_error(lbm_status s, const char* fmt, ...);

// launchers (lbm_kernels.cu)
cudaError_t launch_step(int prec, const PhysDesc& ph, const InstDesc* d_inst,
                        const WorkItem* d_items, int n_items, int parity, int bx, int stages,
                        cudaStream_t s);
cudaError_t launch_step_persistent(int prec, const PhysDesc& ph, const InstDesc* d_inst,
                                   const WorkItem* d_items,
                                   int n_items, int parity0, long n_steps, int bx, int stages,
                                   unsigned* d_barrier, cudaStream_t s);
int persistent_max_blocks(int prec, int bx, int stages);
// warp strips (one row per lane, or the FP32 column pairs) for n steps in one
// cooperative launch: item
// i of a step starts when the items nbr[nbr_off[i] .. nbr_off[i+1]) have
// finished the previous step (done: n_items counters, zeroed here first;
// err: the kernel's error word, ERR_TIMEOUT when a wait gave up)
// pipe: PIPE_COLS for the FP32 column-pair strips (60-column items), else
// one row per lane (30-column items)
cudaError_t launch_step_dataflow(int prec, const PhysDesc& ph, const InstDesc* d_inst,
                                 const WorkItem* d_items, const int* d_nbr_off, const int* d_nbr,
                                 int n_items, int parity0, long n_steps, int bx, int pipe,
                                 unsigned* d_done, int* d_err, cudaStream_t s);
cudaError_t launch_barrier_selftest(unsigned* d_bar, int* d_err, double seconds, cudaStream_t s);
cudaError_t launch_init(int prec, const InstDesc& h_inst, const InstDesc* d_inst, int parity,
                        const double* d_rho0, cudaStream_t s);
cudaError_t launch_row_rho(int prec, const InstDesc& h_inst, const InstDesc* d_inst, int parity,
                           int row, double* d_out, cudaStream_t s);
// contact radius from one row of rho (lbm_diag.cu); writes out[0]
cudaError_t launch_contact_scan(const double* d_row, int nx, double level, int xi, double* d_out,
                                cudaStream_t s);
// the whole batch at once: instance k's nodes are [offs[k], offs[k+1]) of
// the concatenated fields, total = offs[n]
cudaError_t launch_init_all(int prec, const InstDesc* d_inst, const long long* d_offs, int n,
                            long long total, int parity, const double* d_rho0, cudaStream_t s);
cudaError_t launch_macro_all(int prec, const InstDesc* d_inst, const long long* d_offs, int n,
                             long long total, int parity, double* d_rho, double* d_psi,
                             double* d_ux, double* d_uy, cudaStream_t s);
// ghost = false leaves psi on solid nodes unset (the adjoint fills it in its
// reverse step)
cudaError_t launch_macro(int prec, const InstDesc& h_inst, const InstDesc* d_inst, int parity,
                         double* d_rho, double* d_psi, double* d_ux, double* d_uy, double* d_f,
                         cudaStream_t s, bool ghost = true);
}  // namespace lbm
