// Diagnostics kernels: density extrema, mass, max |v| and the contact angle
// (circle fitted to the rho = (rho_L + rho_V)/2 contour, Sec. III.A).
//
// Contour points: on every edge between two fluid nodes ((x,y)-(x+1,y) with
// periodic x, (x,y)-(x,y+1) without crossing the y seam) where rho crosses
// the level, the linearly interpolated crossing; x is unwrapped about x_ref
// into [-nx/2, nx/2) and points with y - y_w < d_min are dropped.  The
// algebraic circle x^2 + y^2 + D x + E y + F = 0 is fitted by least squares;
// theta = 90 deg + asin((y_c - y_w) / R).
#include <math.h>
#include <string.h>

#include <mutex>

#include "lbm.h"
#include "lbm_diag.cuh"
#include "lbm_internal.cuh"

namespace lbm {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// crossing on the edge from node i to node j; returns false if none
__device__ __forceinline__ bool crossing(double ra, double rb, double level, double xa, double ya,
                                         double dx, double dy, int nx, double x_ref, double y_w,
                                         double d_min, double& X, double& Y) {
  if ((ra >= level) == (rb >= level)) return false;
  const double t = (level - ra) / (rb - ra);
  X = xa + t * dx - x_ref;
  X -= nx * floor(X / nx + 0.5);
  Y = ya + t * dy - y_w;
  return Y >= d_min;
}

// solid test of node i: the library's node flags, or a plain 0/1 mask
// (NULL = no solid node)
__device__ __forceinline__ bool is_solid(const uint16_t* flags, long long i) {
  return (flags[i] & NF_SELF_SOLID) != 0;
}
__device__ __forceinline__ bool is_solid(const uint8_t* mask, long long i) {
  return mask != nullptr && mask[i] != 0;
}

// Spreading (contact) radius along one row (Sec. III.A, Fig. 7): from the
// node xi, walk right and left to the first node below the level; the
// crossing is interpolated linearly between that node and the one before
// it.  One thread: a row holds at most a few thousand nodes and the call is
// a diagnostic taken every few steps.
__global__ void k_contact_scan(const double* __restrict__ row, int nx, double level, int xi,
                               double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!(row[xi] >= level)) {
    out[0] = 0.0;  // the droplet does not touch the row at xi
    return;
  }
  double xr = -1.0, xl = -1.0;
  for (int k = 0; k < nx; ++k) {
    const double a = row[(xi + k) % nx], b = row[(xi + k + 1) % nx];
    if (b < level) {
      xr = k + (level - a) / (b - a);
      break;
    }
  }
  for (int k = 0; k < nx; ++k) {
    const double a = row[((xi - k) % nx + nx) % nx], b = row[((xi - k - 1) % nx + nx) % nx];
    if (b < level) {
      xl = k + (level - a) / (b - a);
      break;
    }
  }
  out[0] = (xr < 0.0 || xl < 0.0) ? 0.5 * nx : 0.5 * (xr + xl);
}

cudaError_t launch_contact_scan(const double* d_row, int nx, double level, int xi, double* d_out,
                                cudaStream_t s) {
  k_contact_scan<<<1, 32, 0, s>>>(d_row, nx, level, xi, d_out);
  return cudaGetLastError();
}

// mode 0: statistics and fit sums; mode 1: sum of squared radial residuals
template <int MODE, typename MaskT>
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag(int nx, int ny, const double* __restrict__ rho, const double* __restrict__ ux,
           const double* __restrict__ uy, const MaskT* __restrict__ flags, double level,
           double y_w, double x_ref, double d_min, double xc, double yc, double R,
           double* __restrict__ part) {
  const long long N = (long long)nx * ny;
  double acc[DIAG_W];
#pragma unroll
  for (int k = 0; k < DIAG_W; ++k) acc[k] = 0.0;
  acc[1] = -INFINITY;
  acc[2] = INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    if (is_solid(flags, i)) continue;
    const int x = (int)(i % nx), y = (int)(i / nx);
    const double ra = rho[i];
    if (MODE == 0) {
      acc[0] += ra;
      acc[1] = fmax(acc[1], ra);
      acc[2] = fmin(acc[2], ra);
      // a NaN anywhere must surface: fmax/fmin drop NaN, so count it in slot 15
      if (!(ra == ra)) acc[15] += 1.0;
      const double u2 = ux[i] * ux[i] + uy[i] * uy[i];
      acc[3] = fmax(acc[3], u2);
      if (!(u2 == u2)) acc[15] += 1.0;
    }
    for (int dir = 0; dir < 2; ++dir) {
      long long j;
      if (dir == 0) {
        j = (long long)y * nx + (x + 1 == nx ? 0 : x + 1);
      } else {
        if (y + 1 >= ny) continue;
        j = i + nx;
      }
      if (is_solid(flags, j)) continue;
      double X, Y;
      if (!crossing(ra, rho[j], level, (double)x, (double)y, dir == 0 ? 1.0 : 0.0,
                    dir == 0 ? 0.0 : 1.0, nx, x_ref, y_w, d_min, X, Y))
        continue;
      if (MODE == 0) {
        const double r2 = X * X + Y * Y;
        acc[4] += 1.0;
        acc[5] += X;
        acc[6] += Y;
        acc[7] += X * X;
        acc[8] += X * Y;
        acc[9] += Y * Y;
        acc[10] += X * r2;
        acc[11] += Y * r2;
        acc[12] += r2;
      } else {
        const double dr = sqrt((X - xc) * (X - xc) + (Y - yc) * (Y - yc)) - R;
        acc[14] += dr * dr;
      }
    }
  }
  // block reduction: warp shuffles, then one warp over the warp results
  __shared__ double sh[DIAG_THREADS / 32][DIAG_W];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < DIAG_W; ++k) {
    double v = k == 1 ? warp_max(acc[k]) : (k == 2 || k == 3 ? (k == 2 ? warp_min(acc[k]) : warp_max(acc[k])) : warp_sum(acc[k]));
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_W) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < DIAG_THREADS / 32; ++w) {
      const double u = sh[w][k];
      v = k == 1 || k == 3 ? fmax(v, u) : (k == 2 ? fmin(v, u) : v + u);
    }
    part[blockIdx.x * DIAG_W + k] = v;
  }
}

// fixed-order reduction of the block partials (deterministic for a given
// number of blocks): warp k reduces quantity k, lane l the partials l,
// l + 32, ... in order, then the 32 lane results in a fixed shuffle tree
constexpr int DIAG_FINAL_THREADS = DIAG_W * 32;
__global__ void __launch_bounds__(DIAG_FINAL_THREADS)
    k_diag_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= DIAG_W) return;
  const bool is_max = k == 1 || k == 3, is_min = k == 2;
  auto op = [&](double a, double b) { return is_max ? fmax(a, b) : (is_min ? fmin(a, b) : a + b); };
  double v = is_max ? -INFINITY : (is_min ? INFINITY : 0.0);
  for (int b = lane; b < nblocks; b += 32) v = op(v, part[b * DIAG_W + k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) out[k] = v;
}

static void solve3(const double A[3][3], const double b[3], double x[3]) {
  auto det3 = [](const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  };
  const double d = det3(A);
  for (int c = 0; c < 3; ++c) {
    double B[3][3];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) B[r][k] = (k == c) ? b[r] : A[r][k];
    x[c] = det3(B) / d;
  }
}

template <typename MaskT>
static cudaError_t diagnostics_into_t(double* part, double* out, double* h, int nx, int ny,
                                      const double* rho, const double* ux, const double* uy,
                                      const MaskT* flags, double level, double y_w,
                                      double x_ref, double d_min, cudaStream_t s,
                                      DiagResult* r) {
  const long long N = (long long)nx * ny;
  int blocks = (int)((N + DIAG_THREADS - 1) / DIAG_THREADS);
  if (blocks > DIAG_BLOCKS) blocks = DIAG_BLOCKS;
  k_diag<0, MaskT><<<blocks, DIAG_THREADS, 0, s>>>(nx, ny, rho, ux, uy, flags, level, y_w,
                                                   x_ref, d_min, 0.0, 0.0, 0.0, part);
  k_diag_final<<<1, DIAG_FINAL_THREADS, 0, s>>>(part, blocks, out);
  cudaError_t e = cudaMemcpyAsync(h, out, DIAG_W * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  r->mass = h[0];
  r->rho_max = h[15] > 0 ? NAN : h[1];
  r->rho_min = h[15] > 0 ? NAN : h[2];
  r->u_max = h[15] > 0 ? NAN : sqrt(h[3]);
  r->n = (int)h[4];
  r->theta_deg = r->fit_rms = r->xc = r->yc = r->radius = NAN;
  if (r->n < 3) return cudaSuccess;
  // normal equations of min sum (X^2 + Y^2 + D X + E Y + F)^2
  const double A[3][3] = {{h[7], h[8], h[5]}, {h[8], h[9], h[6]}, {h[5], h[6], h[4]}};
  const double b[3] = {-h[10], -h[11], -h[12]};
  double sol[3];
  solve3(A, b, sol);
  const double xc = -0.5 * sol[0], yc = -0.5 * sol[1];
  const double R = sqrt(xc * xc + yc * yc - sol[2]);
  double ratio = yc / R;
  ratio = ratio > 1.0 ? 1.0 : (ratio < -1.0 ? -1.0 : ratio);
  r->theta_deg = 90.0 + asin(ratio) * (180.0 / M_PI);
  r->xc = xc + x_ref;
  r->yc = yc + y_w;
  r->radius = R;
  k_diag<1, MaskT><<<blocks, DIAG_THREADS, 0, s>>>(nx, ny, rho, ux, uy, flags, level, y_w,
                                                   x_ref, d_min, xc, yc, R, part);
  k_diag_final<<<1, DIAG_FINAL_THREADS, 0, s>>>(part, blocks, out);
  e = cudaMemcpyAsync(h, out, DIAG_W * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  r->fit_rms = sqrt(h[14] / r->n);
  return cudaGetLastError();
}

cudaError_t diagnostics_into(double* part, double* out, double* h, int nx, int ny,
                             const double* rho, const double* ux, const double* uy,
                             const uint16_t* flags, double level, double y_w, double x_ref,
                             double d_min, cudaStream_t s, DiagResult* r) {
  return diagnostics_into_t<uint16_t>(part, out, h, nx, ny, rho, ux, uy, flags, level, y_w, x_ref,
                                      d_min, s, r);
}

cudaError_t run_diagnostics(DiagScratch& sc, int nx, int ny, const double* rho, const double* ux,
                            const double* uy, const uint16_t* flags, double level, double y_w,
                            double x_ref, double d_min, cudaStream_t s, DiagResult* r) {
  cudaError_t e = cudaSuccess;
  if (!sc.d_part) e = cudaMalloc(&sc.d_part, DIAG_BLOCKS * DIAG_W * sizeof(double));
  if (e == cudaSuccess && !sc.d_out) e = cudaMalloc(&sc.d_out, DIAG_W * sizeof(double));
  if (e == cudaSuccess && !sc.h_out) e = cudaMallocHost(&sc.h_out, DIAG_W * sizeof(double));
  if (e != cudaSuccess) return e;
  return diagnostics_into(sc.d_part, sc.d_out, sc.h_out, nx, ny, rho, ux, uy, flags, level, y_w,
                          x_ref, d_min, s, r);
}

void diag_free(DiagScratch& sc) {
  cudaFree(sc.d_part);
  cudaFree(sc.d_out);
  cudaFreeHost(sc.h_out);
  sc = DiagScratch{};
}

}  // namespace lbm

// ---------------------------------------------------------------------------
// Diagnostics without allocation (lbm_diagnostics_noalloc).
//
// The block partials and the reduced result live in one file-scope device
// array instead of memory obtained from cudaMalloc.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress (with that device current) and
// keeps it; every later call on that device reuses it.  Each call overwrites
// every partial it reads, so nothing needs clearing between calls, but all
// calls on a device share the array: calls whose kernels overlap on the GPU
// (other streams, other host threads) race and must be serialised by the
// caller.
// ---------------------------------------------------------------------------
namespace lbm {

constexpr int NOALLOC_MAX_DEVICES = 64;
static __device__ __align__(256) double g_noalloc_scratch[DIAG_BLOCKS * DIAG_W + DIAG_W];
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace lbm

extern "C" lbm_status lbm_diagnostics_noalloc(int nx, int ny, const double* rho,
                                              const double* ux, const double* uy,
                                              const uint8_t* solid, double level, double y_w,
                                              double x_ref, double d_min, void* stream,
                                              lbm_diag* out) {
  using namespace lbm;
  if (!out) return set_error(LBM_ERR_ARG, "lbm_diagnostics_noalloc: out is NULL");
  memset(out, 0, sizeof *out);
  if (!rho || !ux || !uy)
    return set_error(LBM_ERR_ARG, "lbm_diagnostics_noalloc: rho, ux and uy are required");
  if (nx < 1 || ny < 1 || (long long)nx * ny > LBM_NOALLOC_MAX_NODES)
    return set_error(LBM_ERR_ARG,
                     "lbm_diagnostics_noalloc: nx * ny must be in [1, %lld] (got %d x %d)",
                     (long long)LBM_NOALLOC_MAX_NODES, nx, ny);
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess)
    return set_error(LBM_ERR_CUDA, "lbm_diagnostics_noalloc: scratch address: %s",
                     cudaGetErrorString(e));
  double h[DIAG_W];
  DiagResult r;
  e = diagnostics_into_t<uint8_t>(scratch, scratch + DIAG_BLOCKS * DIAG_W, h, nx, ny, rho, ux, uy,
                                  solid, level, y_w, x_ref, d_min, (cudaStream_t)stream, &r);
  if (e != cudaSuccess)
    return set_error(LBM_ERR_CUDA, "lbm_diagnostics_noalloc: %s", cudaGetErrorString(e));
  out->step = -1;
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
  out->status = LBM_OK;
  if (!(r.mass == r.mass) || !(r.rho_min > 0.0)) {
    out->status = LBM_ERR_NONFINITE;
    return set_error(LBM_ERR_NONFINITE, "lbm_diagnostics_noalloc: non-finite or non-positive density");
  }
  return LBM_OK;
}
