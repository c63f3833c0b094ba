// Diagnostics of one lattice (Sec. III.B max/min densities, Sec. III.C
// spurious currents, and the contact angle of the droplet) on the device.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// per-block partial sums: [0] mass [1] rho_max [2] rho_min [3] max |v|^2
// [4] n [5..13] sums X, Y, XX, XY, YY, X r2, Y r2, r2, (unused) [14] ss
constexpr int DIAG_W = 16;
constexpr int DIAG_BLOCKS = 608;  // 4 per SM on 152 SMs
constexpr int DIAG_THREADS = 256;

struct DiagScratch {
  double* d_part = nullptr;  // [DIAG_BLOCKS][DIAG_W]
  double* d_out = nullptr;   // [DIAG_W]
  double* h_out = nullptr;   // pinned [DIAG_W]
};

struct DiagResult {
  double mass, rho_max, rho_min, u_max, theta_deg, fit_rms, xc, yc, radius;
  int n;
};

// Block partials and their fixed-order reduction, then the 3x3 normal
// equations of the circle fit on the host, then a second pass for the rms.
// part/out: device scratch of DIAG_BLOCKS*DIAG_W and DIAG_W doubles;
// h_out: host buffer of DIAG_W doubles (pinned or pageable).
cudaError_t diagnostics_into(double* part, double* out, double* h_out, int nx, int ny,
                             const double* rho, const double* ux, const double* uy,
                             const uint16_t* flags, double level, double y_w, double x_ref,
                             double d_min, cudaStream_t s, DiagResult* r);

cudaError_t run_diagnostics(DiagScratch& sc, int nx, int ny, const double* rho, const double* ux,
                            const double* uy, const uint16_t* flags, double level, double y_w,
                            double x_ref, double d_min, cudaStream_t s, DiagResult* r);
void diag_free(DiagScratch& sc);

}  // namespace lbm
