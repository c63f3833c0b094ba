// Reverse mode of one time step (FP64), for the gradient of a contact-angle
// loss with respect to the G_w field.
//
// State: f(t), the populations after streaming and the wall rule, [9][N].
// One forward step, per fluid node x (Sec. II, III):
//   rho = sum f, psi = sqrt(a rho + b) (Eq. 15), ghost psi on solid nodes,
//   g = sum_a w_a psi(x+e_a) e_a, F = -G psi g - X A (Eqs. 7, 10, 11, 14),
//   f* = f + M^-1 dm(m, F, |F_m|^2/psi^2 = G^2 |g|^2) (Eqs. 2-4, 9),
//   f'(x + e_a) = f*_a(x) (Eq. 5), then the wall rule / bounce-back gives
//   f(t+1).
// Given lam(t+1) = dL/df(t+1), one reverse step gives lam(t) = dL/df(t) and
// adds dL/dG_w(z) for every solid node z, in three passes over the forward
// state f(t) and its rho and psi on fluid nodes, which the recomputation of
// the forward steps stores beside f(t):
//   k_adj_walls   ghost psi of the solid nodes; adjoint of the wall rule at
//                 NEQ wall nodes: lam' and the
//                 adjoint of the node's force that the rule used
//   k_adj_node    per fluid node: adjoint of streaming (gather of lam'),
//                 of the collision and of the local parts of the force
//   k_adj_gather  per node: transposed psi stencil, ghost sources, d psi /
//                 d rho (from rho and psi), lam(t); on solid nodes the G_w
//                 gradient through A.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.cuh"

namespace lbm {

__constant__ int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

namespace {

__device__ __forceinline__ int wrapn(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ double wgt(int a) { return a == 0 ? 0.0 : (a <= 4 ? 1.0 / 3.0 : 1.0 / 12.0); }

struct Node {
  int x, y;
  long long i;
};

__device__ __forceinline__ bool node_of(const InstDesc& I, Node& n) {
  const long long N = I.plane;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return false;
  n.i = i;
  n.x = (int)(i % I.nx);
  n.y = (int)(i / I.nx);
  return true;
}

__device__ __forceinline__ long long nb(const InstDesc& I, const Node& n, int dx, int dy) {
  return (long long)wrapn(n.y + dy, I.ny) * I.nx + wrapn(n.x + dx, I.nx);
}

// psi^2 = a rho + b (Eq. 15); returns a for d(psi^2)/d(rho)
__device__ __forceinline__ double psi2_and_slope(const InstDesc& I, double rho, double& a) {
  double b;
  if (rho <= I.ph.rho1) {
    a = I.ph.aV;
    b = 0.0;
  } else if (rho <= I.ph.rho2) {
    a = I.ph.aM;
    b = I.ph.bM;
  } else {
    a = I.ph.aL;
    b = I.ph.bL;
  }
  return a * rho + b;
}

}  // namespace

__device__ __forceinline__ int ghost_offset(const InstDesc& I, uint16_t fl) {
  if (I.ph.ghost != LBM_GHOST_COPY && I.ph.ghost != LBM_GHOST_MIRROR) return 0;
  const int d = I.ph.ghost == LBM_GHOST_COPY ? 1 : 2;
  if (fl & NF_GHOST_UP) return d;
  if (fl & NF_GHOST_DOWN) return -d;
  return 0;
}

// adjoint of the NEQ wall rule (Sec. III.A) at wall nodes; elsewhere lam' = lam
// (and the ghost psi of solid nodes from the fluid psi of the forward state)
__global__ void k_adj_walls(const InstDesc* __restrict__ insts, const double* __restrict__ lam,
                            double* lamp, double2* lamF_bc, double* psi) {
  const InstDesc& I = insts[0];
  Node n;
  if (!node_of(I, n)) return;
  const long long N = I.plane;
  {
    const uint16_t fs = I.flags[n.i];
    if (fs & NF_SELF_SOLID) {
      const int d = ghost_offset(I, fs);
      psi[n.i] = d ? psi[nb(I, n, 0, d)] : 0.0;
    }
  }
  double l[Q];
  for (int a = 0; a < Q; ++a) l[a] = lam[a * N + n.i];
  const uint16_t fl = I.flags[n.i];
  double Fx = 0.0, Fy = 0.0;
  if (I.ph.wall == LBM_WALL_NEQ_ONNODE && (fl & NF_NEQ_BOTTOM)) {
    // f2 = f4', f5 = f7' - (f1' - f3')/2 - (Fx + Fy)/4, f6 = f8' + (f1' - f3')/2 + (Fx - Fy)/4
    const double l2 = l[2], l5 = l[5], l6 = l[6];
    l[1] += -0.5 * l5 + 0.5 * l6;
    l[3] += 0.5 * l5 - 0.5 * l6;
    l[4] += l2;
    l[7] += l5;
    l[8] += l6;
    Fx = -0.25 * l5 + 0.25 * l6;
    Fy = -0.25 * l5 - 0.25 * l6;
    l[2] = l[5] = l[6] = 0.0;
  } else if (I.ph.wall == LBM_WALL_NEQ_ONNODE && (fl & NF_NEQ_TOP)) {
    // f4 = f2', f8 = f6' - (f1' - f3')/2 - (Fx - Fy)/4, f7 = f5' + (f1' - f3')/2 + (Fx + Fy)/4
    const double l4 = l[4], l8 = l[8], l7 = l[7];
    l[1] += -0.5 * l8 + 0.5 * l7;
    l[3] += 0.5 * l8 - 0.5 * l7;
    l[2] += l4;
    l[6] += l8;
    l[5] += l7;
    Fx = -0.25 * l8 + 0.25 * l7;
    Fy = 0.25 * l8 + 0.25 * l7;
    l[4] = l[7] = l[8] = 0.0;
  }
  for (int a = 0; a < Q; ++a) lamp[a * N + n.i] = l[a];
  lamF_bc[n.i] = make_double2(Fx, Fy);
}

// per fluid node: adjoint of streaming, collision and the local force terms
__global__ void k_adj_node(const InstDesc* __restrict__ insts, const double* __restrict__ f,
                           const double* __restrict__ rho, const double* __restrict__ psi,
                           const double* __restrict__ lam, const double* __restrict__ lamp,
                           const double2* __restrict__ lamF_bc, double* lam_dir,
                           double2* lam_g, double* lam_psi_loc, double* lam_rho_loc,
                           double2* lam_A) {
  const InstDesc& I = insts[0];
  Node n;
  if (!node_of(I, n)) return;
  const long long N = I.plane;
  const uint16_t fl = I.flags[n.i];
  if (fl & NF_SELF_SOLID) return;
  const Consts<double>& K = I.ph.cd;
  // forward quantities at x
  double fx[Q];
  for (int a = 0; a < Q; ++a) fx[a] = f[a * N + n.i];
  const double r = rho[n.i], p = psi[n.i];
  double gx = 0.0, gy = 0.0;
  for (int a = 1; a < Q; ++a) {
    const double pn = psi[nb(I, n, EX[a], EY[a])];
    gx += wgt(a) * pn * EX[a];
    gy += wgt(a) * pn * EY[a];
  }
  const bool skip = I.ph.ghost == LBM_GHOST_SKIP && (fl & NF_SRC_SOLID);
  const double G = K.G;
  double Fx = skip ? 0.0 : -G * p * gx, Fy = skip ? 0.0 : -G * p * gy;
  const double2 A = I.A[n.i];
  const double X = I.fsi == LBM_FSI_DENSITY ? r : (I.fsi == LBM_FSI_PSI ? p : p * p);
  Fx -= X * A.x;
  Fy -= X * A.y;
  // streaming adjoint: lam*_a(x) = lam'_a(x + e_a) from fluid destinations;
  // bounce-back returns f*_a(x) as f_abar(x, t+1)
  double ls[Q];
  for (int a = 0; a < Q; ++a) {
    const long long j = nb(I, n, EX[a], EY[a]);
    if (!(I.flags[j] & NF_SELF_SOLID)) ls[a] = lamp[a * N + j];
    else ls[a] = I.ph.wall == LBM_WALL_HALFWAY_BB ? lam[OPP[a] * N + n.i] : 0.0;
  }
  // moment-space adjoint: lam_dm = D^-1 M lam*
  const double a13 = ls[1] + ls[3], a24 = ls[2] + ls[4], a57 = ls[5] + ls[7], a68 = ls[6] + ls[8];
  const double d13 = ls[1] - ls[3], d24 = ls[2] - ls[4], d57 = ls[5] - ls[7], d68 = ls[6] - ls[8];
  const double s14 = a13 + a24, s58 = a57 + a68;
  // the diagonal of M^-1 as products (a division by 36, 6 or 12 costs an
  // FP64 division sequence; the gradient is checked to 1e-5, not bitwise)
  constexpr double i36 = 1.0 / 36.0, i6 = 1.0 / 6.0, i12 = 1.0 / 12.0;
  const double ae = (-4.0 * ls[0] - s14 + 2.0 * s58) * i36;
  const double az = (4.0 * ls[0] - 2.0 * s14 + s58) * i36;
  const double ajx = (d13 + d57 - d68) * i6;
  const double aqx = (-2.0 * d13 + d57 - d68) * i12;
  const double ajy = (d24 + d57 + d68) * i6;
  const double aqy = (-2.0 * d24 + d57 + d68) * i12;
  const double axx = (a13 - a24) * 0.25;
  const double axy = (a57 - a68) * 0.25;
  // forward moments and velocity
  const double jx = fx[1] - fx[3] + fx[5] - fx[6] - fx[7] + fx[8];
  const double jy = fx[2] - fx[4] + fx[5] + fx[6] - fx[7] - fx[8];
  const double mx = jx + 0.5 * Fx, my = jy + 0.5 * Fy;
  const double ir = 1.0 / r;
  const double vx = mx * ir, vy = my * ir;
  const double s_nu = K.s_nu, h_nu = K.h_nu;
  // reverse of dm (see the forward collision)
  double l_rho = -2.0 * K.s_e * ae + K.s_z * az;
  const double l_e = -K.s_e * ae, l_z = -K.s_z * az;
  const double l_qx = -K.s_q * aqx, l_qy = -K.s_q * aqy;
  const double l_pxx = -s_nu * axx, l_pxy = -s_nu * axy;
  const double l_vF = 6.0 * K.h_e * ae - 6.0 * K.h_z * az;
  const double l_g2 = K.c_e * ae - K.c_z * az;
  const double l_rv2 = 3.0 * K.s_e * ae - 3.0 * K.s_z * az;
  double l_mx = -K.s_q * aqx, l_my = -K.s_q * aqy;
  double l_Fx = ajx - K.h_q * aqx, l_Fy = ajy - K.h_q * aqy;
  double l_vx = 0.0, l_vy = 0.0;
  // dxx = 2 h_nu (vx Fx - vy Fy) - s_nu (pxx - (mx vx - my vy))
  l_vx += 2.0 * h_nu * axx * Fx;
  l_Fx += 2.0 * h_nu * axx * vx;
  l_vy -= 2.0 * h_nu * axx * Fy;
  l_Fy -= 2.0 * h_nu * axx * vy;
  l_mx += s_nu * axx * vx;
  l_vx += s_nu * axx * mx;
  l_my -= s_nu * axx * vy;
  l_vy -= s_nu * axx * my;
  // dxy = h_nu (vx Fy + vy Fx) - s_nu (pxy - mx vy)
  l_vx += h_nu * axy * Fy;
  l_Fy += h_nu * axy * vx;
  l_vy += h_nu * axy * Fx;
  l_Fx += h_nu * axy * vy;
  l_mx += s_nu * axy * vy;
  l_vy += s_nu * axy * mx;
  // vF = vx Fx + vy Fy; rv2 = mx vx + my vy
  l_vx += l_vF * Fx;
  l_vy += l_vF * Fy;
  l_Fx += l_vF * vx;
  l_Fy += l_vF * vy;
  l_mx += l_rv2 * vx;
  l_vx += l_rv2 * mx;
  l_my += l_rv2 * vy;
  l_vy += l_rv2 * my;
  // v = m / rho
  l_mx += l_vx * ir;
  l_my += l_vy * ir;
  l_rho += -(l_vx * mx + l_vy * my) * ir * ir;
  // m = j + F/2
  const double l_jx = l_mx, l_jy = l_my;
  l_Fx += 0.5 * l_mx;
  l_Fy += 0.5 * l_my;
  // the wall rule of the next state used this node's force
  const double2 Fb = lamF_bc[n.i];
  l_Fx += Fb.x;
  l_Fy += Fb.y;
  // lam(f) = lam* (increment form) + M^T lam_m
  const double lm[Q] = {l_rho, l_e, l_z, l_jx, l_qx, l_jy, l_qy, l_pxx, l_pxy};
  for (int a = 0; a < Q; ++a) {
    const double e2 = (double)(EX[a] * EX[a] + EY[a] * EY[a]);
    const double row[Q] = {1.0,
                           -4.0 + 3.0 * e2,
                           4.0 - 10.5 * e2 + 4.5 * e2 * e2,
                           (double)EX[a],
                           (3.0 * e2 - 5.0) * EX[a],
                           (double)EY[a],
                           (3.0 * e2 - 5.0) * EY[a],
                           (double)(EX[a] * EX[a] - EY[a] * EY[a]),
                           (double)(EX[a] * EY[a])};
    double v = ls[a];
    for (int k = 0; k < Q; ++k) v += row[k] * lm[k];
    lam_dir[a * N + n.i] = v;
  }
  // force adjoint, local parts: F = -G psi g - X A, g2 = G^2 |g|^2
  double lgx = 0.0, lgy = 0.0, lpsi = 0.0, lrho = 0.0;
  if (!skip) {
    lgx = -G * p * l_Fx + 2.0 * G * G * gx * l_g2;
    lgy = -G * p * l_Fy + 2.0 * G * G * gy * l_g2;
    lpsi = -G * (gx * l_Fx + gy * l_Fy);
  }
  const double lX = -(A.x * l_Fx + A.y * l_Fy);
  if (I.fsi == LBM_FSI_DENSITY) lrho += lX;
  else if (I.fsi == LBM_FSI_PSI) lpsi += lX;
  else lpsi += 2.0 * p * lX;
  lam_g[n.i] = make_double2(lgx, lgy);
  lam_psi_loc[n.i] = lpsi;
  lam_rho_loc[n.i] = lrho;
  lam_A[n.i] = make_double2(-X * l_Fx, -X * l_Fy);
}

// lam_psi(z) collected from the stencils that read psi(z)
__device__ __forceinline__ double stencil_adjoint(const InstDesc& I, const Node& n,
                                                  const double2* __restrict__ lam_g) {
  double s = 0.0;
  for (int a = 1; a < Q; ++a) {
    // node x = z - e_a read psi(x + e_a) = psi(z) with weight w_a e_a
    const long long j = nb(I, n, -EX[a], -EY[a]);
    if (I.flags[j] & NF_SELF_SOLID) continue;
    const double2 lg = lam_g[j];
    s += wgt(a) * (EX[a] * lg.x + EY[a] * lg.y);
  }
  return s;
}

__global__ void k_adj_gather(const InstDesc* __restrict__ insts, const double* __restrict__ rho,
                             const double* __restrict__ psi,
                             const double* __restrict__ lam_dir, const double2* __restrict__ lam_g,
                             const double* __restrict__ lam_psi_loc,
                             const double* __restrict__ lam_rho_loc,
                             const double2* __restrict__ lam_A, double* lam_out, double* grad) {
  const InstDesc& I = insts[0];
  Node n;
  if (!node_of(I, n)) return;
  const long long N = I.plane;
  const uint16_t fl = I.flags[n.i];
  if (fl & NF_SELF_SOLID) {
    for (int a = 0; a < Q; ++a) lam_out[a * N + n.i] = 0.0;
    // dL/dG_w(z): A(x) = sum_a omega_a G_w(x + e_a) s(x + e_a) e_a
    const double scale = I.ph.omega_cs2w ? 1.0 / 3.0 : 1.0;
    double g = 0.0;
    for (int a = 1; a < Q; ++a) {
      const long long j = nb(I, n, -EX[a], -EY[a]);
      if (I.flags[j] & NF_SELF_SOLID) continue;
      const double2 la = lam_A[j];
      g += scale * wgt(a) * (EX[a] * la.x + EY[a] * la.y);
    }
    grad[n.i] += g;
    return;
  }
  double lpsi = lam_psi_loc[n.i] + stencil_adjoint(I, n, lam_g);
  // this node may be the ghost source of a solid node s (psi(s) = psi(z))
  if (I.ph.ghost == LBM_GHOST_COPY || I.ph.ghost == LBM_GHOST_MIRROR) {
    const int d = I.ph.ghost == LBM_GHOST_COPY ? 1 : 2;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      Node s;
      s.x = n.x;
      s.y = wrapn(n.y + sgn * d, I.ny);
      s.i = (long long)s.y * I.nx + s.x;
      const uint16_t sf = I.flags[s.i];
      if ((sf & NF_SELF_SOLID) && ghost_offset(I, sf) == -sgn * d)
        lpsi += stencil_adjoint(I, s, lam_g);
    }
  }
  // d psi / d rho = (d psi^2 / d rho) / (2 psi) on the branch of Eq. (15)
  double slope;
  psi2_and_slope(I, rho[n.i], slope);
  const double lrho = lam_rho_loc[n.i] + lpsi * slope / (2.0 * psi[n.i]);
  for (int a = 0; a < Q; ++a) lam_out[a * N + n.i] = lam_dir[a * N + n.i] + lrho;
}

cudaError_t launch_adjoint_step(const InstDesc& h, const InstDesc* d_inst, const double* f,
                                const double* rho, double* psi, const double* lam_next,
                                double* lam_out, double* grad, AdjScratch& s, cudaStream_t st) {
  const long long N = h.plane;
  // 64-thread blocks: a 256 x 128 lattice gives 512 blocks, enough for
  // every SM (256-thread blocks left 24 of 152 SMs idle and the rest with
  // one block each, latency bound on the FP64 pipe)
  const int tb = 64;
  const unsigned grid = (unsigned)((N + tb - 1) / tb);
  k_adj_walls<<<grid, tb, 0, st>>>(d_inst, lam_next, s.lamp, s.lamF_bc, psi);
  k_adj_node<<<grid, tb, 0, st>>>(d_inst, f, rho, psi, lam_next, s.lamp, s.lamF_bc, s.lam_dir,
                                  s.lam_g, s.lam_psi_loc, s.lam_rho_loc, s.lam_A);
  k_adj_gather<<<grid, tb, 0, st>>>(d_inst, rho, psi, s.lam_dir, s.lam_g, s.lam_psi_loc,
                                    s.lam_rho_loc, s.lam_A, lam_out, grad);
  return cudaGetLastError();
}

}  // namespace lbm
