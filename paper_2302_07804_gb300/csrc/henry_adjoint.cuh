// Discrete adjoint of the implicit-Euler scenario solve: kernels.
//
// Q = w . qoi(x_N) depends on the random inputs theta through the states
// x_n, which satisfy F_n(x_n, x_{n-1}, theta) = 0 (the scaled residual of
// Sec. 2.3, the same one the Newton solver drives to zero).  The adjoint
// recursion, backwards over the steps,
//   J_N^T lam_N = dQ/dx_N,   J_n^T lam_n = -(dF_{n+1}/dx_n)^T lam_{n+1},
// gives dQ/dtheta = dQ/dtheta|_x - sum_n lam_n^T dF_n/dtheta.
//
// The random inputs act through per-cell coefficients only: the porosity
// phi_P, k_P = K_P / mu, d_P = phi_P Dm and the inflow q_in.  Every flux is
// linear in its face coefficient (the harmonic mean of k or of d over the
// face, or the cell's own value on the boundary), so lam^T dF/d(face
// coefficient) is the flux with unit coefficient, contracted with the
// multiplier difference across the face.  These face and cell
// sensitivities are summed over the steps (per cell, 8 planes), and only at
// the end chained through the harmonic means to the cells and through the
// coefficient model to theta.
#pragma once
#include "henry_kernels.cuh"
#include "henry_misc.cuh"

namespace hk {

// Planes of the per-cell sensitivity sums S[s][k][cell] (storage order):
enum {
  A_PHI = 0,  // accumulation terms with respect to phi_P, minus the QoI's explicit dQ/dphi_P
  A_KE = 1,   // east face, with respect to its K/mu
  A_DE = 2,   // east face, with respect to its phi Dm
  A_KN = 3,   // north face, K/mu
  A_DN = 4,   // north face, phi Dm
  A_KB = 5,   // seaside boundary face, K_P/mu
  A_DB = 6,   // land or seaside boundary face, phi_P Dm
  A_Q = 7,    // land side, q_in
  A_NPLANE = 8
};

// In-place transpose of a 5-point 2x2-block operator (planes C, W, E, S, N,
// C^-1).  In A^T the block coupling P to its west neighbour W is the
// transposed east block of W, and so on; the thread of cell P swaps the
// pair of blocks of the face to its west and of the face below it, each
// transposed, and transposes C_P and C_P^-1 in place.  Every block is
// touched by exactly one thread.
template <typename B4>
__device__ __forceinline__ B4 tr_blk(B4 b) {
  const auto t = b.a01;
  b.a01 = b.a10;
  b.a10 = t;
  return b;
}
template <typename T>
__global__ void __launch_bounds__(TPB) k_transpose_blocks(int B, int nx, int ny, typename VT<T>::b4* __restrict__ J,
                                                          int64_t plane, const int* __restrict__ active) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  if (!active[s]) return;
  const int i = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(i, nx, ix, iy);
  auto* Js = J + (int64_t)s * N;
  Js[i] = tr_blk(Js[i]);
  Js[5 * plane + i] = tr_blk(Js[5 * plane + i]);
  if (ix > 0) {
    const int w = st_of(ix - 1, iy, nx);
    const auto a = Js[plane + i], b = Js[2 * plane + w];  // W of P, E of W
    Js[plane + i] = tr_blk(b);
    Js[2 * plane + w] = tr_blk(a);
  }
  if (iy > 0) {
    const int sb = st_of(ix, iy - 1, nx);
    const auto a = Js[3 * plane + i], b = Js[4 * plane + sb];  // S of P, N of the cell below
    Js[3 * plane + i] = tr_blk(b);
    Js[4 * plane + sb] = tr_blk(a);
  }
}

// Per-cell coefficients of sample s: (phi, k = K/mu); phi Dm = phi * Dm.
__device__ __forceinline__ double2 cell_coef(const Coef* coef, const double2* cc, int s, int64_t e) {
  if (cc) return cc[e];
  const Coef c = coef[s];
  return make_double2(c.phi, c.kmu);
}

// Right-hand side of the last step: rhs = dQ/dx_N with Q = w0 mass + w1
// c_point (the QoIs of k_qoi: mass = sum phi rho(c) c h^2, c_point = mean of
// the four cells at (1.5, 0.25)); also starts the sensitivity sums, with
// S_phi = -w0 rho(c) c h^2 (the explicit dQ/dphi, entered with the sign of
// the residual terms) and every other plane 0.
__global__ void __launch_bounds__(TPB) k_adj_start(int B, int nx, int ny, double h, double rho0, double drho,
                                                   const Coef* __restrict__ coef, const double2* __restrict__ cc,
                                                   const double* __restrict__ w, const double2* __restrict__ x,
                                                   double2* __restrict__ rhs, double* __restrict__ S,
                                                   const int* __restrict__ active) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  const int i = (int)(e - (int64_t)s * N);
  double* Ss = S + (int64_t)s * A_NPLANE * N;
  for (int k = 0; k < A_NPLANE; ++k) Ss[(int64_t)k * N + i] = 0.0;
  if (!active[s]) {
    rhs[e] = make_double2(0.0, 0.0);
    return;
  }
  int ix, iy;
  xy_of(i, nx, ix, iy);
  const double phi = cell_coef(coef, cc, s, e).x;
  const double c = x[e].y;
  const double w0 = w[2 * (int64_t)s], w1 = w[2 * (int64_t)s + 1];
  const int ix0 = (3 * ny) / 2 - 1, iy0 = ny / 4 - 1;
  const bool pt = (ix == ix0 || ix == ix0 + 1) && (iy == iy0 || iy == iy0 + 1);
  rhs[e] = make_double2(0.0, w0 * phi * h * h * (rho0 + 2.0 * drho * c) + (pt ? 0.25 * w1 : 0.0));
  Ss[(int64_t)A_PHI * N + i] = -w0 * (rho0 + drho * c) * c * h * h;
}

// F <- -rhs (the Krylov solver solves J dx = -F).
__global__ void __launch_bounds__(TPB) k_adj_neg(int64_t n, const double2* __restrict__ rhs, double2* __restrict__ F) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= n) return;
  const double2 v = rhs[e];
  F[e] = make_double2(-v.x, -v.y);
}

// After an adjoint solve (which clears the samples' Krylov flags as they
// finish): a sample still in the sweep (status 0) whose solve failed
// (BiCGStab iters < 0) gets status 2 (linear solve not converged) and
// leaves; active = status == 0 for the sensitivity kernel.
__global__ void k_adj_lin_status(int B, const int* __restrict__ iters, int* __restrict__ status,
                                 int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  if (status[s] == 0 && iters[s] < 0) status[s] = 2;
  active[s] = status[s] == 0 ? 1 : 0;
}

// One step of the backward sweep, after lam = lam_m is known (x = x_m, xo =
// x_{m-1}):
//  * S += lam^T dF_m/d(coefficients) (face and cell sensitivities, unscaled
//    coefficients; F carries the factor inv_s of the residual scaling);
//  * rhs = -(dF_m/dx_{m-1})^T lam: only the accumulation terms of the cell
//    itself involve the old state, and only through its mass fraction:
//    dF^m/dc_old = -phi drho vt, dF^s/dc_old = -phi (rho0 + 2 drho c_old) vt.
// Face fluxes, densities, upwinding and boundary terms are those of the
// residual (assemble_cell).
__global__ void __launch_bounds__(TPB) k_adj_step(Phys ph, const Coef* __restrict__ coef, int B, int nx, int ny,
                                                  double h, double inv_h, double vt, double inv_s,
                                                  const double2* __restrict__ x, const double2* __restrict__ xo,
                                                  const double2* __restrict__ lam, const double2* __restrict__ cc,
                                                  double* __restrict__ S, double2* __restrict__ rhs,
                                                  const int* __restrict__ active) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  if (!active[s]) return;
  const int i = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(i, nx, ix, iy);
  const int64_t b = (int64_t)s * N;
  double* Ss = S + (int64_t)s * A_NPLANE * N;
  const double2 xP = x[e], xO = xo[e], lP = lam[e];
  const double pP = xP.x, cP = xP.y, cO = xO.y;
  const double rho0 = ph.rho0, drho = ph.drho;
  const double rhoP = rho0 + drho * cP, rhoO = rho0 + drho * cO;
  const double phi = cell_coef(coef, cc, s, e).x;
  // accumulation: F^m = phi (rhoP - rhoO) vt, F^s = phi (rhoP cP - rhoO cO) vt
  Ss[(int64_t)A_PHI * N + i] += lP.x * (rhoP - rhoO) * vt + lP.y * (rhoP * cP - rhoO * cO) * vt;
  rhs[e] = make_double2(0.0, phi * vt * (lP.x * drho + lP.y * (rho0 + 2.0 * drho * cO)));
  // interior faces east (k = 0) and north (k = 1), owned by P
  for (int k = 0; k < 2; ++k) {
    const int jx = ix + (k == 0 ? 1 : 0), jy = iy + (k == 1 ? 1 : 0);
    if (jx >= nx || jy >= ny) continue;
    const int sn = st_of(jx, jy, nx);
    const double2 xN = x[b + sn], lN = lam[b + sn];
    const double pN = xN.x, cN = xN.y;
    const double rhof = 0.5 * (rhoP + (rho0 + drho * cN));
    const double sg = k == 1 ? ph.g : 0.0;
    const double Fu = -rhof * fma((pN - pP), inv_h, sg * rhof) * h * inv_s;  // mass flux with unit K/mu
    const double cup = Fu >= 0.0 ? cP : cN;
    const double dl_m = lP.x - lN.x, dl_s = lP.y - lN.y;
    Ss[(int64_t)(k == 0 ? A_KE : A_KN) * N + i] += dl_m * Fu + dl_s * Fu * cup;
    Ss[(int64_t)(k == 0 ? A_DE : A_DN) * N + i] += dl_s * (-rhof * (cN - cP) * inv_s);
  }
  if (ix == 0) {  // land side: F = -rho0 q_in h, salt carried in only on outflow, c_b = 0
    const double qin = coef[s].qin;
    const double dFdq = -rho0 * h * inv_s;
    const bool up = dFdq * qin >= 0.0;
    const double rb = 0.5 * (rhoP + rho0);
    Ss[(int64_t)A_Q * N + i] += lP.x * dFdq + lP.y * dFdq * (up ? cP : 0.0);
    Ss[(int64_t)A_DB * N + i] += lP.y * 2.0 * rb * cP * inv_s;
  }
  if (ix == nx - 1) {  // seaside: hydrostatic brine pressure, c_b = 1
    const double yP = (iy + 0.5) * h;
    const double pb = ph.rho1 * ph.g * (ph.Ly - yP);
    const double rb = 0.5 * (rhoP + ph.rho1);
    const double Fu = -rb * (pb - pP) * (2.0 * inv_h) * h * inv_s;
    const double cup = Fu >= 0.0 ? cP : 1.0;
    Ss[(int64_t)A_KB * N + i] += lP.x * Fu + lP.y * Fu * cup;
    Ss[(int64_t)A_DB * N + i] += lP.y * (-2.0 * rb * (1.0 - cP) * inv_s);
  }
}

// d(2ab/(a+b))/da = 2 b^2 / (a+b)^2
__device__ __forceinline__ double dharm(double a, double b) {
  const double t = b / (a + b);
  return 2.0 * t * t;
}

// Per cell: dQ/dphi_P and dQ/dK_P (into g[e] = (dQ/dphi, dQ/dK)), from the
// summed sensitivities of the cell's faces chained through the harmonic
// means (a face's K/mu is 2 k_P k_Nb / (k_P + k_Nb), the boundary face uses
// k_P itself; the same for phi Dm), and the accumulation terms.  With the
// per-sample scalars of the three-parameter model the faces take the scalar
// itself; splitting its derivative 1 as 1/2 + 1/2 between the two cells of
// the face (dharm(k, k) = 1/2) gives the same sums over the cells.
__global__ void __launch_bounds__(TPB) k_adj_cell_grad(int B, int nx, int ny, double mu, double Dm,
                                                       const Coef* __restrict__ coef, const double2* __restrict__ cc,
                                                       const double* __restrict__ S, double2* __restrict__ g,
                                                       const int* __restrict__ active) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  if (!active[s]) {
    g[e] = make_double2(0.0, 0.0);
    return;
  }
  const int i = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(i, nx, ix, iy);
  const double* Ss = S + (int64_t)s * A_NPLANE * N;
  const int64_t b = (int64_t)s * N;
  const double2 cP = cell_coef(coef, cc, s, e);
  const double kP = cP.y, dP = cP.x * Dm;
  double gk = Ss[(int64_t)A_KB * N + i], gd = Ss[(int64_t)A_DB * N + i];
  for (int k = 0; k < 4; ++k) {  // E, W, N, S faces of P; the face's sums live with its west / lower cell
    const int jx = ix + (k == 0 ? 1 : (k == 1 ? -1 : 0));
    const int jy = iy + (k == 2 ? 1 : (k == 3 ? -1 : 0));
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
    const int sn = st_of(jx, jy, nx);
    const double2 cN = cell_coef(coef, cc, s, b + sn);
    const int owner = (k == 0 || k == 2) ? i : sn;
    const int pk = (k < 2) ? A_KE : A_KN, pd = (k < 2) ? A_DE : A_DN;
    gk += Ss[(int64_t)pk * N + owner] * dharm(kP, cN.y);
    gd += Ss[(int64_t)pd * N + owner] * dharm(dP, cN.x * Dm);
  }
  // dQ/dtheta = -(sum of lam^T dF/dtheta), the explicit QoI term included in A_PHI
  g[e] = make_double2(-(Ss[(int64_t)A_PHI * N + i] + Dm * gd), -gk / mu);
}

// Chain to the model's inputs, one CTA per sample: grad[s][*] from the cell
// derivatives g = (dQ/dphi, dQ/dK) and the summed q_in sensitivity.
//   MODEL 0 (three parameters): dphi/dxi1 = phi_mean phi_amp,
//     dK/dxi2 = K logK_amp, dq_in/dxi3 = qin_mean qin_amp.
//   MODEL 1 (KL): dK_P/dtheta_K,t = K_P sigma_K sqrt(lam_t) psi_t(P),
//     dphi_P/dtheta_phi,t = sigma_phi sqrt(lam_t) psi_t(P) where phi_P is
//     not clipped (0 where it is), dq_in/dxi3 as above.
//   MODEL 2 (two-layer, Eq. poro_2levels with Kozeny-Carman K): K = kappa
//     phi^3 / (1 - phi^2) gives dK/dphi = kappa phi^2 (3 - phi^2) / (1 -
//     phi^2)^2, and phi's derivatives with respect to xi1 and xi2 follow from
//     the formula of k_fields_two_layer.
struct AdjModel {
  int model, n_in, terms;
  double phi_mean, phi_amp, K_mean, logK_amp, qin_mean, qin_amp, mu;
  double sigma_logK, sigma_phi, phi_lo, phi_hi;  // KL
  double kappa, Ly, y_if, h;                     // two-layer
};
__global__ void __launch_bounds__(TPB) k_adj_project(AdjModel M, int B, int nx, int ny, const Coef* __restrict__ coef,
                                                     const double2* __restrict__ cc, const double2* __restrict__ g,
                                                     const double* __restrict__ S, const int* __restrict__ ti,
                                                     const int* __restrict__ tj, const double* __restrict__ sl,
                                                     const double* __restrict__ psx, const double* __restrict__ psy,
                                                     const double* __restrict__ inp, double* __restrict__ grad,
                                                     const int* __restrict__ active) {
  __shared__ double sh[40];
  const int s = blockIdx.x;
  const int N = nx * ny;
  double* out = grad + (int64_t)s * M.n_in;
  if (!active[s]) {
    for (int k = threadIdx.x; k < M.n_in; k += blockDim.x) out[k] = 0.0;
    return;
  }
  const int64_t b = (int64_t)s * N;
  const double* Sq = S + ((int64_t)s * A_NPLANE + A_Q) * N;
  double q = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) q += Sq[i];
  q = block_reduce<false>(q, sh);
  if (threadIdx.x == 0) out[M.n_in - 1] = -q * M.qin_mean * M.qin_amp;
  if (M.model == 0) {
    double a = 0.0, k = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double2 v = g[b + i];
      a += v.x;
      k += v.y;
    }
    a = block_reduce<false>(a, sh);
    k = block_reduce<false>(k, sh);
    if (threadIdx.x == 0) {
      out[0] = a * M.phi_mean * M.phi_amp;
      out[1] = k * coef[s].kmu * M.mu * M.logK_amp;
    }
  } else if (M.model == 1) {
    for (int t = 0; t < 2 * M.terms; ++t) {
      const int tt = t < M.terms ? t : t - M.terms;
      const double* px = psx + (int64_t)ti[tt] * nx;
      const double* py = psy + (int64_t)tj[tt] * ny;
      double a = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int ix, iy;
        xy_of(i, nx, ix, iy);
        const double2 v = g[b + i];
        const double2 c = cc[b + i];
        double d;
        if (t < M.terms) d = v.y * c.y * M.mu * M.sigma_logK;  // dQ/dK_P * K_P sigma_K
        else d = (c.x > M.phi_lo && c.x < M.phi_hi) ? v.x * M.sigma_phi : 0.0;
        a = fma(d, px[ix] * py[iy], a);
      }
      a = block_reduce<false>(a, sh);
      if (threadIdx.x == 0) out[t] = a * sl[tt];
    }
  } else {
    const double* in = inp + (int64_t)s * M.n_in;
    const double xi1 = in[0], xi2 = in[1];
    const double pi = 3.14159265358979323846;
    double a1 = 0.0, a2 = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      int ix, iy;
      xy_of(i, nx, ix, iy);
      const double x = (ix + 0.5) * M.h, yp = (iy + 0.5) * M.h - M.Ly;
      const bool lower = yp < M.y_if;
      const double c0 = lower ? 1.0 + 0.2 * xi1 : 1.0 - 0.2 * xi1;
      const double dc0 = lower ? 0.2 : -0.2;
      const double wv = 1.0 + 0.15 * (xi2 * cos(pi * x / 2.0) + xi2 * sin(2.0 * pi * yp) + xi1 * cos(2.0 * pi * x));
      const double phi = M.phi_mean * wv * c0;
      const double one = 1.0 - phi * phi;
      const double dKdphi = M.kappa * phi * phi * (3.0 - phi * phi) / (one * one);
      const double2 v = g[b + i];
      const double gp = v.x + v.y * dKdphi;
      a1 = fma(gp, M.phi_mean * (0.15 * cos(2.0 * pi * x) * c0 + wv * dc0), a1);
      a2 = fma(gp, M.phi_mean * 0.15 * (cos(pi * x / 2.0) + sin(2.0 * pi * yp)) * c0, a2);
    }
    a1 = block_reduce<false>(a1, sh);
    a2 = block_reduce<false>(a2, sh);
    if (threadIdx.x == 0) {
      out[0] = a1;
      out[1] = a2;
    }
  }
}

}  // namespace hk
