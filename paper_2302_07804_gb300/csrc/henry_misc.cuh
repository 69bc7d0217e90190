// Sampling, coefficients, initial state, QoIs, layout conversion and the
// MLMC accumulation kernels (sm_103a).
#pragma once
#include "henry_kernels.cuh"

namespace hk {

// ---------------------------------------------------------------------------
// a1: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64-bit multiplications whose high halves are XORed with the other
// two counter words and the round key; the key advances by the Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}
// Two words -> (2u + 1 - 2^52) 2^-52 with u = (w0 << 20) | (w1 >> 12): an odd
// multiple of 2^-52 in (-1, 1), formed exactly in integers.
__device__ __forceinline__ double words_to_unit(uint32_t w0, uint32_t w1) {
  const int64_t u = ((int64_t)w0 << 20) | (int64_t)(w1 >> 12);
  const int64_t k = 2 * u + 1 - ((int64_t)1 << 52);
  return (double)k * 0x1p-52;
}
__global__ void k_sample_xi(uint64_t seed, int level, uint64_t first, int n, double* __restrict__ xi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t sidx = first + (uint64_t)i;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4((uint32_t)level, (uint32_t)sidx, (uint32_t)(sidx >> 32), 0u), key);
  const uint4 b = philox4x32_10(make_uint4((uint32_t)level, (uint32_t)sidx, (uint32_t)(sidx >> 32), 1u), key);
  xi[3 * (int64_t)i + 0] = words_to_unit(a.x, a.y);
  xi[3 * (int64_t)i + 1] = words_to_unit(a.z, a.w);
  xi[3 * (int64_t)i + 2] = words_to_unit(b.x, b.y);
}

// a2: phi = phi_mean (1 + phi_amp xi1), K = K_mean exp(logK_amp xi2),
// q_in = qin_mean (1 + qin_amp xi3); stored as (phi, K / mu, phi Dm, q_in).
struct CoefModel {
  double phi_mean, K_mean, qin_mean, phi_amp, logK_amp, qin_amp, mu, Dm;
};
__global__ void k_coefficients(CoefModel m, int n, const double* __restrict__ xi, Coef* __restrict__ coef,
                               int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x1 = xi[3 * (int64_t)i], x2 = xi[3 * (int64_t)i + 1], x3 = xi[3 * (int64_t)i + 2];
  Coef c;
  c.phi = m.phi_mean * (1.0 + m.phi_amp * x1);
  const double K = m.K_mean * exp(m.logK_amp * x2);
  c.kmu = K / m.mu;
  c.PD = c.phi * m.Dm;
  c.qin = m.qin_mean * (1.0 + m.qin_amp * x3);
  coef[i] = c;
  const bool ok = (c.phi > 0.0) && (c.phi < 1.0) && (K > 0.0) && (K <= 1.0e300) && (c.qin == c.qin) &&
                  (fabs(c.qin) <= 1.0e300);
  status[i] = ok ? 0 : 3;
}

// ---------------------------------------------------------------------------
// Random-field coefficient model (KL expansions of log K and phi, see
// henry_kl.cuh): per sample the inputs are theta_K[terms], theta_phi[terms]
// (iid N(0,1), drawn by the caller) and xi3 (uniform, for q_in).  cc[e] =
// (phi, K / mu) at the cell centre:
//   K = K_mean exp(sigma_K sum_t sqrt(lam_t) theta_K,t psi_t),
//   phi = clip(phi_mean + sigma_phi sum_t sqrt(lam_t) theta_phi,t psi_t, phi_lo, phi_hi),
// psi_t(x, y) = psi_x[ti_t](x) psi_y[tj_t](y) from the 1-D tables of this grid.
struct KLParams {
  int terms, n_in, m;
  double K_mean, sigma_logK, phi_mean, sigma_phi, phi_lo, phi_hi, mu;
};
__global__ void __launch_bounds__(TPB) k_fields_kl(KLParams P, int B, int nx, int ny, const double* __restrict__ inp,
                                                   const int* __restrict__ ti, const int* __restrict__ tj,
                                                   const double* __restrict__ sl, const double* __restrict__ psx,
                                                   const double* __restrict__ psy, double2* __restrict__ cc,
                                                   int* __restrict__ status) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  int ix, iy;
  xy_of((int)(e - (int64_t)s * N), nx, ix, iy);
  const double* in = inp + (int64_t)s * P.n_in;
  double gK = 0.0, gp = 0.0;
  for (int t = 0; t < P.terms; ++t) {
    const double mode = psy[(int64_t)tj[t] * ny + iy] * psx[(int64_t)ti[t] * nx + ix];
    gK = fma(sl[t] * in[t], mode, gK);
    gp = fma(sl[t] * in[P.terms + t], mode, gp);
  }
  const double K = P.K_mean * exp(P.sigma_logK * gK);
  const double phi = fmin(fmax(P.phi_mean + P.sigma_phi * gp, P.phi_lo), P.phi_hi);
  cc[e] = make_double2(phi, K / P.mu);
  if (!(K > 0.0 && K <= 1.0e300 && phi == phi)) atomicExch(status + s, 3);
}

// Two-layer porosity of the paper's experiments (Eq. poro_2levels) with the
// Kozeny-Carman permeability (Eq. e_perm_Kozeny_Carman) K = kappa phi^3 /
// (1 - phi^2), kappa fixed by K(E[phi]) = K_mean; the paper's y in [-1, 0]
// is y - Ly here, the layer interface at -0.75 is y = Ly - 0.75.
struct TwoLayerParams {
  int n_in;
  double phi_mean, kappa, mu, Ly, y_if;
};
__global__ void __launch_bounds__(TPB) k_fields_two_layer(TwoLayerParams P, int B, int nx, int ny, double h,
                                                          const double* __restrict__ inp, double2* __restrict__ cc,
                                                          int* __restrict__ status) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  int ix, iy;
  xy_of((int)(e - (int64_t)s * N), nx, ix, iy);
  const double* in = inp + (int64_t)s * P.n_in;
  const double xi1 = in[0], xi2 = in[1];
  const double x = (ix + 0.5) * h, yp = (iy + 0.5) * h - P.Ly;  // paper coordinates
  const double pi = 3.14159265358979323846;
  const double c0 = (yp < P.y_if) ? 1.0 + 0.2 * xi1 : 1.0 - 0.2 * xi1;
  const double phi = P.phi_mean * (1.0 + 0.15 * (xi2 * cos(pi * x / 2.0) + xi2 * sin(2.0 * pi * yp) + xi1 * cos(2.0 * pi * x))) * c0;
  const double K = P.kappa * phi * phi * phi / (1.0 - phi * phi);
  cc[e] = make_double2(phi, K / P.mu);
  if (!(phi > 0.0 && phi < 1.0 && K > 0.0 && K <= 1.0e300)) atomicExch(status + s, 3);
}

// Coarse multigrid cells: mean of the children's (phi, K / mu).
__global__ void __launch_bounds__(TPB) k_restrict_cc(int B, int ncx, int ncy, const double2* __restrict__ ccf,
                                                     double2* __restrict__ ccc) {
  const int Nc = ncx * ncy;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * Nc) return;
  const int s = (int)(e / Nc);
  int IX, IY;
  xy_of((int)(e - (int64_t)s * Nc), ncx, IX, IY);
  const int nxf = 2 * ncx;
  const int64_t bf = (int64_t)s * Nc * 4;
  const double2 a = ccf[bf + st_of(2 * IX, 2 * IY, nxf)], b = ccf[bf + st_of(2 * IX + 1, 2 * IY, nxf)];
  const double2 c = ccf[bf + st_of(2 * IX, 2 * IY + 1, nxf)], d = ccf[bf + st_of(2 * IX + 1, 2 * IY + 1, nxf)];
  ccc[e] = make_double2(0.25 * (((a.x + b.x) + c.x) + d.x), 0.25 * (((a.y + b.y) + c.y) + d.y));
}

// Face coefficients: harmonic means 2 a b / (a + b) of K / mu and of phi Dm on
// the east (.x, .y) and north (.z, .w) face of every cell, 0 on the boundary.
__global__ void __launch_bounds__(TPB) k_face_coefs(int B, int nx, int ny, double Dm, const double2* __restrict__ cc,
                                                    double4_32a* __restrict__ fc) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  const int st = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(st, nx, ix, iy);
  const double2* c = cc + (int64_t)s * N;
  const double2 P = c[st];
  double4_32a f;
  f.x = f.y = f.z = f.w = 0.0;
  auto harm = [](double a, double b) { return 2.0 * a * b / (a + b); };
  if (ix + 1 < nx) {
    const double2 E = c[st_of(ix + 1, iy, nx)];
    f.x = harm(P.y, E.y);
    f.y = harm(P.x * Dm, E.x * Dm);
  }
  if (iy + 1 < ny) {
    const double2 Nn = c[st_of(ix, iy + 1, nx)];
    f.z = harm(P.y, Nn.y);
    f.w = harm(P.x * Dm, Nn.x * Dm);
  }
  fc[e] = f;
}

// a2 for the field models: q_in from its uniform input (index iq).
__global__ void k_coefficients_qin(int n, int n_in, int iq, double qin_mean, double qin_amp,
                                   const double* __restrict__ inp, Coef* __restrict__ coef, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Coef c;
  c.phi = 0.0;
  c.kmu = 0.0;
  c.PD = 0.0;
  c.qin = qin_mean * (1.0 + qin_amp * inp[(int64_t)i * n_in + iq]);
  coef[i] = c;
  status[i] = (c.qin == c.qin && fabs(c.qin) <= 1.0e300) ? 0 : 3;
}

// a3: c = 0 and fresh-water hydrostatic pressure rho0 g (Ly - y).
__global__ void __launch_bounds__(TPB) k_init_state(int B, int nx, int ny, double h, double rho0g, double Ly,
                                                    double2* __restrict__ x) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int st = (int)(e % N);
  const int iy = st / nx;
  x[e] = make_double2(rho0g * (Ly - (iy + 0.5) * h), 0.0);
}

// a11: QoIs, one CTA per sample, qoi[s][nq]: salt mass sum phi rho c h^2 and c at
// (1.5, 0.25) = mean of the cells (ix0, iy0), (ix0+1, iy0), (ix0, iy0+1),
// (ix0+1, iy0+1) with ix0 = 1.5 / h - 1, iy0 = 0.25 / h - 1.
// With per-cell coefficients (cc != NULL) the porosity weights each cell.
// QS >= 1 (the paper's QoIs, Sec. 2.2 and 4) adds [2] the freshwater integral
// Q_FW of Eq. (integral_fw), the area of the cells with c <= 0.012178, and
// [3..14] c at the 12 points of Eq. (12points) (paper y in [-1, 0], here y +
// Ly) by bilinear interpolation of the four surrounding cell centres (the
// stencil clamped to the grid); QS = 2
// adds [15..] the c field averaged over the cells of the nx0 x ny0 level-0
// grid, row-major.
struct QoiSpec {
  int set, nq, nx0, ny0;
  double Lx, Ly;
};
__device__ __forceinline__ double cell_c(const double2* xs, int ix, int iy, int nx) { return xs[st_of(ix, iy, nx)].y; }
__global__ void __launch_bounds__(TPB) k_qoi(int B, int nx, int ny, double h, double rho0, double drho,
                                             const Coef* __restrict__ coef, const double2* __restrict__ x,
                                             double* __restrict__ qoi, const double2* __restrict__ cc = nullptr,
                                             QoiSpec Q = QoiSpec{0, 2, 0, 0, 2.0, 1.0}) {
  __shared__ double sh[40];
  const int s = blockIdx.x;
  const int N = nx * ny;
  const double2* xs = x + (int64_t)s * N;
  double* out = qoi + (int64_t)s * Q.nq;
  double acc = 0.0, fresh = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double c = xs[i].y;
    const double w = cc ? cc[(int64_t)s * N + i].x : 1.0;
    acc += w * (rho0 + drho * c) * c;
    fresh += (c <= 0.012178) ? 1.0 : 0.0;
  }
  acc = block_reduce<false>(acc, sh);
  if (Q.set >= 1) fresh = block_reduce<false>(fresh, sh);
  if (threadIdx.x == 0) {
    const int ix0 = (3 * ny) / 2 - 1, iy0 = ny / 4 - 1;
    const double c00 = xs[st_of(ix0, iy0, nx)].y, c10 = xs[st_of(ix0 + 1, iy0, nx)].y;
    const double c01 = xs[st_of(ix0, iy0 + 1, nx)].y, c11 = xs[st_of(ix0 + 1, iy0 + 1, nx)].y;
    out[0] = (cc ? 1.0 : coef[s].phi) * acc * h * h;
    out[1] = 0.25 * (((c00 + c10) + c01) + c11);
    if (Q.set >= 1) out[2] = fresh * h * h;
  }
  if (Q.set < 1) return;
  if (threadIdx.x < 12) {
    const double px = 1.10 + 0.25 * (threadIdx.x & 3);
    const int row = threadIdx.x >> 2;
    const double py = (row == 0 ? -0.95 : (row == 1 ? -0.75 : -0.50)) + Q.Ly;
    const double tx = px * nx / Q.Lx - 0.5, ty = py * ny / Q.Ly - 0.5;
    // the 2 x 2 stencil is kept on the grid (linear extrapolation for a point
    // outside the hull of the cell centres, which only coarse user grids have)
    const int ix = min(max((int)floor(tx), 0), nx - 2), iy = min(max((int)floor(ty), 0), ny - 2);
    const double fx = tx - ix, fy = ty - iy;
    out[3 + threadIdx.x] = (1 - fy) * ((1 - fx) * cell_c(xs, ix, iy, nx) + fx * cell_c(xs, ix + 1, iy, nx)) +
                           fy * ((1 - fx) * cell_c(xs, ix, iy + 1, nx) + fx * cell_c(xs, ix + 1, iy + 1, nx));
  }
  if (Q.set != 2) return;
  const int f = nx / Q.nx0;
  for (int c0 = threadIdx.x; c0 < Q.nx0 * Q.ny0; c0 += blockDim.x) {
    const int IY = c0 / Q.nx0, IX = c0 - IY * Q.nx0;
    double a = 0.0;
    for (int jy = 0; jy < f; ++jy)
      for (int jx = 0; jx < f; ++jx) a += cell_c(xs, IX * f + jx, IY * f + jy, nx);
    out[15 + c0] = a / (double)(f * f);
  }
}

// The freshwater integral of Eq. (integral_fw) of the current state, one CTA
// per sample, into out[s * stride] (the Q_FW(t) series of QoI set 3).
__global__ void __launch_bounds__(TPB) k_qfw(int B, int N, double h, const double2* __restrict__ x,
                                             double* __restrict__ out, int stride, const int* __restrict__ status) {
  __shared__ double sh[40];
  const int s = blockIdx.x;
  const double2* xs = x + (int64_t)s * N;
  double fresh = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) fresh += (xs[i].y <= 0.012178) ? 1.0 : 0.0;
  fresh = block_reduce<false>(fresh, sh);
  if (threadIdx.x == 0) out[(int64_t)s * stride] = status[s] == 0 ? fresh * h * h : 0.0;
}

// Natural layout [B][ny][nx] <-> storage layout (colour-split rows).
template <typename V2>
__global__ void __launch_bounds__(TPB) k_to_storage(int B, int nx, int ny, const double2* __restrict__ in,
                                                    V2* __restrict__ out) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int64_t s = e / N;
  const int nat = (int)(e - s * N);
  const int iy = nat / nx, ix = nat - iy * nx;
  const double2 v = in[e];
  V2 o;
  o.x = v.x;
  o.y = v.y;
  out[s * N + st_of(ix, iy, nx)] = o;
}
template <typename V2>
__global__ void __launch_bounds__(TPB) k_from_storage(int B, int nx, int ny, const V2* __restrict__ in,
                                                      double2* __restrict__ out) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int64_t s = e / N;
  const int nat = (int)(e - s * N);
  const int iy = nat / nx, ix = nat - iy * nx;
  const V2 v = in[s * N + st_of(ix, iy, nx)];
  out[e] = make_double2((double)v.x, (double)v.y);
}
// Jacobian planes -> natural [B][ny][nx][5][2][2] FP64.
template <typename B4>
__global__ void __launch_bounds__(TPB) k_blocks_out(int B, int nx, int ny, const B4* __restrict__ J, int64_t plane,
                                                    double* __restrict__ out) {
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int64_t s = e / N;
  const int nat = (int)(e - s * N);
  const int iy = nat / nx, ix = nat - iy * nx;
  const int64_t src = s * N + st_of(ix, iy, nx);
  for (int k = 0; k < 5; ++k) {
    const B4 b = J[k * plane + src];
    double* o = out + e * 20 + 4 * k;
    o[0] = (double)b.a00;
    o[1] = (double)b.a01;
    o[2] = (double)b.a10;
    o[3] = (double)b.a11;
  }
}

// Row permutation of a [n][w] array (uneven mixed-level batches): gather
// dst[i] = src[perm[i]] or scatter dst[perm[i]] = src[i].
template <typename E, bool SCATTER>
__global__ void k_permute_rows(int n, int w, const int* __restrict__ perm, const E* __restrict__ src,
                               E* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * w) return;
  const int i = (int)(t / w), k = (int)(t % w);
  const int64_t j = perm[i];
  if (SCATTER) dst[j * w + k] = src[t];
  else dst[t] = src[j * w + k];
}
// Zero the rows perm[i], i in [0, n), of a [*][w] array.
__global__ void k_zero_rows(int n, int w, const int* __restrict__ perm, double* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * w) return;
  dst[(int64_t)perm[t / w] * w + t % w] = 0.0;
}

__global__ void __launch_bounds__(TPB) k_scale_d2(int64_t n, double a, double2* __restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e < n) {
    double2 v = x[e];
    x[e] = make_double2(a * v.x, a * v.y);
  }
}

// ---------------------------------------------------------------------------
// a12: MLMC accumulation, one CTA.  For each (quantity, QoI): the batch's
// count, mean and centred sum of squares M2 (two passes over the batch), then
// Chan's pairwise merge into the running (count, mean, M2).
__global__ void __launch_bounds__(1024) k_mlmc_accumulate(int n, int n_qoi, const double* __restrict__ qf,
                                                          const double* __restrict__ qc,
                                                          const int32_t* __restrict__ status,
                                                          double* __restrict__ sums) {
  __shared__ double sh[40];
  {  // block (q, which): the moments of one QoI of Y (which = 0) or of the fine QoI (which = 1)
    const int which = blockIdx.y, q = blockIdx.x;
    {
      double cnt = 0.0, sum = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (status && status[i] != 0) continue;
        double y = qf[(int64_t)i * n_qoi + q];
        if (which == 0 && qc) y -= qc[(int64_t)i * n_qoi + q];
        cnt += 1.0;
        sum += y;
      }
      cnt = block_reduce<false>(cnt, sh);
      sum = block_reduce<false>(sum, sh);
      if (cnt == 0.0) return;  // uniform: every thread holds the reduced count
      const double mb = sum / cnt;
      double m2 = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (status && status[i] != 0) continue;
        double y = qf[(int64_t)i * n_qoi + q];
        if (which == 0 && qc) y -= qc[(int64_t)i * n_qoi + q];
        m2 += (y - mb) * (y - mb);
      }
      m2 = block_reduce<false>(m2, sh);
      if (threadIdx.x == 0) {
        double* S = sums + ((int64_t)which * n_qoi + q) * 3;
        const double na = S[0], ma = S[1], m2a = S[2];
        const double nn = na + cnt;
        const double d = mb - ma;
        S[0] = nn;
        S[1] = ma + d * (cnt / nn);
        S[2] = m2a + m2 + d * d * (na * cnt / nn);
      }
      __syncthreads();
    }
  }
}

}  // namespace hk
