// Fused per-sample solver for small grids (sm_103a).
//
// When a sample's whole multigrid hierarchy fits in one CTA's shared memory
// (fine grid of at most CTA_MAX_CELLS cells: MLMC level 0, 32 x 16), one CTA
// runs the complete scenario - every implicit-Euler step, Newton iteration,
// BiCGStab iteration and V-cycle - in a single launch.  The Jacobian
// hierarchy, the Newton iterate, the restricted states, and the Krylov and
// multigrid vectors live in shared memory; only the old state (read by the
// assembly, written once per step) and the QoIs touch global memory.  The
// per-cell arithmetic is the same device code as the multi-kernel path
// (assemble_cell, sweep_cell, restrict_cell, spmv_cell), and the steps follow
// the same order, so both paths compute the same iterates up to the
// summation order of the dot products.
#pragma once
#include "henry_kernels.cuh"

namespace hk {

constexpr int CTA_MAX_CELLS = 512;
constexpr int CTA_THREADS = 256;
constexpr int CTA_MAX_LEVELS = 8;

// Shared-memory layout of the fused solver (bytes, 32-byte aligned offsets).
struct CtaLayout {
  int K;                       // index of the coarsest level (2 x 1 cells)
  int nx[CTA_MAX_LEVELS], ny[CTA_MAX_LEVELS];
  int J[CTA_MAX_LEVELS];       // 6 planes of B4 per level
  int X[CTA_MAX_LEVELS];       // double2 state per level (fine: Newton iterate; coarse: restricted)
  int XO[CTA_MAX_LEVELS];      // double2 restricted old state (coarse levels only; fine old state is global)
  int MX[CTA_MAX_LEVELS], MB[CTA_MAX_LEVELS];  // multigrid vectors (coarse levels)
  int r, rh, p, v, t, ph, dx;  // fine Krylov vectors (s shares r, s_hat shares p_hat)
  int ainv, red;
  int bytes;
};

__host__ __device__ inline int cta_align(int o) { return (o + 31) & ~31; }

// Returns false if the grid is not eligible (too many cells, too many levels).
__host__ __device__ inline bool cta_layout(int nx0, int ny0, int tsize, CtaLayout* L) {
  if (nx0 * ny0 > CTA_MAX_CELLS) return false;
  const int b4 = 4 * tsize, v2 = 2 * tsize;
  int o = 0, k = 0, nx = nx0, ny = ny0;
  for (;;) {
    if (k >= CTA_MAX_LEVELS) return false;
    const int N = nx * ny;
    L->nx[k] = nx;
    L->ny[k] = ny;
    L->J[k] = o; o = cta_align(o + 6 * b4 * N);
    L->X[k] = o; o = cta_align(o + 16 * N);
    if (k > 0) {
      L->XO[k] = o; o = cta_align(o + 16 * N);
      L->MX[k] = o; o = cta_align(o + v2 * N);
      L->MB[k] = o; o = cta_align(o + v2 * N);
    } else {
      L->XO[k] = L->MX[k] = L->MB[k] = -1;
    }
    if (nx <= 2 || ny <= 1) break;
    nx >>= 1;
    ny >>= 1;
    ++k;
  }
  L->K = k;
  const int N0 = nx0 * ny0;
  L->r = o; o = cta_align(o + v2 * N0);
  L->rh = o; o = cta_align(o + v2 * N0);
  L->p = o; o = cta_align(o + v2 * N0);
  L->v = o; o = cta_align(o + v2 * N0);
  L->t = o; o = cta_align(o + v2 * N0);
  L->ph = o; o = cta_align(o + v2 * N0);
  L->dx = o; o = cta_align(o + v2 * N0);
  L->ainv = o; o = cta_align(o + 16 * tsize);
  L->red = o; o = cta_align(o + 40 * 8);
  L->bytes = o + 32;  // slack for aligning the base
  return true;
}

struct CtaParams {
  Phys ph;
  int nx0, ny0, steps, nu1, nu2, newton_maxit, lin_maxit;
  double h0, tau, inv_s, inv_pref, atol, dxtol, rtol2, predictor, dc_limit;
  int predictor_order;  // 1: linear, 2: quadratic from step 2 on (xoo_g holds x^{n-2})
  double rho0g, Ly;
};

// Global-memory operands of the tail, by tail level: the level's block planes
// (6 planes of plane[k] blocks, a sample's N_k blocks at offset s N_k), the
// right-hand side b and result x of the first level ([B][N_0] vectors), and
// the coarsest inverses ([B][16]).
struct TailArgs {
  const void* J[CTA_MAX_LEVELS];
  int64_t plane[CTA_MAX_LEVELS];
  const void* b;
  void* x;
  const void* ainv;
};

// A CTA's view of its shared memory.  J(k) is level k's 6 block planes with
// plane stride plane(k): in shared memory (stride N_k), or, for a tail level
// whose layout has no room for them (L->J[k] < 0), the sample's blocks in
// global memory (stride A->plane[k]), read through L2 at every use.
template <typename T>
struct CtaSmem {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  unsigned char* base;
  const CtaLayout* L;
  const TailArgs* A = nullptr;  // the tail's global operands (streamed levels only)
  int s = 0;                    // the CTA's sample
  __device__ B4* J(int k) const {
    if (L->J[k] >= 0) return reinterpret_cast<B4*>(base + L->J[k]);
    return const_cast<B4*>(reinterpret_cast<const B4*>(A->J[k])) + (int64_t)s * (L->nx[k] * L->ny[k]);
  }
  __device__ int64_t plane(int k) const { return L->J[k] >= 0 ? (int64_t)L->nx[k] * L->ny[k] : A->plane[k]; }
  __device__ double2* X(int k) const { return reinterpret_cast<double2*>(base + L->X[k]); }
  __device__ double2* XO(int k) const { return reinterpret_cast<double2*>(base + L->XO[k]); }
  __device__ V2* MX(int k) const { return reinterpret_cast<V2*>(base + L->MX[k]); }
  __device__ V2* MB(int k) const { return reinterpret_cast<V2*>(base + L->MB[k]); }
  __device__ V2* vec(int off) const { return reinterpret_cast<V2*>(base + off); }
  __device__ T* ainv() const { return reinterpret_cast<T*>(base + L->ainv); }
  __device__ double* red() const { return reinterpret_cast<double*>(base + L->red); }
};

// CTA-wide sum of a per-thread partial (deterministic order).
__device__ __forceinline__ double cta_sum(double v, double* sh) { return block_reduce<false>(v, sh); }
__device__ __forceinline__ double cta_max(double v, double* sh) { return block_reduce<true>(v, sh); }

// One half-sweep over colour col of level k, then a barrier.
template <typename T, int MODE>
__device__ __forceinline__ void cta_sweep(const CtaSmem<T>& S, int k, int col, const typename VT<T>::v2* b,
                                          typename VT<T>::v2* x, const typename VT<T>::v2* xc) {
  const int nx = S.L->nx[k], ny = S.L->ny[k], N = nx * ny, half = nx >> 1;
  const typename VT<T>::b4* J = S.J(k);
  const int64_t ps = S.plane(k);
  for (int u = threadIdx.x; u < (N >> 1); u += blockDim.x) {
    const int iy = u / half, j = u - iy * half;
    const int ix = 2 * j + ((col ^ iy) & 1);
    const int i = iy * nx + col * half + j;
    x[i] = sweep_cell<T, MODE>(nx, ny, ix, iy, i, J, ps, b, x, xc);
  }
  __syncthreads();
}

// One V(nu1, nu2) cycle in shared memory: x = M^{-1} b on level 0.
template <typename T>
__device__ void cta_vcycle(const CtaSmem<T>& S, int nu1, int nu2, const typename VT<T>::v2* b0,
                           typename VT<T>::v2* x0) {
  typedef typename VT<T>::v2 V2;
  const int K = S.L->K;
  for (int k = 0; k < K; ++k) {
    const V2* b = k == 0 ? b0 : S.MB(k);
    V2* x = k == 0 ? x0 : S.MX(k);
    const int nx = S.L->nx[k], N = nx * S.L->ny[k];
    const int ncx = S.L->nx[k + 1], ncy = S.L->ny[k + 1];
    V2* bc = S.MB(k + 1);
    if (nu1 > 0) {
      cta_sweep<T, 0>(S, k, 0, b, x, nullptr);
      cta_sweep<T, 1>(S, k, 1, b, x, nullptr);
      for (int i = 1; i < nu1; ++i) {
        cta_sweep<T, 1>(S, k, 0, b, x, nullptr);
        cta_sweep<T, 1>(S, k, 1, b, x, nullptr);
      }
      for (int c = threadIdx.x; c < ncx * ncy; c += blockDim.x) {
        int IX, IY;
        xy_of(c, ncx, IX, IY);
        bc[c] = restrict_cell<T, 0>(ncx, ncy, IX, IY, S.J(k), S.plane(k), b, x);
      }
    } else {
      for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = mk2<V2>((T)0, (T)0);
      for (int c = threadIdx.x; c < ncx * ncy; c += blockDim.x) {
        int IX, IY;
        xy_of(c, ncx, IX, IY);
        bc[c] = restrict_cell<T, 1>(ncx, ncy, IX, IY, S.J(k), S.plane(k), b, x);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // coarsest 2 x 1 grid: explicit 4 x 4 inverse
    const V2 b0c = S.MB(K)[0], b1c = S.MB(K)[1];
    const T v[4] = {b0c.x, b0c.y, b1c.x, b1c.y};
    const T* M = S.ainv();
    T o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = M[4 * i] * v[0] + M[4 * i + 1] * v[1] + M[4 * i + 2] * v[2] + M[4 * i + 3] * v[3];
    S.MX(K)[0] = mk2<V2>(o[0], o[1]);
    S.MX(K)[1] = mk2<V2>(o[2], o[3]);
  }
  __syncthreads();
  for (int k = K - 1; k >= 0; --k) {
    const V2* b = k == 0 ? b0 : S.MB(k);
    V2* x = k == 0 ? x0 : S.MX(k);
    if (nu2 > 0) {
      cta_sweep<T, 2>(S, k, 0, b, x, S.MX(k + 1));
      cta_sweep<T, 1>(S, k, 1, b, x, nullptr);
      for (int i = 1; i < nu2; ++i) {
        cta_sweep<T, 1>(S, k, 0, b, x, nullptr);
        cta_sweep<T, 1>(S, k, 1, b, x, nullptr);
      }
    } else {
      const int nx = S.L->nx[k], N = nx * S.L->ny[k];
      const V2* xc = S.MX(k + 1);
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int ix, iy;
        xy_of(i, nx, ix, iy);
        const V2 c = xc[st_of(ix >> 1, iy >> 1, nx >> 1)];
        V2 vv = x[i];
        vv.x += c.x;
        vv.y += c.y;
        x[i] = vv;
      }
      __syncthreads();
    }
  }
}

// Coarsest 4 x 4 inverse (thread 0), FP64 Gauss-Jordan with partial pivoting.
template <typename T>
__device__ void cta_coarse_inverse(const CtaSmem<T>& S) {
  if (threadIdx.x != 0) return;
  const int K = S.L->K;
  const typename VT<T>::b4* J = S.J(K);
  const int ps = 2;
  const auto Ca = J[0], Ea = J[2 * ps + 0], Wb = J[ps + 1], Cb = J[1];
  double M[4][8];
  const double blk[4][4] = {{Ca.a00, Ca.a01, Ea.a00, Ea.a01},
                            {Ca.a10, Ca.a11, Ea.a10, Ea.a11},
                            {Wb.a00, Wb.a01, Cb.a00, Cb.a01},
                            {Wb.a10, Wb.a11, Cb.a10, Cb.a11}};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      M[i][j] = blk[i][j];
      M[i][4 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (piv != col)
      for (int j = 0; j < 8; ++j) {
        const double tt = M[col][j];
        M[col][j] = M[piv][j];
        M[piv][j] = tt;
      }
    const double inv = 1.0 / M[col][col];
    for (int j = 0; j < 8; ++j) M[col][j] *= inv;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      for (int j = 0; j < 8; ++j) M[r][j] -= f * M[col][j];
    }
  }
  T* A = S.ainv();
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i * 4 + j] = (T)M[i][4 + j];
}

// The fused scenario solve: one CTA per sample.  xo_g: the sample's old state
// in global memory ([B][N0] double2, storage layout), xoo_g the state before
// it (quadratic predictor; may be NULL with predictor_order 1); qoi[B][2]; status[B]
// (0 on entry for samples to solve).  totals[0] += Newton iterations,
// totals[1] += BiCGStab iterations.
template <typename T>
__global__ void __launch_bounds__(CTA_THREADS) k_cta_solve(const __grid_constant__ CtaParams P,
                                                           const __grid_constant__ CtaLayout L, int B,
                                                           const Coef* __restrict__ coef,
                                                           double2* __restrict__ xo_g, double2* __restrict__ xoo_g,
                                                           double* __restrict__ qoi,
                                                           int* __restrict__ status,
                                                           unsigned long long* __restrict__ totals) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  typedef typename std::conditional<std::is_same<T, float>::value, float, double>::type SC;  // coarse flux type
  extern __shared__ unsigned char smem_raw[];
  const int s = blockIdx.x;
  if (s >= B) return;
  if (status[s] != 0) {
    if (threadIdx.x == 0) {
      qoi[2 * (int64_t)s] = NAN;
      qoi[2 * (int64_t)s + 1] = NAN;
    }
    return;
  }
  CtaSmem<T> S;
  S.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 31) & ~uintptr_t(31));
  S.L = &L;
  double* sh = S.red();
  const int nx0 = P.nx0, ny0 = P.ny0, N0 = nx0 * ny0, K = L.K;
  const Coef cf = coef[s];
  double2* xo = xo_g + (int64_t)s * N0;
  const bool quad = P.predictor_order == 2 && xoo_g;
  double2* xoo = quad ? xoo_g + (int64_t)s * N0 : nullptr;
  double2* x = S.X(0);
  V2 *r = S.vec(L.r), *rh = S.vec(L.rh), *p = S.vec(L.p), *v = S.vec(L.v), *t = S.vec(L.t);
  V2 *ph = S.vec(L.ph), *dx = S.vec(L.dx);
  const double inv_tau = 1.0 / P.tau;
  unsigned long long newton_total = 0, lin_total = 0;
  int fail = 0;

  // a3: initial state, fresh-water hydrostatic pressure, c = 0
  for (int i = threadIdx.x; i < N0; i += blockDim.x) {
    const int iy = i / nx0;
    const double2 v0 = make_double2(P.rho0g * (P.Ly - (iy + 0.5) * P.h0), 0.0);
    x[i] = v0;
    xo[i] = v0;
    if (quad) xoo[i] = v0;
  }
  __syncthreads();

  for (int step = 0; step < P.steps && !fail; ++step) {
    // a10: x_old <- x (and Newton's first iterate by the predictor)
    for (int i = threadIdx.x; i < N0; i += blockDim.x) {
      const double2 a = x[i], b = xo[i];
      double2 c = b;
      if (quad) {
        c = xoo[i];
        xoo[i] = b;
      }
      xo[i] = a;
      if (quad && step > 1 && P.predictor > 0.0) {  // as k_step_begin_predict2
        const double dx = 2.0 * (a.x - b.x) - (b.x - c.x), dy = 2.0 * (a.y - b.y) - (b.y - c.y);
        x[i] = make_double2(fma(P.predictor, dx, a.x), fma(P.predictor, dy, a.y));
      } else if (step > 0 && P.predictor > 0.0) {
        x[i] = make_double2(fma(P.predictor, a.x - b.x, a.x), fma(P.predictor, a.y - b.y, a.y));
      }
    }
    __syncthreads();
    // restricted old states of the coarse levels
    for (int k = 1; k <= K; ++k) {
      const int ncx = L.nx[k], Nc = ncx * L.ny[k], nxf = 2 * ncx;
      const double2* xf = k == 1 ? xo : S.XO(k - 1);
      double2* xc = S.XO(k);
      for (int c = threadIdx.x; c < Nc; c += blockDim.x) {
        int IX, IY;
        xy_of(c, ncx, IX, IY);
        const double2 a = xf[st_of(2 * IX, 2 * IY, nxf)], b = xf[st_of(2 * IX + 1, 2 * IY, nxf)];
        const double2 cc = xf[st_of(2 * IX, 2 * IY + 1, nxf)], d = xf[st_of(2 * IX + 1, 2 * IY + 1, nxf)];
        xc[c] = make_double2(0.25 * (((a.x + b.x) + cc.x) + d.x), 0.25 * (((a.y + b.y) + cc.y) + d.y));
      }
      __syncthreads();
    }

    for (int it = 0;; ++it) {
      // a4: fine residual and Jacobian; r = r_hat = -F
      double rloc = 0.0;
      T rrT = (T)0;
      for (int i = threadIdx.x; i < N0; i += blockDim.x) {
        int ix, iy;
        xy_of(i, nx0, ix, iy);
        CellSys<T, double> o;
        assemble_cell<T, double>(P.ph, cf, nx0, ny0, P.h0, 1.0 / P.h0, P.h0 * P.h0 * inv_tau * P.inv_s, P.inv_s, x,
                                 xo, i, ix, iy, o);
        store_blocks<T>(S.J(0), N0, i, o.C, o.Nb);
        const V2 ri = mk2<V2>((T)(-o.fm), (T)(-o.fs));
        r[i] = ri;
        rh[i] = ri;
        double l = fmax(fabs(o.fm), fabs(o.fs));
        if (!(l <= 1.0e300)) l = INFINITY;
        rloc = fmax(rloc, l);
        rrT = fma_(ri.x, ri.x, fma_(ri.y, ri.y, rrT));
      }
      const double rmax = cta_max(rloc, sh);
      if (!(rmax <= 1.0e300)) {
        fail = 3;
        break;
      }
      if (rmax <= P.atol) break;
      if (it >= P.newton_maxit) {
        fail = 1;
        break;
      }
      ++newton_total;
      // a5: restricted states and rediscretised coarse operators
      for (int k = 1; k <= K; ++k) {
        const int ncx = L.nx[k], ncy = L.ny[k], Nc = ncx * ncy, nxf = 2 * ncx;
        const double2* xf = S.X(k - 1);
        double2* xc = S.X(k);
        for (int c = threadIdx.x; c < Nc; c += blockDim.x) {
          int IX, IY;
          xy_of(c, ncx, IX, IY);
          const double2 a = xf[st_of(2 * IX, 2 * IY, nxf)], b = xf[st_of(2 * IX + 1, 2 * IY, nxf)];
          const double2 cc = xf[st_of(2 * IX, 2 * IY + 1, nxf)], d = xf[st_of(2 * IX + 1, 2 * IY + 1, nxf)];
          xc[c] = make_double2(0.25 * (((a.x + b.x) + cc.x) + d.x), 0.25 * (((a.y + b.y) + cc.y) + d.y));
        }
        __syncthreads();
        const double hk = P.h0 * (double)(1 << k);
        for (int c = threadIdx.x; c < Nc; c += blockDim.x) {
          int IX, IY;
          xy_of(c, ncx, IX, IY);
          CellSys<T, SC> o;
          assemble_cell<T, SC>(P.ph, cf, ncx, ncy, hk, 1.0 / hk, hk * hk * inv_tau * P.inv_s, P.inv_s, xc,
                               S.XO(k), c, IX, IY, o);
          store_blocks<T>(S.J(k), Nc, c, o.C, o.Nb);
        }
      }
      __syncthreads();
      cta_coarse_inverse<T>(S);
      // a6: BiCGStab, right-preconditioned by the V-cycle (a7), SpMV (a8)
      const double bn2 = cta_sum((double)rrT, sh);
      double rho = bn2, rho_prev = 1.0, alpha = 1.0, omega = 1.0, rn2 = bn2;
      for (int i = threadIdx.x; i < N0; i += blockDim.x) {
        p[i] = mk2<V2>((T)0, (T)0);
        v[i] = mk2<V2>((T)0, (T)0);
        dx[i] = mk2<V2>((T)0, (T)0);
      }
      __syncthreads();
      int lit = 0;
      for (; lit < P.lin_maxit; ++lit) {
        if (!(rn2 <= 1.0e300) || !(rho == rho)) {
          fail = 3;
          break;
        }
        if (rn2 <= P.rtol2 * bn2) break;
        const double beta = (lit == 0) ? 0.0 : (rho / rho_prev) * (alpha / omega);
        const T bt = (T)beta, om = (T)omega;
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
          const V2 rr_ = r[i], pp = p[i], vv = v[i];
          p[i] = lit == 0 ? rr_ : mk2<V2>(rr_.x + bt * (pp.x - om * vv.x), rr_.y + bt * (pp.y - om * vv.y));
        }
        __syncthreads();
        cta_vcycle<T>(S, P.nu1, P.nu2, p, ph);
        // per-thread partial sums in T, widened once for the CTA reduction
        T rvT = (T)0;
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
          int ix, iy;
          xy_of(i, nx0, ix, iy);
          const V2 yy = spmv_cell<T>(nx0, ny0, ix, iy, i, S.J(0), N0, ph);
          v[i] = yy;
          const V2 w = rh[i];
          rvT = fma_(w.x, yy.x, fma_(w.y, yy.y, rvT));
        }
        const double rv = cta_sum((double)rvT, sh);
        alpha = rho / rv;
        const T a = (T)alpha;
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
          const V2 rr_ = r[i], vv = v[i], pp = ph[i], d = dx[i];
          r[i] = mk2<V2>(rr_.x - a * vv.x, rr_.y - a * vv.y);  // s
          dx[i] = mk2<V2>(d.x + a * pp.x, d.y + a * pp.y);
        }
        __syncthreads();
        cta_vcycle<T>(S, P.nu1, P.nu2, r, ph);  // s_hat in ph
        T tsT = (T)0, ttT = (T)0;
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
          int ix, iy;
          xy_of(i, nx0, ix, iy);
          const V2 yy = spmv_cell<T>(nx0, ny0, ix, iy, i, S.J(0), N0, ph);
          t[i] = yy;
          const V2 ss = r[i];
          tsT = fma_(yy.x, ss.x, fma_(yy.y, ss.y, tsT));
          ttT = fma_(yy.x, yy.x, fma_(yy.y, yy.y, ttT));
        }
        const double ts = cta_sum((double)tsT, sh);
        const double tt = cta_sum((double)ttT, sh);
        omega = tt > 0.0 ? ts / tt : 0.0;
        const T w = (T)omega;
        T rhnT = (T)0, rnnT = (T)0;
        for (int i = threadIdx.x; i < N0; i += blockDim.x) {
          const V2 ss = r[i], tv = t[i], sv = ph[i], d = dx[i], hh = rh[i];
          dx[i] = mk2<V2>(d.x + w * sv.x, d.y + w * sv.y);
          const V2 rn = mk2<V2>(ss.x - w * tv.x, ss.y - w * tv.y);
          r[i] = rn;
          rhnT = fma_(hh.x, rn.x, fma_(hh.y, rn.y, rhnT));
          rnnT = fma_(rn.x, rn.x, fma_(rn.y, rn.y, rnnT));
        }
        rho_prev = rho;
        rho = cta_sum((double)rhnT, sh);
        rn2 = cta_sum((double)rnnT, sh);
      }
      lin_total += lit;
      if (fail) break;
      // a9: Newton update (step limited to max |dc| <= dc_limit) and the update test
      double dloc = 0.0, cloc = 0.0;
      for (int i = threadIdx.x; i < N0; i += blockDim.x) {
        const V2 d = dx[i];
        double dc = fabs((double)d.y);
        double l = fmax(fabs((double)d.x) * P.inv_pref, dc);
        if (!(l <= 1.0e300)) l = INFINITY;
        if (!(dc <= 1.0e300)) dc = INFINITY;
        dloc = fmax(dloc, l);
        cloc = fmax(cloc, dc);
      }
      const double dmax = cta_max(dloc, sh);
      const double cmax = cta_max(cloc, sh);
      const double th = (P.dc_limit > 0.0 && cmax > P.dc_limit) ? P.dc_limit / cmax : 1.0;
      for (int i = threadIdx.x; i < N0; i += blockDim.x) {
        const V2 d = dx[i];
        double2 xx = x[i];
        xx.x = fma(th, (double)d.x, xx.x);
        xx.y = fma(th, (double)d.y, xx.y);
        x[i] = xx;
      }
      __syncthreads();
      if (!(dmax <= 1.0e300)) {
        fail = 3;
        break;
      }
      if (dmax <= P.dxtol) break;
    }
  }
  // a11: QoIs
  double acc = 0.0;
  for (int i = threadIdx.x; i < N0; i += blockDim.x) {
    const double c = x[i].y;
    acc += (P.ph.rho0 + P.ph.drho * c) * c;
  }
  acc = cta_sum(acc, sh);
  if (threadIdx.x == 0) {
    const int ix0 = (3 * ny0) / 2 - 1, iy0 = ny0 / 4 - 1;
    const double c00 = x[st_of(ix0, iy0, nx0)].y, c10 = x[st_of(ix0 + 1, iy0, nx0)].y;
    const double c01 = x[st_of(ix0, iy0 + 1, nx0)].y, c11 = x[st_of(ix0 + 1, iy0 + 1, nx0)].y;
    qoi[2 * (int64_t)s] = cf.phi * acc * P.h0 * P.h0;
    qoi[2 * (int64_t)s + 1] = 0.25 * (((c00 + c10) + c01) + c11);
    if (fail) status[s] = fail;
    atomicAdd(&totals[0], newton_total);
    atomicAdd(&totals[1], lin_total);
  }
}

}  // namespace hk

namespace hk {

// ---------------------------------------------------------------------------
// a7, fused multigrid tail: the part of a V-cycle below a coarse level kt,
// i.e. the V(nu1, nu2) cycle that solves A_kt x_kt = b_kt approximately from
// x_kt = 0, run by one CTA per sample with every tail level's operator and
// vectors in shared memory.  The multi-kernel V-cycle launches ~9 kernels per
// coarse level (sweeps, residual + restriction) on grids of 128 cells per
// sample or fewer; here the sample's coarse operators are read from global
// memory once per V-cycle and every phase of those levels costs a CTA barrier
// instead of a kernel launch.  The arithmetic is cta_vcycle's, which is the
// multi-kernel cycle's per cell and in the same order (sweep_cell,
// restrict_cell, the coarsest 4 x 4 product), so the result is bit-identical
// to the multi-kernel V-cycle's.

// Shared-memory layout of a tail starting on an nx x ny grid: per level the
// 6 block planes and the multigrid vectors x, b (level 0 of the layout is the
// tail's first level kt), the coarsest inverse and a reduction buffer.  The
// first n_stream levels keep their block planes in global memory (J = -1).
__host__ __device__ inline bool tail_layout(int nx0, int ny0, int tsize, CtaLayout* L, int n_stream = 0) {
  const int b4 = 4 * tsize, v2 = 2 * tsize;
  int o = 0, k = 0, nx = nx0, ny = ny0;
  for (;;) {
    if (k >= CTA_MAX_LEVELS) return false;
    const int N = nx * ny;
    L->nx[k] = nx;
    L->ny[k] = ny;
    if (k < n_stream) {
      L->J[k] = -1;
    } else {
      L->J[k] = o; o = cta_align(o + 6 * b4 * N);
    }
    L->MX[k] = o; o = cta_align(o + v2 * N);
    L->MB[k] = o; o = cta_align(o + v2 * N);
    L->X[k] = L->XO[k] = -1;
    if (nx <= 2 || ny <= 1) break;
    nx >>= 1;
    ny >>= 1;
    ++k;
  }
  L->K = k;
  if (n_stream > k) return false;  // the coarsest level's blocks stay in shared memory
  L->r = L->rh = L->p = L->v = L->t = L->ph = L->dx = -1;
  L->ainv = o; o = cta_align(o + 16 * tsize);
  L->red = o; o = cta_align(o + 40 * 8);
  L->bytes = o + 32;
  return true;
}


// Copy n 16-byte words from global to shared memory (all threads of the CTA).
__device__ __forceinline__ void cta_copy16(void* dst, const void* src, int n) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = __ldg(s + i);
}

constexpr int TAIL_MAX_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(TAIL_MAX_THREADS) k_vcycle_tail(const __grid_constant__ CtaLayout L,
                                                                  const __grid_constant__ TailArgs A, int B, int nu1,
                                                                  int nu2, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  extern __shared__ unsigned char smem_raw[];
  const int s = blockIdx.x;
  if (s >= B || !active[s]) return;
  CtaSmem<T> S;
  S.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 31) & ~uintptr_t(31));
  S.L = &L;
  S.A = &A;
  S.s = s;
  const int K = L.K;
  // the sample's operators of every tail level held in shared memory: 6
  // contiguous runs of N_k blocks (streamed levels are read where used)
  for (int k = 0; k <= K; ++k) {
    if (L.J[k] < 0) continue;
    const int N = L.nx[k] * L.ny[k];
    const int words = N * (int)sizeof(B4) / 16;
    const B4* Jg = reinterpret_cast<const B4*>(A.J[k]) + (int64_t)s * N;
    B4* Js = S.J(k);
    for (int q = 0; q < 6; ++q) cta_copy16(Js + q * N, Jg + q * A.plane[k], words);
  }
  const int N0 = L.nx[0] * L.ny[0];
  cta_copy16(S.MB(0), reinterpret_cast<const V2*>(A.b) + (int64_t)s * N0, N0 * (int)sizeof(V2) / 16);
  {
    const T* ai = reinterpret_cast<const T*>(A.ainv) + (int64_t)s * 16;
    for (int i = threadIdx.x; i < 16; i += blockDim.x) S.ainv()[i] = ai[i];
  }
  __syncthreads();
  cta_vcycle<T>(S, nu1, nu2, S.MB(0), S.MX(0));  // ends with a barrier
  V2* xg = reinterpret_cast<V2*>(A.x) + (int64_t)s * N0;
  const V2* xs = S.MX(0);
  for (int i = threadIdx.x; i < N0; i += blockDim.x) xg[i] = xs[i];
}

}  // namespace hk
