// Device kernels of the batched Henry-problem solver (sm_103a).
//
// Data layout (per multigrid level k of a batch of B samples, grid nx x ny):
//  * every per-cell array is [B][N] with N = nx ny, sample-major;
//  * inside a sample, cells are stored row by row, and inside each row the
//    cells of colour 0 ((ix + iy) even) come first, then those of colour 1:
//        st(ix, iy) = iy nx + colour (nx / 2) + ix / 2.
//    A red or black Gauss-Seidel half-sweep therefore streams contiguous
//    memory, and the two colours never share a 32-byte sector.
//  * the Jacobian of a level is 6 planes of 2x2 blocks [6][B N]: centre,
//    west, east, south, north, and the inverse of the centre block (so the
//    smoother needs no division); block = {a00, a01, a10, a11}, row = equation
//    (fluid mass, salt), column = unknown (p, c).
//  * states (p, c) and residuals are FP64 double2; the Jacobian, Krylov and
//    multigrid vectors are T (double, or float in the mixed-precision mode).
//
// The discrete equations are the cell-centred finite-volume form of Eqs.
// (e_cont_eq), (e_tran_eq) with Darcy's law (e_Darcy_vel), rho(c) linear
// (e_lin_density), D = phi Dm (e_mol_diff) and the boundary conditions of
// Sec. 2.1 of arXiv 2302.07804; every flux is taken outward from the cell:
//   interior face P|Nb:  rho_f = (rho_P + rho_Nb)/2,
//       q = -(K/mu) ((p_Nb - p_P)/h + sigma rho_f g),  sigma = +1 north, -1 south, 0 east/west
//       F = rho_f q h,  G = F c_up - rho_f phi Dm (c_Nb - c_P),  c_up = c_P if F >= 0 else c_Nb
//   x = 0:  F = -rho0 q_in h,  G = F c_up(c_b = 0) + 2 rho_b phi Dm c_P,  rho_b = (rho_P + rho0)/2
//   x = Lx: q = -(K/mu)(p_b - p_P)/(h/2), p_b = rho1 g (Ly - y_P), rho_b = (rho_P + rho1)/2,
//           F = rho_b q h, c_up = c_P if F >= 0 else 1, G = F c_up - 2 rho_b phi Dm (1 - c_P)
//   R^m = phi (rho - rho_old) h^2/tau + sum F,   R^s = phi (rho c - rho_old c_old) h^2/tau + sum G
// and every residual and Jacobian entry is multiplied by inv_s = 1 / (rho0 h_fine^2 / tau).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hk {

constexpr int TPB = 256;  // threads per CTA of every cell kernel

struct __align__(32) d4_t { double a00, a01, a10, a11; };
struct __align__(16) f4_t { float a00, a01, a10, a11; };

template <typename T> struct VT;
template <> struct VT<double> { typedef double2 v2; typedef d4_t b4; };
template <> struct VT<float> { typedef float2 v2; typedef f4_t b4; };

template <typename V2, typename T>
__device__ __forceinline__ V2 mk2(T a, T b) { V2 v; v.x = a; v.y = b; return v; }

// Physics constants passed by value.
struct Phys {
  double rho0, rho1, drho, g, Ly, Dm;
};

// Per-sample coefficients: porosity, K / mu, phi * Dm, inflow velocity.
struct Coef {
  double phi, kmu, PD, qin;
};

// Per-sample scalars of BiCGStab.
struct LinScal {
  double rho, alpha, omega, bnorm2;
};

// Partial-sum slots of the fine-level reductions: [q][B][nct].
enum { P_RR = 0, P_RN = 1, P_RV = 2, P_TS = 3, P_TT = 4, P_MAX = 5, P_DC = 6, NPART = 7 };

__host__ __device__ __forceinline__ int st_of(int ix, int iy, int nx) {
  return iy * nx + (((ix + iy) & 1) ? (nx >> 1) : 0) + (ix >> 1);
}
__device__ __forceinline__ void xy_of(int st, int nx, int& ix, int& iy) {
  iy = st / nx;
  const int r = st - iy * nx, half = nx >> 1;
  const int col = r >= half ? 1 : 0;
  const int j = r - col * half;
  ix = 2 * j + ((col ^ iy) & 1);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Deterministic CTA-wide sum / max; the result is returned to every thread.
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = MAX ? warp_max(v) : warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double u = lane < nw ? sh[lane] : (MAX ? -INFINITY : 0.0);
    u = MAX ? warp_max(u) : warp_sum(u);
    if (lane == 0) sh[32] = u;
  }
  __syncthreads();
  return sh[32];
}
// The same sum with fewer FP64 instructions: a shared-memory tree (halving
// the active threads each stage) down to one warp, then shuffles.  The FP64
// pipe (2 FMA units per SM on GB300) bounds the Krylov and SpMV kernels, and
// block_reduce's shuffle stage runs its adds in every warp: 5 per warp, 45
// warp instructions per 256-thread CTA, against 12 here.  sh: blockDim.x + 1
// doubles; blockDim.x a power of two >= 64.  Deterministic order.
__device__ __forceinline__ double block_sum_tree(double v, double* sh) {
  const int t = threadIdx.x, n = blockDim.x;
  sh[t] = v;
  __syncthreads();
  for (int s = n >> 1; s >= 32; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  if (t < 32) {
    double u = warp_sum(sh[t]);
    if (t == 0) sh[n] = u;
  }
  __syncthreads();
  return sh[n];
}
// CTA-wide max of non-negative doubles without NaNs (+inf allowed) on the
// integer pipes: for such values the IEEE-754 bit patterns order like the
// values, so the max of the 64-bit patterns is the max of the values (the
// same result as block_reduce<true>, with no FP64 instruction).
__device__ __forceinline__ double block_max_nonneg(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, u, o);
    u = x > u ? x : u;
  }
  unsigned long long* su = reinterpret_cast<unsigned long long*>(sh);
  __syncthreads();
  if (lane == 0) su[w] = u;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = lane < nw ? su[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
      x = y > x ? y : x;
    }
    if (lane == 0) su[32] = x;
  }
  __syncthreads();
  return __longlong_as_double((long long)su[32]);
}
// Sum of a sample's nct partials, computed identically by every CTA of the
// sample (fixed order), returned to every thread.
__device__ __forceinline__ double sample_sum(const double* __restrict__ p, int nct, double* sh) {
  double v = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < nct; i += 32) v += p[i];
    v = warp_sum(v);
    if (threadIdx.x == 0) sh[33] = v;
  }
  __syncthreads();
  v = sh[33];
  __syncthreads();
  return v;
}
// The same sum read from the finalised per-sample values when `fin` is set
// (large grids: one warp per sample summed the partials in the same order).
__device__ __forceinline__ double sample_sum_or_fin(const double* __restrict__ part, const double* __restrict__ fin,
                                                    int slot, int64_t stride, int s, int nct, double* sh) {
  if (fin) return fin[(int64_t)s * NPART + slot];
  return sample_sum(part + slot * stride + (int64_t)s * nct, nct, sh);
}
// One warp per sample: fin[s][slot] = sum of the sample's partials of up to
// two slots (slot_b < 0: one), in the order sample_sum uses.
__global__ void k_finalize(int B, int nct, const double* __restrict__ part, int slot_a, int slot_b,
                           double* __restrict__ fin) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= B) return;
  const int64_t stride = (int64_t)B * nct;
  for (int q = 0; q < 2; ++q) {
    const int slot = q == 0 ? slot_a : slot_b;
    if (slot < 0) continue;
    const double* p = part + slot * stride + (int64_t)s * nct;
    double v = 0.0;
    for (int i = lane; i < nct; i += 32) v += p[i];
    v = warp_sum(v);
    if (lane == 0) fin[(int64_t)s * NPART + slot] = v;
  }
}
// Max of a sample's nct non-negative partial maxima, by one warp (lanes
// stride over the partials; a max does not depend on the order), returned
// to every lane.  Wide grids have thousands of partials per sample.
__device__ __forceinline__ double warp_sample_max(const double* __restrict__ p, int nct, int lane) {
  double v = 0.0;
  for (int i = lane; i < nct; i += 32) v = fmax(v, p[i]);
  return warp_max(v);
}

// 2x2 block helpers as explicit fused multiply-add chains: two FMAs per row
// (written as r - a x - b y the compiler would issue a MUL, an FMA and an
// ADD, and on GB300 the FP64 pipe is the smoother's bottleneck).
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
template <typename B4, typename T>
__device__ __forceinline__ void bmv_sub(const B4& A, T x0, T x1, T& r0, T& r1) {
  r0 = fma_(-A.a00, x0, fma_(-A.a01, x1, r0));
  r1 = fma_(-A.a10, x0, fma_(-A.a11, x1, r1));
}
template <typename B4, typename T>
__device__ __forceinline__ void bmv_add(const B4& A, T x0, T x1, T& r0, T& r1) {
  r0 = fma_(A.a00, x0, fma_(A.a01, x1, r0));
  r1 = fma_(A.a10, x0, fma_(A.a11, x1, r1));
}
template <typename B4, typename T>
__device__ __forceinline__ void bmv(const B4& A, T x0, T x1, T& y0, T& y1) {
  y0 = fma_(A.a00, x0, A.a01 * x1);
  y1 = fma_(A.a10, x0, A.a11 * x1);
}
template <typename B4>
__device__ __forceinline__ B4 mkblk(double a00, double a01, double a10, double a11) {
  B4 b;
  b.a00 = a00; b.a01 = a01; b.a10 = a10; b.a11 = a11;
  return b;
}

// Land (ix = 0) and seaside (ix = nx - 1) boundary terms of one cell, added
// to its scaled residuals and centre block (assemble_cell and the tile
// assembly share them).
template <typename T, typename S, bool DROP, bool JAC = true>
__device__ __forceinline__ void boundary_terms(const Phys& ph, double qin, double inv_s, S kmu, S PD, int nx, int ix,
                                               int iy, S hS, S ihS, S rhoP, S pP, S cP, S& Rm, S& Rs, T& C00,
                                               T& C01, T& C10, T& C11) {
  const S drho = (S)ph.drho, rho0 = (S)ph.rho0;
  const T kmuP_T = (T)kmu, PDP_T = (T)PD, hT = (T)hS, hdT = (T)(0.5 * ph.drho);
  if (ix == 0) {  // land side: prescribed inflow of fresh water, c_b = 0
    const S Fl = -rho0 * (S)(qin * inv_s) * hS;
    const S rb = (S)0.5 * (rhoP + rho0);
    const bool up = Fl >= (S)0;
    Rm += Fl;
    Rs += fma_(Fl, up ? cP : (S)0, (S)2 * rb * PD * cP);
    if constexpr (JAC) C11 += (up ? (T)Fl : (T)0) + PDP_T * (T)fma_(drho, cP, (S)2 * rb);
  }
  if (ix == nx - 1) {  // seaside: hydrostatic brine pressure, c_b = 1
    const S yP = ((S)iy + (S)0.5) * hS;
    const S pb = (S)ph.rho1 * (S)ph.g * ((S)ph.Ly - yP);
    const S rb = (S)0.5 * (rhoP + (S)ph.rho1);
    const S q = -kmu * (pb - pP) * ((S)2 * ihS);
    const S Fr = rb * q * hS;
    const bool up = Fr >= (S)0;
    const S cup = up ? cP : (S)1;
    const S dif = PD * ((S)1 - cP);
    Rm += Fr;
    Rs += fma_(Fr, cup, -(S)2 * rb * dif);
    if constexpr (JAC) {
      const T dFdp = (T)2 * (T)rb * kmuP_T;
      const T dFdc = DROP ? (T)0 : hdT * (T)q * hT;
      C00 += dFdp;
      C01 += dFdc;
      C10 = fma_(dFdp, (T)cup, C10);
      C11 += fma_(dFdc, (T)cup, (up ? (T)Fr : (T)0) - ((T)drho * (T)dif - (T)2 * (T)rb * PDP_T));
    }
  }
}

// ---------------------------------------------------------------------------
// a4 (and coarse operators by rediscretisation): residual and Jacobian of one
// cell.  `xs`, `xos` point at the cell arrays of one sample (storage layout;
// global or shared memory).  The per-sample K/mu and phi Dm and the
// accumulation factor h^2/tau arrive already multiplied by inv_s, so every
// flux and derivative comes out scaled.  Fluxes and residuals are formed in S
// (FP64 on the fine grid), derivative blocks in T; in the mixed mode
// (T = float) the coarse operators are assembled entirely in FP32 (S = T) and
// the fine Jacobian's derivative terms are formed in FP32 from FP64 fluxes.
template <typename T, typename S>
struct CellSys {
  S fm, fs;      // scaled residuals (fluid mass, salt)
  T C[4];        // centre block
  T Nb[4][4];    // W, E, S, N blocks
};

// FIELDS: per-cell coefficients instead of the sample's scalars: cc[st] =
// (phi, K/mu) of the cell and fc[st] = (K/mu, phi Dm) harmonic means on its
// east face (.x, .y) and north face (.z, .w), zero across the boundary.
// JAC = false: the residual alone (no derivative terms; the residual's
// arithmetic is the same code, so it is bit-identical to the JAC = true
// form's).
// DROP: the fallback preconditioner operator - the Jacobian without the
// derivatives of the face densities with respect to c (dF/dc = 0 in both
// rows), an operator whose diagonal blocks stay definite where density
// contrasts over heterogeneous K make point-block Gauss-Seidel diverge.
template <typename T, typename S, bool FIELDS = false, bool DROP = false, bool JAC = true>
__device__ __forceinline__ void assemble_cell(const Phys& ph, const Coef& cf, int nx, int ny, double h, double inv_h,
                                              double vt_s, double inv_s, const double2* xs, const double2* xos,
                                              int st, int ix, int iy, CellSys<T, S>& o,
                                              const double2* cc = nullptr, const double4_32a* fc = nullptr) {
  S kmu, PD, phi;
  if (FIELDS) {
    const double2 c = cc[st];
    phi = (S)c.x;
    kmu = (S)(c.y * inv_s);
    PD = (S)(c.x * ph.Dm * inv_s);
  } else {
    kmu = (S)(cf.kmu * inv_s);
    PD = (S)(cf.PD * inv_s);
    phi = (S)cf.phi;
  }
  const S hS = (S)h, ihS = (S)inv_h, drho = (S)ph.drho, rho0 = (S)ph.rho0;
  const double2 xP = xs[st], xO = xos[st];
  const S pP = (S)xP.x, cP = (S)xP.y, cO = (S)xO.y;
  const S rhoP = rho0 + drho * cP;
  const S rhoO = rho0 + drho * cO;
  const S vt = (S)vt_s;
  S Rm = phi * (rhoP - rhoO) * vt;
  S Rs = phi * (rhoP * cP - rhoO * cO) * vt;
  T C00 = (T)0, C01 = (T)(phi * drho * vt), C10 = (T)0, C11 = (T)(phi * (drho * cP + rhoP) * vt);
#pragma unroll
  for (int k = 0; k < 4; ++k) o.Nb[k][0] = o.Nb[k][1] = o.Nb[k][2] = o.Nb[k][3] = (T)0;
  const T kmuP_T = (T)kmu, PDP_T = (T)PD, hT = (T)h, hdT = (T)(0.5 * ph.drho);

  // interior faces W, E, S, N
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jx = ix + (k == 0 ? -1 : (k == 1 ? 1 : 0));
    const int jy = iy + (k == 2 ? -1 : (k == 3 ? 1 : 0));
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
    const S sg = (S)(k == 2 ? -ph.g : (k == 3 ? ph.g : 0.0));
    const int sn = st_of(jx, jy, nx);
    S kmu_f = kmu, PD_f = PD;
    if (FIELDS) {  // the face's harmonic means, stored with the cell west of / below the face
      const double4_32a f = fc[(k == 0 || k == 2) ? sn : st];
      kmu_f = (S)(((k < 2) ? f.x : f.z) * inv_s);
      PD_f = (S)(((k < 2) ? f.y : f.w) * inv_s);
    }
    const T kmuT = (T)kmu_f, PDT = (T)PD_f;
    const double2 xN = xs[sn];
    const S pN = (S)xN.x, cN = (S)xN.y;
    const S rhoN = rho0 + drho * cN;
    const S rhof = (S)0.5 * (rhoP + rhoN);
    const S q = -kmu_f * fma_((pN - pP), ihS, sg * rhof);
    const S Ff = rhof * q * hS;
    const bool up = Ff >= (S)0;
    const S cup = up ? cP : cN;
    const S dif = PD_f * (cN - cP);
    Rm += Ff;
    Rs += fma_(Ff, cup, -rhof * dif);
    if constexpr (!JAC) continue;
    // derivatives of (F, G) w.r.t. the unknowns of P and of the neighbour
    const T rhofT = (T)rhof, cupT = (T)cup, FfT = (T)Ff, difT = (T)dif;
    const T dFdp = rhofT * kmuT;
    const T dFdc = DROP ? (T)0 : hdT * hT * fma_((T)q, (T)1, -rhofT * kmuT * (T)sg);
    const T dGdifP = fma_(hdT, difT, -rhofT * PDT);
    const T dGdifN = fma_(hdT, difT, rhofT * PDT);
    C00 += dFdp;
    C01 += dFdc;
    C10 = fma_(dFdp, cupT, C10);
    C11 += fma_(dFdc, cupT, (up ? FfT : (T)0) - dGdifP);
    o.Nb[k][0] = -dFdp;
    o.Nb[k][1] = dFdc;
    o.Nb[k][2] = -dFdp * cupT;
    o.Nb[k][3] = fma_(dFdc, cupT, (up ? (T)0 : FfT) - dGdifN);
  }
  boundary_terms<T, S, DROP, JAC>(ph, cf.qin, inv_s, kmu, PD, nx, ix, iy, hS, ihS, rhoP, pP, cP, Rm, Rs, C00, C01, C10,
                             C11);
  o.fm = Rm;
  o.fs = Rs;
  o.C[0] = C00; o.C[1] = C01; o.C[2] = C10; o.C[3] = C11;
}

// Store a cell's Jacobian blocks (6 planes with stride `ps`, incl. C^-1).
template <typename T>
__device__ __forceinline__ void store_blocks(typename VT<T>::b4* J, int64_t ps, int64_t i, const T C[4],
                                             const T Nb[4][4]) {
  typedef typename VT<T>::b4 B4;
  J[i] = mkblk<B4>(C[0], C[1], C[2], C[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) J[(k + 1) * ps + i] = mkblk<B4>(Nb[k][0], Nb[k][1], Nb[k][2], Nb[k][3]);
  const T idet = (T)1 / (C[0] * C[3] - C[1] * C[2]);
  J[5 * ps + i] = mkblk<B4>(C[3] * idet, -C[1] * idet, -C[2] * idet, C[0] * idet);
}

// One thread per cell; FINE: CTAs never straddle samples (N % TPB == 0) and
// write the per-CTA max |F| (inf for non-finite) to rmax_part[s][ct].
template <typename T, bool FINE, bool FIELDS = false, bool DROP = false, bool JAC = true>
__global__ void __launch_bounds__(TPB) k_assemble(Phys ph, const Coef* __restrict__ coef, int B, int nx, int ny,
                                                  double h, double inv_h, double vt_s, double inv_s,
                                                  const double2* __restrict__ x, const double2* __restrict__ xo,
                                                  const int* __restrict__ active, double2* __restrict__ F,
                                                  typename VT<T>::b4* __restrict__ J, int64_t plane,
                                                  double* __restrict__ rmax_part, const double2* __restrict__ cc = nullptr,
                                                  const double4_32a* __restrict__ fc = nullptr) {
  typedef typename std::conditional<FINE, double, T>::type S;
  __shared__ double sh[40];
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int64_t total = (int64_t)B * N;
  const int s = (int)(e / N);
  if (FINE) {
    if (!active[s]) return;  // uniform over the CTA
  } else {
    if (e >= total || !active[s]) return;
  }
  const int st = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(st, nx, ix, iy);
  const int64_t base = e - st;
  CellSys<T, S> o;
  assemble_cell<T, S, FIELDS, DROP, JAC>(ph, coef[s], nx, ny, h, inv_h, vt_s, inv_s, x + base, xo + base, st, ix, iy, o,
                              FIELDS ? cc + base : nullptr, FIELDS ? fc + base : nullptr);
  if (FINE) {
    const double fm = (double)o.fm, fs = (double)o.fs;
    if (F) F[e] = make_double2(fm, fs);
    double loc = fmax(fabs(fm), fabs(fs));
    if (!(loc <= 1.0e300)) loc = INFINITY;  // NaN or inf
    const double bm = block_max_nonneg(loc, sh);
    if (threadIdx.x == 0) {
      const int nct = N / TPB;
      rmax_part[(int64_t)s * nct + (st / TPB)] = bm;
    }
  }
  if constexpr (JAC) {
    if (J) store_blocks<T>(J, plane, e, o.C, o.Nb);
  }
}

// ---------------------------------------------------------------------------
// a4, face-once form.  A face between a left/lower cell L and a right/upper
// cell R carries the scaled mass and salt fluxes F, G from L to R; L's
// residuals gain +F, +G and R's lose them, so R's derivative terms are the
// negated ones of L.  The tile kernel evaluates each face once (assemble_cell
// evaluates every interior face from both sides): the same arithmetic from
// L's side, upwinding included (at the tie F = 0 the upwind value is L's,
// the same tie-break as assemble_cell's from L's side).
template <typename T, typename S, bool JAC = true>
struct FaceData {
  S F, G;   // fluxes L -> R (scaled)
  T aL[4];  // d(F, G)/d(p_L, c_L): dF/dp, dF/dc, dG/dp, dG/dc
  T aR[4];  // d(F, G)/d(p_R, c_R)
};
// Residual-only evaluation (JAC = false): the fluxes alone.
template <typename T, typename S>
struct FaceData<T, S, false> {
  S F, G;
};

// JAC = false: the fluxes only, with exactly the arithmetic of the JAC =
// true form (the derivative terms come after F and G and feed nothing back),
// so both forms give bit-identical residuals.
template <typename T, typename S, bool DROP, bool JAC = true>
__device__ __forceinline__ void face_eval(const Phys& ph, S kmu_f, S PD_f, S sg, S hS, S ihS, double2 xL, double2 xR,
                                          FaceData<T, S, JAC>& f) {
  const S drho = (S)ph.drho, rho0 = (S)ph.rho0;
  const S pL = (S)xL.x, cL = (S)xL.y, pR = (S)xR.x, cR = (S)xR.y;
  const S rhoL = rho0 + drho * cL, rhoR = rho0 + drho * cR;
  const S rhof = (S)0.5 * (rhoL + rhoR);
  const S q = -kmu_f * fma_((pR - pL), ihS, sg * rhof);
  const S Ff = rhof * q * hS;
  const bool up = Ff >= (S)0;
  const S cup = up ? cL : cR;
  const S dif = PD_f * (cR - cL);
  f.F = Ff;
  f.G = fma_(Ff, cup, -rhof * dif);
  if constexpr (!JAC) return;
  else {
  const T kmuT = (T)kmu_f, PDT = (T)PD_f, hT = (T)hS, hdT = (T)(0.5 * ph.drho);
  const T rhofT = (T)rhof, cupT = (T)cup, FfT = (T)Ff, difT = (T)dif;
  const T dFdp = rhofT * kmuT;
  const T dFdc = DROP ? (T)0 : hdT * hT * fma_((T)q, (T)1, -rhofT * kmuT * (T)sg);
  const T dGdifL = fma_(hdT, difT, -rhofT * PDT);
  const T dGdifR = fma_(hdT, difT, rhofT * PDT);
  f.aL[0] = dFdp;
  f.aL[1] = dFdc;
  f.aL[2] = dFdp * cupT;
  f.aL[3] = fma_(dFdc, cupT, (up ? FfT : (T)0) - dGdifL);
  f.aR[0] = -dFdp;
  f.aR[1] = dFdc;
  f.aR[2] = -dFdp * cupT;
  f.aR[3] = fma_(dFdc, cupT, (up ? (T)0 : FfT) - dGdifR);
  }
}

// The residual and Jacobian of one cell from its faces' data (sgn = +1: the
// cell is the face's L, -1: its R; k = 0 W, 1 E, 2 S, 3 N).
template <typename T, typename S, bool JAC = true>
__device__ __forceinline__ void add_face(const FaceData<T, S, JAC>& f, bool cell_is_L, int k, S& Rm, S& Rs, T C[4],
                                         T Nb[4][4]) {
  if (cell_is_L) {
    Rm += f.F;
    Rs += f.G;
    if constexpr (JAC) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        C[j] += f.aL[j];
        Nb[k][j] = f.aR[j];
      }
    }
  } else {
    Rm -= f.F;
    Rs -= f.G;
    if constexpr (JAC) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        C[j] -= f.aR[j];
        Nb[k][j] = -f.aL[j];
      }
    }
  }
}

// Tile assembly: a CTA holds TPB consecutive cells in storage order, i.e.
// TPB / nx whole rows (nx <= TPB), possibly of several samples.  Phase 1:
// every cell evaluates its east and north faces into shared memory.  Phase
// 2: every cell sums its four faces (a cell of the tile's first row
// evaluates the face below it itself: its other cell lies in another tile),
// its accumulation and boundary terms, and stores F, the blocks and C^-1
// like k_assemble (same arguments; FINE: N % TPB == 0, one sample per CTA).
// Shared memory: 2 x TPB faces (40 KB in FP64).
template <typename T, bool FINE, bool FIELDS = false, bool DROP = false, bool JAC = true>
__global__ void __launch_bounds__(TPB) k_assemble_tile(Phys ph, const Coef* __restrict__ coef, int B, int nx, int ny,
                                                       double h, double inv_h, double vt_s, double inv_s,
                                                       const double2* __restrict__ x, const double2* __restrict__ xo,
                                                       const int* __restrict__ active, double2* __restrict__ F,
                                                       typename VT<T>::b4* __restrict__ J, int64_t plane,
                                                       double* __restrict__ rmax_part,
                                                       const double2* __restrict__ cc = nullptr,
                                                       const double4_32a* __restrict__ fc = nullptr) {
  typedef typename std::conditional<FINE, double, T>::type S;
  __shared__ FaceData<T, S, JAC> fE[TPB], fN[TPB];
  __shared__ double sh[40];
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int64_t total = (int64_t)B * N;
  const int s = (int)(e / N);
  if (FINE) {
    if (!active[s]) return;  // uniform over the CTA
  }
  const bool on = e < total && active[s];
  const int st = (int)(e - (int64_t)s * N);
  int ix = 0, iy = 0;
  xy_of(st, nx, ix, iy);
  const int64_t base = e - st;
  // tile slot of the cell (ix, row r of the tile); rows hold nx consecutive storage entries
  const int r = threadIdx.x / nx;
  const int slot = r * nx + ix;
  const S hS = (S)h, ihS = (S)inv_h;
  const Coef cf = on ? coef[s] : Coef{};
  S kmu = (S)0, PD = (S)0, phi = (S)0;
  if (on) {
    if (FIELDS) {
      const double2 c = cc[base + st];
      phi = (S)c.x;
      kmu = (S)(c.y * inv_s);
      PD = (S)(c.x * ph.Dm * inv_s);
    } else {
      kmu = (S)(cf.kmu * inv_s);
      PD = (S)(cf.PD * inv_s);
      phi = (S)cf.phi;
    }
    const double2 xP = x[base + st];
    if (ix + 1 < nx) {  // east face, P = L
      S kf = kmu, pf = PD;
      if (FIELDS) {
        const double4_32a q = fc[base + st];
        kf = (S)(q.x * inv_s);
        pf = (S)(q.y * inv_s);
      }
      face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)0, hS, ihS, xP, x[base + st_of(ix + 1, iy, nx)], fE[slot]);
    }
    if (iy + 1 < ny) {  // north face, P = L
      S kf = kmu, pf = PD;
      if (FIELDS) {
        const double4_32a q = fc[base + st];
        kf = (S)(q.z * inv_s);
        pf = (S)(q.w * inv_s);
      }
      face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)ph.g, hS, ihS, xP, x[base + st_of(ix, iy + 1, nx)], fN[slot]);
    }
  }
  __syncthreads();
  if (!on) return;
  const double2 xP = x[base + st], xO = xo[base + st];
  const S drho = (S)ph.drho, rho0 = (S)ph.rho0;
  const S pP = (S)xP.x, cP = (S)xP.y, cO = (S)xO.y;
  const S rhoP = rho0 + drho * cP;
  const S rhoO = rho0 + drho * cO;
  const S vt = (S)vt_s;
  S Rm = phi * (rhoP - rhoO) * vt;
  S Rs = phi * (rhoP * cP - rhoO * cO) * vt;
  T C[4] = {(T)0, (T)(phi * drho * vt), (T)0, (T)(phi * (drho * cP + rhoP) * vt)};
  T Nb[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Nb[k][0] = Nb[k][1] = Nb[k][2] = Nb[k][3] = (T)0;
  if (ix > 0) add_face<T, S, JAC>(fE[slot - 1], false, 0, Rm, Rs, C, Nb);                     // W: P = R
  if (ix + 1 < nx) add_face<T, S, JAC>(fE[slot], true, 1, Rm, Rs, C, Nb);                     // E: P = L
  if (iy > 0) {  // S: P = R
    if (r > 0) {
      add_face<T, S, JAC>(fN[slot - nx], false, 2, Rm, Rs, C, Nb);
    } else {  // the lower cell is in another tile: evaluate the face here
      const int sb = st_of(ix, iy - 1, nx);
      S kf = kmu, pf = PD;
      if (FIELDS) {
        const double4_32a q = fc[base + sb];
        kf = (S)(q.z * inv_s);
        pf = (S)(q.w * inv_s);
      }
      FaceData<T, S, JAC> fb;
      face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)ph.g, hS, ihS, x[base + sb], xP, fb);
      add_face<T, S, JAC>(fb, false, 2, Rm, Rs, C, Nb);
    }
  }
  if (iy + 1 < ny) add_face<T, S, JAC>(fN[slot], true, 3, Rm, Rs, C, Nb);                     // N: P = L
  boundary_terms<T, S, DROP, JAC>(ph, cf.qin, inv_s, kmu, PD, nx, ix, iy, hS, ihS, rhoP, pP, cP, Rm, Rs, C[0], C[1], C[2],
                             C[3]);
  if (FINE) {
    const double fm = (double)Rm, fs = (double)Rs;
    if (F) F[e] = make_double2(fm, fs);
    double loc = fmax(fabs(fm), fabs(fs));
    if (!(loc <= 1.0e300)) loc = INFINITY;  // NaN or inf
    const double bm = block_max_nonneg(loc, sh);
    if (threadIdx.x == 0) {
      const int nct = N / TPB;
      rmax_part[(int64_t)s * nct + (st / TPB)] = bm;
    }
  }
  if constexpr (JAC) {
    if (J) store_blocks<T>(J, plane, e, C, Nb);
  }
}

// Tile assembly in 2-D tiles: a CTA covers a TILE_W x (TPB / TILE_W) block
// of cells of one sample, mapped by position, not by storage order (nx a
// multiple of TILE_W, ny of TPB / TILE_W).  Phase 1: every cell evaluates its
// east and north faces into shared memory.  Phase 2: a cell takes its west
// and south faces from the tile, or, on the tile's west or south edge,
// evaluates them itself: 2 + 1 / TH + 1 / TILE_W face evaluations per cell
// (TH = TPB / TILE_W rows; 2.5 for 128 x 2, 2.16 for 32 x 8).  The per-tile
// max |F| goes to slot (tile index) of the sample's N / TPB partials.
constexpr int TILE_W_DEFAULT = 128;  // for grids wider than TPB cells
template <typename T, bool FINE, bool FIELDS = false, bool DROP = false, bool JAC = true, int TILE_W = TILE_W_DEFAULT>
__global__ void __launch_bounds__(TPB) k_assemble_tile2d(Phys ph, const Coef* __restrict__ coef, int B, int nx,
                                                         int ny, double h, double inv_h, double vt_s, double inv_s,
                                                         const double2* __restrict__ x, const double2* __restrict__ xo,
                                                         const int* __restrict__ active, double2* __restrict__ F,
                                                         typename VT<T>::b4* __restrict__ J, int64_t plane,
                                                         double* __restrict__ rmax_part,
                                                         const double2* __restrict__ cc = nullptr,
                                                         const double4_32a* __restrict__ fc = nullptr) {
  typedef typename std::conditional<FINE, double, T>::type S;
  constexpr int TH = TPB / TILE_W;
  __shared__ FaceData<T, S, JAC> fE[TPB], fN[TPB];
  __shared__ double sh[40];
  const int N = nx * ny;
  const int tiles = N / TPB;  // per sample
  const int s = (int)(blockIdx.x / tiles);
  const int tile = (int)(blockIdx.x - (int64_t)s * tiles);
  if (s >= B || !active[s]) return;  // uniform over the CTA
  const int tx = threadIdx.x % TILE_W, ty = threadIdx.x / TILE_W;
  const int tpr = nx / TILE_W;  // tiles per row band
  const int ix = (tile % tpr) * TILE_W + tx, iy = (tile / tpr) * TH + ty;
  const int st = st_of(ix, iy, nx);
  const int64_t base = (int64_t)s * N;
  const int slot = threadIdx.x;
  const S hS = (S)h, ihS = (S)inv_h;
  const Coef cf = coef[s];
  S kmu, PD, phi;
  if (FIELDS) {
    const double2 c = cc[base + st];
    phi = (S)c.x;
    kmu = (S)(c.y * inv_s);
    PD = (S)(c.x * ph.Dm * inv_s);
  } else {
    kmu = (S)(cf.kmu * inv_s);
    PD = (S)(cf.PD * inv_s);
    phi = (S)cf.phi;
  }
  const double2 xP = x[base + st];
  auto face_coef = [&](int owner, bool north, S& kf, S& pf) {
    kf = kmu;
    pf = PD;
    if (FIELDS) {
      const double4_32a q = fc[base + owner];
      kf = (S)((north ? q.z : q.x) * inv_s);
      pf = (S)((north ? q.w : q.y) * inv_s);
    }
  };
  if (ix + 1 < nx) {  // east face, P = L
    S kf, pf;
    face_coef(st, false, kf, pf);
    face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)0, hS, ihS, xP, x[base + st_of(ix + 1, iy, nx)], fE[slot]);
  }
  if (iy + 1 < ny) {  // north face, P = L
    S kf, pf;
    face_coef(st, true, kf, pf);
    face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)ph.g, hS, ihS, xP, x[base + st_of(ix, iy + 1, nx)], fN[slot]);
  }
  __syncthreads();
  const double2 xO = xo[base + st];
  const S drho = (S)ph.drho, rho0 = (S)ph.rho0;
  const S pP = (S)xP.x, cP = (S)xP.y, cO = (S)xO.y;
  const S rhoP = rho0 + drho * cP;
  const S rhoO = rho0 + drho * cO;
  const S vt = (S)vt_s;
  S Rm = phi * (rhoP - rhoO) * vt;
  S Rs = phi * (rhoP * cP - rhoO * cO) * vt;
  T C[4] = {(T)0, (T)(phi * drho * vt), (T)0, (T)(phi * (drho * cP + rhoP) * vt)};
  T Nb[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Nb[k][0] = Nb[k][1] = Nb[k][2] = Nb[k][3] = (T)0;
  if (ix > 0) {  // W: P = R
    if (tx > 0) {
      add_face<T, S, JAC>(fE[slot - 1], false, 0, Rm, Rs, C, Nb);
    } else {
      const int sw = st_of(ix - 1, iy, nx);
      S kf, pf;
      face_coef(sw, false, kf, pf);
      FaceData<T, S, JAC> fw;
      face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)0, hS, ihS, x[base + sw], xP, fw);
      add_face<T, S, JAC>(fw, false, 0, Rm, Rs, C, Nb);
    }
  }
  if (ix + 1 < nx) add_face<T, S, JAC>(fE[slot], true, 1, Rm, Rs, C, Nb);  // E: P = L
  if (iy > 0) {  // S: P = R
    if (ty > 0) {
      add_face<T, S, JAC>(fN[slot - TILE_W], false, 2, Rm, Rs, C, Nb);
    } else {
      const int sb = st_of(ix, iy - 1, nx);
      S kf, pf;
      face_coef(sb, true, kf, pf);
      FaceData<T, S, JAC> fb;
      face_eval<T, S, DROP, JAC>(ph, kf, pf, (S)ph.g, hS, ihS, x[base + sb], xP, fb);
      add_face<T, S, JAC>(fb, false, 2, Rm, Rs, C, Nb);
    }
  }
  if (iy + 1 < ny) add_face<T, S, JAC>(fN[slot], true, 3, Rm, Rs, C, Nb);  // N: P = L
  boundary_terms<T, S, DROP, JAC>(ph, cf.qin, inv_s, kmu, PD, nx, ix, iy, hS, ihS, rhoP, pP, cP, Rm, Rs, C[0], C[1], C[2],
                             C[3]);
  const int64_t e = base + st;
  if (FINE) {
    const double fm = (double)Rm, fs = (double)Rs;
    if (F) F[e] = make_double2(fm, fs);
    double loc = fmax(fabs(fm), fabs(fs));
    if (!(loc <= 1.0e300)) loc = INFINITY;  // NaN or inf
    const double bm = block_max_nonneg(loc, sh);
    if (threadIdx.x == 0) rmax_part[(int64_t)s * tiles + tile] = bm;
  }
  if constexpr (JAC) {
    if (J) store_blocks<T>(J, plane, e, C, Nb);
  }
}

// Coarse states: mean of the 2x2 children (both the iterate and the old state).
__global__ void __launch_bounds__(TPB) k_restrict_state(int B, int ncx, int ncy, const double2* __restrict__ xf,
                                                        double2* __restrict__ xc, const int* __restrict__ active) {
  const int Nc = ncx * ncy;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * Nc) return;
  const int s = (int)(e / Nc);
  if (!active[s]) return;
  const int stc = (int)(e - (int64_t)s * Nc);
  int IX, IY;
  xy_of(stc, ncx, IX, IY);
  const int nxf = 2 * ncx;
  const int64_t bf = (int64_t)s * Nc * 4;
  const double2 a = xf[bf + st_of(2 * IX, 2 * IY, nxf)];
  const double2 b = xf[bf + st_of(2 * IX + 1, 2 * IY, nxf)];
  const double2 c = xf[bf + st_of(2 * IX, 2 * IY + 1, nxf)];
  const double2 d = xf[bf + st_of(2 * IX + 1, 2 * IY + 1, nxf)];
  xc[e] = make_double2(0.25 * (((a.x + b.x) + c.x) + d.x), 0.25 * (((a.y + b.y) + c.y) + d.y));
}

// a5 (Galerkin option): A_c = R A P with piecewise-constant P, R = P^T.
template <typename T>
__global__ void __launch_bounds__(TPB) k_galerkin(int B, int ncx, int ncy, const typename VT<T>::b4* __restrict__ Jf,
                                                  int64_t plane_f, typename VT<T>::b4* __restrict__ Jc,
                                                  int64_t plane_c, const int* __restrict__ active) {
  typedef typename VT<T>::b4 B4;
  const int Nc = ncx * ncy;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * Nc) return;
  const int s = (int)(e / Nc);
  if (!active[s]) return;
  const int stc = (int)(e - (int64_t)s * Nc);
  int IX, IY;
  xy_of(stc, ncx, IX, IY);
  const int nxf = 2 * ncx;
  const int64_t bf = (int64_t)s * Nc * 4;
  const int64_t ia = bf + st_of(2 * IX, 2 * IY, nxf), ib = bf + st_of(2 * IX + 1, 2 * IY, nxf);
  const int64_t ic = bf + st_of(2 * IX, 2 * IY + 1, nxf), id = bf + st_of(2 * IX + 1, 2 * IY + 1, nxf);
  auto ld = [&](int k, int64_t i) { return Jf[k * plane_f + i]; };
  auto add = [](B4& acc, const B4& v) { acc.a00 += v.a00; acc.a01 += v.a01; acc.a10 += v.a10; acc.a11 += v.a11; };
  B4 C = ld(0, ia);
  add(C, ld(0, ib)); add(C, ld(0, ic)); add(C, ld(0, id));
  add(C, ld(2, ia)); add(C, ld(1, ib)); add(C, ld(2, ic)); add(C, ld(1, id));
  add(C, ld(4, ia)); add(C, ld(3, ic)); add(C, ld(4, ib)); add(C, ld(3, id));
  B4 W = ld(1, ia); add(W, ld(1, ic));
  B4 E = ld(2, ib); add(E, ld(2, id));
  B4 S = ld(3, ia); add(S, ld(3, ib));
  B4 Nn = ld(4, ic); add(Nn, ld(4, id));
  Jc[e] = C;
  Jc[plane_c + e] = W;
  Jc[2 * plane_c + e] = E;
  Jc[3 * plane_c + e] = S;
  Jc[4 * plane_c + e] = Nn;
  const double a = C.a00, b = C.a01, c = C.a10, d = C.a11;
  const double idet = 1.0 / (a * d - b * c);
  Jc[5 * plane_c + e] = mkblk<B4>(d * idet, -b * idet, -c * idet, a * idet);
}

// Coarsest grid (2 x 1 cells, 4 unknowns): explicit inverse per sample by
// Gauss-Jordan elimination with partial pivoting in FP64.
template <typename T>
__global__ void k_coarse_inverse(int B, const typename VT<T>::b4* __restrict__ J, int64_t plane,
                                 T* __restrict__ Ainv, const int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  // cells: st 0 = (0,0) colour 0, st 1 = (1,0) colour 1
  const int64_t a = (int64_t)s * 2, b = a + 1;
  const auto Ca = J[a], Ea = J[2 * plane + a], Wb = J[plane + b], Cb = J[b];
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
        const double t = M[col][j];
        M[col][j] = M[piv][j];
        M[piv][j] = t;
      }
    const double inv = 1.0 / M[col][col];
    for (int j = 0; j < 8; ++j) M[col][j] *= inv;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      for (int j = 0; j < 8; ++j) M[r][j] -= f * M[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ainv[(int64_t)s * 16 + i * 4 + j] = (T)M[i][4 + j];
}

template <typename T>
__global__ void k_coarse_solve(int B, const T* __restrict__ Ainv, const typename VT<T>::v2* __restrict__ b,
                               typename VT<T>::v2* __restrict__ x, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  const V2 b0 = b[2 * (int64_t)s], b1 = b[2 * (int64_t)s + 1];
  const T v[4] = {b0.x, b0.y, b1.x, b1.y};
  const T* M = Ainv + (int64_t)s * 16;
  T o[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) o[i] = M[4 * i] * v[0] + M[4 * i + 1] * v[1] + M[4 * i + 2] * v[2] + M[4 * i + 3] * v[3];
  x[2 * (int64_t)s] = mk2<V2>(o[0], o[1]);
  x[2 * (int64_t)s + 1] = mk2<V2>(o[2], o[3]);
}

// ---- smoother source begin (the measured sweep-traffic record is keyed to the hash of this region)
// a7: one half-sweep of red-black point-block Gauss-Seidel over colour `col`:
//   x_P = C_P^{-1} (b_P - sum_nb A_nb x_nb).
// MODE 0: x = 0 before the sweep (first pre-smoothing sweep: x_P = C_P^{-1} b_P).
// MODE 1: plain sweep.
// MODE 2: first post-smoothing sweep right after the coarse-grid correction:
//         the neighbours' values are read as x_nb + x_c(parent(nb)), which is
//         x += P x_c followed by the sweep (the swept cells' own old values do
//         not enter point Gauss-Seidel, and the other colour is overwritten by
//         the next half-sweep).
// Cell form: J, b, x point at one sample's arrays (plane stride ps), xc at the
// sample's coarse vector; i = storage index of the swept cell (ix, iy).
template <typename T, int MODE>
__device__ __forceinline__ typename VT<T>::v2 sweep_cell(int nx, int ny, int ix, int iy, int i,
                                                         const typename VT<T>::b4* J, int64_t ps,
                                                         const typename VT<T>::v2* b, const typename VT<T>::v2* x,
                                                         const typename VT<T>::v2* xc) {
  typedef typename VT<T>::v2 V2;
  const V2 bb = b[i];
  T r0 = bb.x, r1 = bb.y;
  if (MODE != 0) {
    const int ncx = nx >> 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int jx = ix + (k == 0 ? -1 : (k == 1 ? 1 : 0));
      const int jy = iy + (k == 2 ? -1 : (k == 3 ? 1 : 0));
      if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
      V2 xn = x[st_of(jx, jy, nx)];
      if (MODE == 2) {
        const V2 cc = xc[st_of(jx >> 1, jy >> 1, ncx)];
        xn.x += cc.x;
        xn.y += cc.y;
      }
      bmv_sub(J[(k + 1) * ps + i], xn.x, xn.y, r0, r1);
    }
  }
  T y0, y1;
  bmv(J[5 * ps + i], r0, r1, y0, y1);
  return mk2<V2>(y0, y1);
}

// NT: threads per CTA (any multiple of 32 up to 1024; every thread owns one cell).
template <typename T, int MODE, int NT = TPB>
__global__ void __launch_bounds__(NT) k_sweep(int B, int nx, int ny, int col, const typename VT<T>::b4* __restrict__ J,
                                               int64_t plane, const typename VT<T>::v2* __restrict__ b,
                                               typename VT<T>::v2* __restrict__ x,
                                               const typename VT<T>::v2* __restrict__ xc,
                                               const int* __restrict__ active) {
  const int N = nx * ny, halfN = N >> 1, half = nx >> 1;
  const int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (t >= (int64_t)B * halfN) return;
  const int s = (int)(t / halfN);
  if (!active[s]) return;
  const int u = (int)(t - (int64_t)s * halfN);
  const int iy = u / half, j = u - iy * half;
  const int ix = 2 * j + ((col ^ iy) & 1);
  const int64_t base = (int64_t)s * N;
  const int i = iy * nx + col * half + j;
  x[base + i] = sweep_cell<T, MODE>(nx, ny, ix, iy, i, J + base, plane, b + base, x + base,
                                    MODE == 2 ? xc + (int64_t)s * (N >> 2) : nullptr);
}
// ---- smoother source end

// Residual r_P = b_P - (A x)_P of one cell (sample-relative arrays).
template <typename T>
__device__ __forceinline__ void residual_cell(int nx, int ny, int ix, int iy, int i, const typename VT<T>::b4* J,
                                              int64_t ps, const typename VT<T>::v2* b,
                                              const typename VT<T>::v2* x, T& r0, T& r1) {
  typedef typename VT<T>::v2 V2;
  const V2 bb = b[i], xx = x[i];
  r0 = bb.x;
  r1 = bb.y;
  bmv_sub(J[i], xx.x, xx.y, r0, r1);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jx = ix + (k == 0 ? -1 : (k == 1 ? 1 : 0));
    const int jy = iy + (k == 2 ? -1 : (k == 3 ? 1 : 0));
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
    const V2 xn = x[st_of(jx, jy, nx)];
    bmv_sub(J[(k + 1) * ps + i], xn.x, xn.y, r0, r1);
  }
}

// Residual b - A x restricted by summation over the 2x2 children of coarse
// cell (IX, IY).  After a red-black sweep the black cells' residuals vanish
// (point Gauss-Seidel makes each swept equation hold), so MODE 0 sums the two
// colour-0 children only; MODE 1 (no pre-smoothing, x = 0) restricts b itself.
template <typename T, int MODE>
__device__ __forceinline__ typename VT<T>::v2 restrict_cell(int ncx, int ncy, int IX, int IY,
                                                            const typename VT<T>::b4* J, int64_t ps,
                                                            const typename VT<T>::v2* b,
                                                            const typename VT<T>::v2* x) {
  typedef typename VT<T>::v2 V2;
  const int nx = 2 * ncx, ny = 2 * ncy;
  T s0 = 0, s1 = 0;
  if (MODE == 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const V2 bb = b[st_of(2 * IX + (c & 1), 2 * IY + (c >> 1), nx)];
      s0 += bb.x;
      s1 += bb.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int ix = 2 * IX + c, iy = 2 * IY + c;  // (0,0) and (1,1): colour 0
      T r0, r1;
      residual_cell<T>(nx, ny, ix, iy, st_of(ix, iy, nx), J, ps, b, x, r0, r1);
      s0 += r0;
      s1 += r1;
    }
  }
  return mk2<V2>(s0, s1);
}

template <typename T, int MODE, int NT = TPB>  // MODE 0: RED_ONLY, 1: ZERO_X
__global__ void __launch_bounds__(NT) k_residual_restrict(int B, int ncx, int ncy,
                                                           const typename VT<T>::b4* __restrict__ J, int64_t plane,
                                                           const typename VT<T>::v2* __restrict__ b,
                                                           const typename VT<T>::v2* __restrict__ x,
                                                           typename VT<T>::v2* __restrict__ bc,
                                                           const int* __restrict__ active) {
  const int Nc = ncx * ncy;
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= (int64_t)B * Nc) return;
  const int s = (int)(e / Nc);
  if (!active[s]) return;
  const int stc = (int)(e - (int64_t)s * Nc);
  int IX, IY;
  xy_of(stc, ncx, IX, IY);
  const int64_t base = (int64_t)s * Nc * 4;
  bc[e] = restrict_cell<T, MODE>(ncx, ncy, IX, IY, J + base, plane, b + base, x + base);
}

// x += P x_c (used only when there is no post-smoothing to fuse it into).
template <typename T, int NT = TPB>
__global__ void __launch_bounds__(NT) k_prolong_add(int B, int nx, int ny, typename VT<T>::v2* __restrict__ x,
                                                    const typename VT<T>::v2* __restrict__ xc,
                                                    const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int N = nx * ny;
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e >= (int64_t)B * N) return;
  const int s = (int)(e / N);
  if (!active[s]) return;
  int ix, iy;
  xy_of((int)(e - (int64_t)s * N), nx, ix, iy);
  const V2 c = xc[(int64_t)s * (N >> 2) + st_of(ix >> 1, iy >> 1, nx >> 1)];
  V2 v = x[e];
  v.x += c.x;
  v.y += c.y;
  x[e] = v;
}

template <typename T, int NT = TPB>
__global__ void __launch_bounds__(NT) k_zero(int64_t n, typename VT<T>::v2* __restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (e < n) x[e] = mk2<typename VT<T>::v2>((T)0, (T)0);
}

// ---------------------------------------------------------------------------
// a8: y_P = (A x)_P of one cell (sample-relative arrays).
template <typename T>
__device__ __forceinline__ typename VT<T>::v2 spmv_cell(int nx, int ny, int ix, int iy, int i,
                                                        const typename VT<T>::b4* J, int64_t ps,
                                                        const typename VT<T>::v2* x) {
  typedef typename VT<T>::v2 V2;
  const V2 xx = x[i];
  T r0, r1;
  bmv(J[i], xx.x, xx.y, r0, r1);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jx = ix + (k == 0 ? -1 : (k == 1 ? 1 : 0));
    const int jy = iy + (k == 2 ? -1 : (k == 3 ? 1 : 0));
    if (jx < 0 || jx >= nx || jy < 0 || jy >= ny) continue;
    const V2 xn = x[st_of(jx, jy, nx)];
    bmv_add(J[(k + 1) * ps + i], xn.x, xn.y, r0, r1);
  }
  return mk2<V2>(r0, r1);
}

// y = A x (fine level, all cells) with per-CTA partial dot products:
//   NDOT 1: <w1, y>;  NDOT 2: <w1, y>, <y, y>.
template <typename T, int NDOT>
__global__ void __launch_bounds__(TPB) k_spmv(int B, int nx, int ny, const typename VT<T>::b4* __restrict__ J,
                                              int64_t plane, const typename VT<T>::v2* __restrict__ x,
                                              typename VT<T>::v2* __restrict__ y,
                                              const typename VT<T>::v2* __restrict__ w1, double* __restrict__ part,
                                              int slot1, int slot2, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[TPB + 1];
  const int N = nx * ny, nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!active[s]) return;  // uniform over the CTA
  const int st = (int)(e - (int64_t)s * N);
  int ix, iy;
  xy_of(st, nx, ix, iy);
  const int64_t base = e - st;
  const V2 yy = spmv_cell<T>(nx, ny, ix, iy, st, J + base, plane, x + base);
  y[e] = yy;
  if (NDOT >= 1 && part) {
    // per-cell products in T, widened once for the FP64 CTA reduction
    const V2 ww = w1[e];
    const double d1 = block_sum_tree((double)fma_(ww.x, yy.x, ww.y * yy.y), sh);
    double d2 = 0.0;
    if (NDOT == 2) d2 = block_sum_tree((double)fma_(yy.x, yy.x, yy.y * yy.y), sh);
    if (threadIdx.x == 0) {
      const int64_t pi = (int64_t)s * nct + st / TPB, stride = (int64_t)B * nct;
      part[slot1 * stride + pi] = d1;
      if (NDOT == 2) part[slot2 * stride + pi] = d2;
    }
  }
}

// ---------------------------------------------------------------------------
// a6: right-preconditioned BiCGStab (Templates book), per sample, on the fine
// level; per-sample scalars live in LinScal, per-CTA partial sums in part.

// r = r_hat = b (= -F), p = v = dx = 0; partials <r_hat, r>, <r, r>.
template <typename T>
__global__ void __launch_bounds__(TPB) k_bicg_init(int B, int N, const double2* __restrict__ F,
                                                   typename VT<T>::v2* __restrict__ r,
                                                   typename VT<T>::v2* __restrict__ rh,
                                                   typename VT<T>::v2* __restrict__ p, typename VT<T>::v2* __restrict__ v,
                                                   typename VT<T>::v2* __restrict__ dx, double* __restrict__ part,
                                                   const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[TPB + 1];
  const int nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!active[s]) return;
  const double2 f = F[e];
  const V2 rr = mk2<V2>((T)(-f.x), (T)(-f.y));
  const V2 z = mk2<V2>((T)0, (T)0);
  r[e] = rr;
  rh[e] = rr;
  p[e] = z;
  v[e] = z;
  dx[e] = z;
  const double bs = block_sum_tree((double)fma_(rr.x, rr.x, rr.y * rr.y), sh);
  if (threadIdx.x == 0) {
    const int64_t pi = (int64_t)s * nct + (e - (int64_t)s * N) / TPB, stride = (int64_t)B * nct;
    part[P_RR * stride + pi] = bs;
    part[P_RN * stride + pi] = bs;
  }
}

// Start of iteration `it`: rho_it = <r_hat, r>, convergence test on ||r||,
// beta = (rho_it / rho_{it-1}) (alpha / omega), p = r + beta (p - omega v).
// A converged sample's CTA 0 clears lin_active; the last iteration counts
// still-active samples in *n_active and per-sample iterations in iters.
template <typename T>
__global__ void __launch_bounds__(TPB) k_bicg_p(int B, int N, int it, int maxit, double rtol2,
                                                const typename VT<T>::v2* __restrict__ r,
                                                typename VT<T>::v2* __restrict__ p,
                                                const typename VT<T>::v2* __restrict__ v,
                                                const double* __restrict__ part, LinScal* __restrict__ sc,
                                                int* __restrict__ lin_active, int* __restrict__ iters,
                                                int* __restrict__ status, int* __restrict__ n_active,
                                                unsigned long long* __restrict__ lin_total,
                                                const double* __restrict__ fin) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[40];
  const int nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!lin_active[s]) return;
  const int ct = (int)((e - (int64_t)s * N) / TPB);
  const int64_t stride = (int64_t)B * nct;
  const double rho = sample_sum_or_fin(part, fin, P_RR, stride, s, nct, sh);
  const double rn2 = sample_sum_or_fin(part, fin, P_RN, stride, s, nct, sh);
  // The test and the Krylov scalars once per CTA, by thread 0 (an FP64
  // division is a long FP64-pipe sequence, and every thread would compute
  // the same values); bc = (stop code, beta, omega).
  __shared__ double bc[3];
  if (threadIdx.x == 0) {
    const double bn2 = (it == 0) ? rn2 : sc[s].bnorm2;
    const bool finite = (rn2 <= 1.0e300) && (rho == rho);
    const bool conv = rn2 <= rtol2 * bn2;
    bc[0] = (!finite || conv || it >= maxit) ? (!finite ? -2.0 : (conv ? (double)it : -1.0)) : -3.0;
    if (bc[0] != -3.0) {
      // A sample that reaches maxit keeps its last iterate (inexact Newton
      // step; Newton's own test decides); a non-finite one fails.
      if (ct == 0) {
        lin_active[s] = 0;
        iters[s] = (int)bc[0];
        atomicAdd(lin_total, (unsigned long long)it);
      }
    } else {
      if (ct == 0) {
        atomicAdd(n_active, 1);
        if (it == 0) sc[s].bnorm2 = bn2;
      }
      if (it > 0) {
        const LinScal q = sc[s];
        bc[1] = (rho / q.rho) * (q.alpha / q.omega);
        bc[2] = q.omega;
      }
    }
  }
  __syncthreads();
  if (bc[0] != -3.0) return;
  const V2 rr = r[e];
  if (it == 0) {
    p[e] = rr;
    return;
  }
  const double beta = bc[1], omega = bc[2];
  const V2 pp = p[e], vv = v[e];
  const T bt = (T)beta, om = (T)omega;
  p[e] = mk2<V2>(rr.x + bt * (pp.x - om * vv.x), rr.y + bt * (pp.y - om * vv.y));
}

// alpha = rho / <r_hat, v>; s = r - alpha v.  CTA 0 stores rho and alpha.
template <typename T>
__global__ void __launch_bounds__(TPB) k_bicg_s(int B, int N, const typename VT<T>::v2* __restrict__ r,
                                                const typename VT<T>::v2* __restrict__ v,
                                                typename VT<T>::v2* __restrict__ sv, const double* __restrict__ part,
                                                LinScal* __restrict__ sc, const int* __restrict__ lin_active,
                                                const double* __restrict__ fin) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[40];
  const int nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!lin_active[s]) return;
  const int ct = (int)((e - (int64_t)s * N) / TPB);
  const int64_t stride = (int64_t)B * nct;
  const double rho = sample_sum_or_fin(part, fin, P_RR, stride, s, nct, sh);
  const double rv = sample_sum_or_fin(part, fin, P_RV, stride, s, nct, sh);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = rho / rv;  // once per CTA
  __syncthreads();
  const double alpha = bc;
  if (threadIdx.x == 0 && ct == 0) {
    sc[s].rho = rho;
    sc[s].alpha = alpha;
  }
  const V2 rr = r[e], vv = v[e];
  const T a = (T)alpha;
  sv[e] = mk2<V2>(rr.x - a * vv.x, rr.y - a * vv.y);
}

// omega = <t, s> / <t, t>; dx += alpha p_hat + omega s_hat; r = s - omega t;
// partials <r_hat, r>, <r, r>.  CTA 0 stores omega.
template <typename T>
__global__ void __launch_bounds__(TPB) k_bicg_update(int B, int N, typename VT<T>::v2* __restrict__ dx,
                                                     const typename VT<T>::v2* __restrict__ ph,
                                                     const typename VT<T>::v2* __restrict__ shv,
                                                     const typename VT<T>::v2* __restrict__ sv,
                                                     const typename VT<T>::v2* __restrict__ t,
                                                     const typename VT<T>::v2* __restrict__ rh,
                                                     typename VT<T>::v2* __restrict__ r, double* __restrict__ part,
                                                     LinScal* __restrict__ sc, const int* __restrict__ lin_active,
                                                     const double* __restrict__ fin) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[TPB + 1];
  const int nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!lin_active[s]) return;
  const int ct = (int)((e - (int64_t)s * N) / TPB);
  const int64_t stride = (int64_t)B * nct;
  const double ts = sample_sum_or_fin(part, fin, P_TS, stride, s, nct, sh);
  const double tt = sample_sum_or_fin(part, fin, P_TT, stride, s, nct, sh);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = (tt > 0.0) ? ts / tt : 0.0;  // once per CTA
  __syncthreads();
  const double omega = bc;
  const double alpha = sc[s].alpha;
  if (threadIdx.x == 0 && ct == 0) sc[s].omega = omega;
  const T a = (T)alpha, w = (T)omega;
  const V2 x0 = dx[e], p0 = ph[e], s0 = shv[e], sv0 = sv[e], t0 = t[e], rh0 = rh[e];
  dx[e] = mk2<V2>(x0.x + a * p0.x + w * s0.x, x0.y + a * p0.y + w * s0.y);
  const V2 rn = mk2<V2>(sv0.x - w * t0.x, sv0.y - w * t0.y);
  r[e] = rn;
  const double d1 = block_sum_tree((double)fma_(rh0.x, rn.x, rh0.y * rn.y), sh);
  const double d2 = block_sum_tree((double)fma_(rn.x, rn.x, rn.y * rn.y), sh);
  if (threadIdx.x == 0) {
    const int64_t pi = (int64_t)s * nct + ct;
    part[P_RR * stride + pi] = d1;
    part[P_RN * stride + pi] = d2;
  }
}

// Samples whose BiCGStab did not converge (or broke down) in this Newton
// iteration get a second linear solve with the fallback preconditioner.
__global__ void k_mark_retry(int B, const int* __restrict__ newton_active, const int* __restrict__ iters,
                             int* __restrict__ lin_active, int* __restrict__ n_retry) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const int r = newton_active[s] && iters[s] < 0;
  lin_active[s] = r;
  if (r) atomicAdd(n_retry, 1);
}

// ---------------------------------------------------------------------------
// a9 / a10: Newton control.

// Per sample, after the fine assembly: converged if max |F| <= atol; a
// non-finite residual fails the sample; counts samples still iterating.
__global__ void k_newton_res_check(int B, int nct, double atol, int maxit, const double* __restrict__ rmax_part,
                                   int* __restrict__ newton_active, int* __restrict__ lin_active,
                                   int* __restrict__ newton_it, int* __restrict__ status,
                                   int* __restrict__ n_active, unsigned long long* __restrict__ it_total) {
  // one warp per sample
  const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (s >= B) return;
  int act = newton_active[s];
  const double rm = act ? warp_sample_max(rmax_part + (int64_t)s * nct, nct, lane) : 0.0;
  if (lane != 0) return;
  if (act) {
    if (!(rm <= 1.0e300)) {
      status[s] = 3;
      act = 0;
    } else if (rm <= atol) {
      act = 0;
    } else if (newton_it[s] >= maxit) {
      status[s] = status[s] ? status[s] : 1;
      act = 0;
    } else {
      newton_it[s] += 1;
      atomicAdd(n_active, 1);
      atomicAdd(it_total, 1ULL);
    }
  }
  newton_active[s] = act;
  lin_active[s] = act;
}

// Per-CTA maxima of the Newton step: max(|dp| / p_ref, |dc|) (the update
// test) and max |dc| (the step limiter).
template <typename T>
__global__ void __launch_bounds__(TPB) k_newton_step_max(int B, int N, double inv_pref,
                                                         const typename VT<T>::v2* __restrict__ dx,
                                                         double* __restrict__ dmax_part, double* __restrict__ dc_part,
                                                         const int* __restrict__ newton_active) {
  __shared__ double sh[40];
  const int nct = N / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!newton_active[s]) return;
  const auto d = dx[e];
  double dc = fabs((double)d.y);
  double loc = fmax(fabs((double)d.x) * inv_pref, dc);
  if (!(loc <= 1.0e300)) loc = INFINITY;
  if (!(dc <= 1.0e300)) dc = INFINITY;
  const double m = block_max_nonneg(loc, sh);
  const double mc = block_max_nonneg(dc, sh);
  if (threadIdx.x == 0) {
    const int64_t i = (int64_t)s * nct + (e - (int64_t)s * N) / TPB;
    dmax_part[i] = m;
    dc_part[i] = mc;
  }
}

// Per sample: theta = min(1, dc_limit / max |dc|) (a step that would change a
// mass fraction by more than dc_limit is shortened; dc_limit <= 0: theta = 1).
__global__ void k_newton_theta(int B, int nct, double dc_limit, const double* __restrict__ dc_part,
                               const int* __restrict__ newton_active, double* __restrict__ theta) {
  // one warp per sample
  const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (s >= B || !newton_active[s]) return;
  double th = 1.0;
  if (dc_limit > 0.0) {
    const double mc = warp_sample_max(dc_part + (int64_t)s * nct, nct, lane);
    if (mc > dc_limit) th = dc_limit / mc;
  }
  if (lane == 0) theta[s] = th;
}

// a9: x += theta dx.
template <typename T>
__global__ void __launch_bounds__(TPB) k_newton_update(int B, int N, double2* __restrict__ x,
                                                       const typename VT<T>::v2* __restrict__ dx,
                                                       const double* __restrict__ theta,
                                                       const int* __restrict__ newton_active) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / N);
  if (!newton_active[s]) return;
  const double th = theta[s];
  const auto d = dx[e];
  double2 xx = x[e];
  xx.x = fma(th, (double)d.x, xx.x);
  xx.y = fma(th, (double)d.y, xx.y);
  x[e] = xx;
}

__global__ void k_newton_dx_check(int B, int nct, double dxtol, const double* __restrict__ dmax_part,
                                  int* __restrict__ newton_active, int* __restrict__ status) {
  // one warp per sample
  const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (s >= B || !newton_active[s]) return;
  const double dm = warp_sample_max(dmax_part + (int64_t)s * nct, nct, lane);
  if (lane != 0) return;
  if (!(dm <= 1.0e300)) {
    status[s] = 3;
    newton_active[s] = 0;
  } else if (dm <= dxtol) {
    newton_active[s] = 0;
  }
}

// Start of a time step: old state = state; samples that have not failed iterate.
__global__ void __launch_bounds__(TPB) k_step_begin(int64_t n, const double2* __restrict__ x, double2* __restrict__ xo) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e < n) xo[e] = x[e];
}
// Start of a later time step with a linear-in-time predictor for Newton's
// first iterate: x_old <- x^n, x <- x^n + w (x^n - x^{n-1}) (x^{n-1} is the
// old state of the previous step).  Only the starting point changes; Newton
// still stops on the residual and update tests of the step.
__global__ void __launch_bounds__(TPB) k_step_begin_predict(int64_t n, double w, double2* __restrict__ x,
                                                            double2* __restrict__ xo) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= n) return;
  const double2 a = x[e], b = xo[e];
  xo[e] = a;
  x[e] = make_double2(fma(w, a.x - b.x, a.x), fma(w, a.y - b.y, a.y));
}
// The quadratic predictor: x^{n+1} ~ x^n + w (2 (x^n - x^{n-1}) - (x^{n-1} -
// x^{n-2})), i.e. 3 x^n - 3 x^{n-1} + x^{n-2} for w = 1 (extrapolation of the
// parabola through the last three states); xoo <- x^{n-1}, xo <- x^n.
__global__ void __launch_bounds__(TPB) k_step_begin_predict2(int64_t n, double w, double2* __restrict__ x,
                                                             double2* __restrict__ xo, double2* __restrict__ xoo) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= n) return;
  const double2 a = x[e], b = xo[e], c = xoo[e];
  xoo[e] = b;
  xo[e] = a;
  const double dx = 2.0 * (a.x - b.x) - (b.x - c.x), dy = 2.0 * (a.y - b.y) - (b.y - c.y);
  x[e] = make_double2(fma(w, dx, a.x), fma(w, dy, a.y));
}
// xoo <- x^{n-1} ahead of a step that still uses the linear predictor, so
// that the next step has three states.
__global__ void __launch_bounds__(TPB) k_copy_d2(int64_t n, const double2* __restrict__ src, double2* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e < n) dst[e] = src[e];
}
__global__ void k_step_flags(int B, const int* __restrict__ status, int* __restrict__ newton_active,
                             int* __restrict__ newton_it) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  newton_active[s] = status[s] == 0 ? 1 : 0;
  newton_it[s] = 0;
}

}  // namespace hk
