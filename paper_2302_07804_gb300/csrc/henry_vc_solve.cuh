// Batched solver kernels of the vertex-centred scheme (henry_vc.cuh): the
// paper's own discretisation (Sec. 2.3), solved like the cell-centred one -
// Newton per implicit-Euler step, BiCGStab right-preconditioned by one
// geometric-multigrid V-cycle - on the (ny + 1) x (nx + 1) vertex grid.
//
// Data layout (per multigrid level of a batch of B samples):
//  * a sample's vertices are stored row by row (j = 0 .. ny), and inside a
//    row the even-i vertices first, then the odd-i ones:
//        vst(j, i) = j (nx + 1) + (i odd ? he : 0) + i / 2,  he = (nx + 2) / 2
//    so the vertices of one of the four smoother colours (i mod 2, j mod 2)
//    form contiguous runs;
//  * per-vertex arrays are [B][stride] with stride = NV = (nx + 1)(ny + 1) on
//    the coarse levels and NV rounded up to a multiple of 256 on the fine
//    level (the Krylov and Newton kernels reduce over whole 256-entry
//    blocks of one sample; the padding entries stay zero);
//  * the Jacobian of a level is 10 planes of 2x2 blocks [10][B][stride]:
//    plane (dj + 1) 3 + (di + 1) couples vertex (j, i) to (j + dj, i + di)
//    (zero outside the grid), plane 9 is the inverse of the centre block 4.
//
// The multigrid pieces follow the vertex-nested hierarchy (coarse vertex
// (J, I) = fine vertex (2J, 2I)): coarse operators rediscretised at the
// injected states; a four-colour point-block Gauss-Seidel smoother (the
// 9-point stencil couples diagonal neighbours, so two colours would not
// decouple), colours 0..3 before and 3..0 after the coarse correction;
// restriction by full weighting (the transpose of bilinear prolongation) with
// the Dirichlet equations' entries set to zero; a dense solve on the 2 x 1
// element grid (6 vertices, 12 unknowns).
#pragma once
#include "henry_kernels.cuh"
#include "henry_vc.cuh"

namespace hk {

constexpr int VC_COARSE_N = 12;  // unknowns of the coarsest grid (3 x 2 vertices)

__host__ __device__ __forceinline__ int vc_he(int nxv) { return (nxv + 1) >> 1; }
__host__ __device__ __forceinline__ int vst(int j, int i, int nxv) {
  return j * nxv + ((i & 1) ? vc_he(nxv) : 0) + (i >> 1);
}
__host__ __device__ __forceinline__ void vxy(int st, int nxv, int& j, int& i) {
  j = st / nxv;
  const int r = st - j * nxv, he = vc_he(nxv);
  i = r < he ? 2 * r : 2 * (r - he) + 1;
}

// The storage order above as an index functor for vc_vertex_at.
struct VcStorageIndex {
  int nxv;
  __host__ __device__ int operator()(int j, int i) const { return vst(j, i, nxv); }
};

struct VcLevelArgs {
  int nx, ny;      // elements
  int stride;      // per-sample entries of the level's arrays
  int64_t plane;   // B * stride
};

// The vertices of colour (ci, cj) in thread order: rows j = cj, cj + 2, ...,
// columns i = ci, ci + 2, ...; count per sample.
__host__ __device__ __forceinline__ int vc_colour_rows(int nyv, int cj) { return (nyv - cj + 1) >> 1; }
__host__ __device__ __forceinline__ int vc_colour_cols(int nxv, int ci) { return (nxv - ci + 1) >> 1; }

// ---------------------------------------------------------------------------
// Residual and Jacobian of every vertex, scaled by inv_s (the fine level's
// 1 / (rho0 h^2 / tau)), at the storage-ordered states x, xo ([B][stride]).
// FINE: also F (double2, zero on the padding) and the per-CTA max |F| into
// rmax_part[s][stride / TPB] (stride a multiple of TPB); blocks of padding
// entries are zero.  Only samples with active[s] set are touched.  JAC =
// false: the residual alone (bit-identical to the JAC = true residual).
template <typename T, bool FINE, bool JAC = true>
__global__ void __launch_bounds__(TPB) k_vc_assemble_st(VcParams P, const Coef* __restrict__ coef, int B, int stride,
                                                        int64_t plane, double inv_s, const double2* __restrict__ x,
                                                        const double2* __restrict__ xo, const int* __restrict__ active,
                                                        double2* __restrict__ F, typename VT<T>::b4* __restrict__ J,
                                                        double* __restrict__ rmax_part) {
  typedef typename VT<T>::b4 B4;
  __shared__ double sh[40];
  const int nxv = P.nx + 1, NV = nxv * (P.ny + 1);
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / stride);
  if (FINE) {
    if (!active[s]) return;  // uniform over the CTA
  } else {
    if (e >= (int64_t)B * stride || !active[s]) return;
  }
  const int st = (int)(e - (int64_t)s * stride);
  double R[2] = {0.0, 0.0};
  double Jv[36];
  for (int q = 0; q < 36; ++q) Jv[q] = 0.0;
  if (st < NV) {
    int j, i;
    vxy(st, nxv, j, i);
    const Coef cf = coef[s];
    const VcCoef c{cf.phi, cf.kmu, cf.PD, cf.qin};
    const int64_t base = (int64_t)s * stride;
    vc_vertex_at<VcStorageIndex, JAC>(P, c, reinterpret_cast<const double*>(x + base),
                                       reinterpret_cast<const double*>(xo + base), j, i, R, J ? Jv : nullptr,
                                       VcStorageIndex{nxv});
  }
  if (FINE) {
    const double fm = R[0] * inv_s, fs = R[1] * inv_s;
    F[e] = make_double2(fm, fs);
    double loc = fmax(fabs(fm), fabs(fs));
    if (!(loc <= 1.0e300)) loc = INFINITY;
    const double bm = block_max_nonneg(loc, sh);
    if (threadIdx.x == 0) rmax_part[(int64_t)s * (stride / TPB) + st / TPB] = bm;
  }
  if (JAC && J) {
#pragma unroll
    for (int q = 0; q < 9; ++q)
      J[q * plane + e] = mkblk<B4>((T)(Jv[4 * q] * inv_s), (T)(Jv[4 * q + 1] * inv_s), (T)(Jv[4 * q + 2] * inv_s),
                                   (T)(Jv[4 * q + 3] * inv_s));
    B4 inv = mkblk<B4>((T)0, (T)0, (T)0, (T)0);
    if (st < NV) {
      const double a = Jv[16] * inv_s, b = Jv[17] * inv_s, c = Jv[18] * inv_s, d = Jv[19] * inv_s;
      const double idet = 1.0 / (a * d - b * c);
      inv = mkblk<B4>((T)(d * idet), (T)(-b * idet), (T)(-c * idet), (T)(a * idet));
    }
    J[9 * plane + e] = inv;
  }
}

// ---------------------------------------------------------------------------
// Face-once tile assembly (same arguments and outputs as k_vc_assemble_st,
// except that FINE's per-CTA maxima of |F| are per NT entries:
// rmax_part[s][stride / NT]).  A CTA of NT threads takes NT consecutive
// entries of the [B][stride] storage order.
// Every face of the grid has one source corner, the vertex that owns it:
//   E1 = element (j, i) face 0, E2 = element (j - 1, i) face 1 (both towards
//   the east neighbour), N1 = element (j, i) face 2, N2 = element (j, i - 1)
//   face 3 (both towards the north neighbour).
// Phase 1: every vertex evaluates the faces it owns into shared memory.
// Phase 2: every vertex adds its eight faces in vc_vertex_at's order - its
// own four, its west neighbour's E1 and E2, its south neighbour's N1 and N2 -
// read from shared memory, or evaluated again where the neighbour lies
// outside the CTA's range.  About 4.3 face evaluations per vertex instead of
// 8.  Vertices on x = Lx (Dirichlet in both equations) add no faces: their
// rows are replaced anyway.  Shared memory: 4 x NT face records (73.7 KB
// for NT = 128 with the Jacobian, so that three CTAs share an SM).
template <bool JAC>
struct VcFaceRec {
  double F, G, dF[JAC ? 8 : 1], dG[JAC ? 8 : 1];
};

template <bool JAC>
__device__ __forceinline__ void vc_eval_face(const VcParams& P, const VcCoef& C, const double2* xs, int nxv, int ey,
                                             int ex, int f, double ih, VcFaceRec<JAC>& r) {
  double p[4], c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 v = xs[vst(ey + (k >> 1), ex + (k & 1), nxv)];
    p[k] = v.x;
    c[k] = v.y;
  }
  vc_face<JAC>(P, C, p, c, f, ih, r.F, r.dF, r.G, r.dG);
}

template <typename T, bool FINE, bool JAC = true, int NT = 128>
__global__ void __launch_bounds__(NT) k_vc_assemble_tile(VcParams P, const Coef* __restrict__ coef, int B,
                                                          int stride, int64_t plane, double inv_s,
                                                          const double2* __restrict__ x,
                                                          const double2* __restrict__ xo,
                                                          const int* __restrict__ active, double2* __restrict__ F,
                                                          typename VT<T>::b4* __restrict__ J,
                                                          double* __restrict__ rmax_part) {
  typedef typename VT<T>::b4 B4;
  typedef VcFaceRec<JAC> Rec;
  extern __shared__ __align__(16) unsigned char vc_smem[];
  Rec* rec = reinterpret_cast<Rec*>(vc_smem);  // [4][NT]: E1, E2, N1, N2
  __shared__ double sh[40];
  const int nxv = P.nx + 1, NV = nxv * (P.ny + 1);
  const int64_t t0 = (int64_t)blockIdx.x * NT;
  const int64_t e = t0 + threadIdx.x;
  const int s = (int)(e / stride);
  if (FINE) {
    if (!active[s]) return;  // uniform over the CTA (stride % NT == 0)
  }
  const bool on = FINE || (e < (int64_t)B * stride && active[s]);
  const int st = (int)(e - (int64_t)s * stride);
  const bool vtx = on && st < NV;
  int j = 0, i = 0;
  if (vtx) vxy(st, nxv, j, i);
  const double2* xs = x + (int64_t)s * stride;
  VcCoef C{0.0, 0.0, 0.0, 0.0};
  if (vtx) {
    const Coef cf = coef[s];
    C = VcCoef{cf.phi, cf.kmu, cf.PD, cf.qin};
  }
  const double ih = 1.0 / P.h;
  const int tid = threadIdx.x;
  const bool faces = vtx && i < P.nx;  // x = Lx vertices own and add no face
  if (faces) {
    if (j < P.ny) {
      vc_eval_face<JAC>(P, C, xs, nxv, j, i, 0, ih, rec[tid]);            // E1
      vc_eval_face<JAC>(P, C, xs, nxv, j, i, 2, ih, rec[2 * NT + tid]);  // N1
      if (i > 0) vc_eval_face<JAC>(P, C, xs, nxv, j, i - 1, 3, ih, rec[3 * NT + tid]);  // N2
    }
    if (j > 0) vc_eval_face<JAC>(P, C, xs, nxv, j - 1, i, 1, ih, rec[NT + tid]);  // E2
  }
  __syncthreads();
  double Rm = 0.0, Rs = 0.0;
  double Jm[9][2], Js[9][2];
#pragma unroll
  for (int q = 0; q < 9; ++q) Jm[q][0] = Jm[q][1] = Js[q][0] = Js[q][1] = 0.0;
  if (vtx) {
    const double2 xv = xs[st];
    vc_storage<JAC>(P, C, xv.y, xo[(int64_t)s * stride + st].y, j, i, Rm, Rs, Jm, Js);
    if (faces) {
      // a neighbour's record: from shared memory if it is in this CTA's range
      const int64_t ew = (i > 0) ? (int64_t)s * stride + vst(j, i - 1, nxv) - t0 : -1;
      const int64_t es = (j > 0) ? (int64_t)s * stride + vst(j - 1, i, nxv) - t0 : -1;
      const bool w_in = ew >= 0 && ew < NT, s_in = es >= 0 && es < NT;
      Rec tmp;
      if (j < P.ny) {  // element (j, i), corner 0
        const Rec& e1 = rec[tid];
        vc_add_face<JAC>(1.0, 4, e1.F, e1.dF, e1.G, e1.dG, Rm, Rs, Jm, Js);
        const Rec& n1 = rec[2 * NT + tid];
        vc_add_face<JAC>(1.0, 4, n1.F, n1.dF, n1.G, n1.dG, Rm, Rs, Jm, Js);
      }
      if (j < P.ny && i > 0) {  // element (j, i - 1), corner 1
        const Rec* w1 = &tmp;
        if (w_in)
          w1 = &rec[ew];
        else
          vc_eval_face<JAC>(P, C, xs, nxv, j, i - 1, 0, ih, tmp);
        vc_add_face<JAC>(-1.0, 3, w1->F, w1->dF, w1->G, w1->dG, Rm, Rs, Jm, Js);
        const Rec& n2 = rec[3 * NT + tid];
        vc_add_face<JAC>(1.0, 3, n2.F, n2.dF, n2.G, n2.dG, Rm, Rs, Jm, Js);
      }
      if (j > 0) {  // element (j - 1, i), corner 2
        const Rec& e2 = rec[NT + tid];
        vc_add_face<JAC>(1.0, 1, e2.F, e2.dF, e2.G, e2.dG, Rm, Rs, Jm, Js);
        const Rec* s1 = &tmp;
        if (s_in)
          s1 = &rec[2 * NT + es];
        else
          vc_eval_face<JAC>(P, C, xs, nxv, j - 1, i, 2, ih, tmp);
        vc_add_face<JAC>(-1.0, 1, s1->F, s1->dF, s1->G, s1->dG, Rm, Rs, Jm, Js);
      }
      if (j > 0 && i > 0) {  // element (j - 1, i - 1), corner 3
        const Rec* w2 = &tmp;
        if (w_in)
          w2 = &rec[NT + ew];
        else
          vc_eval_face<JAC>(P, C, xs, nxv, j - 1, i - 1, 1, ih, tmp);
        vc_add_face<JAC>(-1.0, 0, w2->F, w2->dF, w2->G, w2->dG, Rm, Rs, Jm, Js);
        const Rec* s2 = &tmp;
        if (s_in)
          s2 = &rec[3 * NT + es];
        else
          vc_eval_face<JAC>(P, C, xs, nxv, j - 1, i - 1, 3, ih, tmp);
        vc_add_face<JAC>(-1.0, 0, s2->F, s2->dF, s2->G, s2->dG, Rm, Rs, Jm, Js);
      }
    }
    vc_boundary<JAC>(P, C, xv.x, xv.y, j, i, Rm, Rs, Jm, Js);
  }
  if (FINE) {
    const double fm = Rm * inv_s, fs = Rs * inv_s;
    F[e] = make_double2(fm, fs);
    double loc = fmax(fabs(fm), fabs(fs));
    if (!(loc <= 1.0e300)) loc = INFINITY;
    const double bm = block_max_nonneg(loc, sh);
    if (threadIdx.x == 0) rmax_part[(int64_t)s * (stride / NT) + st / NT] = bm;
  }
  if (JAC && J && on) {
#pragma unroll
    for (int q = 0; q < 9; ++q)
      J[q * plane + e] = mkblk<B4>((T)(Jm[q][0] * inv_s), (T)(Jm[q][1] * inv_s), (T)(Js[q][0] * inv_s),
                                   (T)(Js[q][1] * inv_s));
    B4 inv = mkblk<B4>((T)0, (T)0, (T)0, (T)0);
    if (vtx) {
      const double a = Jm[4][0] * inv_s, b = Jm[4][1] * inv_s, c = Js[4][0] * inv_s, d = Js[4][1] * inv_s;
      const double idet = 1.0 / (a * d - b * c);
      inv = mkblk<B4>((T)(d * idet), (T)(-b * idet), (T)(-c * idet), (T)(a * idet));
    }
    J[9 * plane + e] = inv;
  }
}

// Dynamic shared memory of k_vc_assemble_tile.
template <bool JAC, int NT = 128>
constexpr int vc_tile_smem() {
  return 4 * NT * (int)sizeof(VcFaceRec<JAC>);
}

// Coarse states by injection: x_c(J, I) = x_f(2J, 2I), for the iterate and
// (old != 0) the old state.
__global__ void __launch_bounds__(TPB) k_vc_inject(int B, int ncx, int ncy, int stride_f, int stride_c,
                                                   const double2* __restrict__ xf, double2* __restrict__ xc,
                                                   const int* __restrict__ active) {
  const int ncxv = ncx + 1, NVc = ncxv * (ncy + 1), nfxv = 2 * ncx + 1;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * NVc) return;
  const int s = (int)(e / NVc);
  if (!active[s]) return;
  const int stc = (int)(e - (int64_t)s * NVc);
  int J, I;
  vxy(stc, ncxv, J, I);
  xc[(int64_t)s * stride_c + stc] = xf[(int64_t)s * stride_f + vst(2 * J, 2 * I, nfxv)];
}

// r = b - sum over the 9 blocks A_q x_nb for vertex (j, i) (sample-relative arrays).
template <typename T>
__device__ __forceinline__ void vc_offdiag(int nxv, int nyv, int j, int i, int st, const typename VT<T>::b4* J,
                                          int64_t ps, const typename VT<T>::v2* x, T& r0, T& r1, bool centre) {
  typedef typename VT<T>::v2 V2;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q == 4 && !centre) continue;
    const int jj = j + q / 3 - 1, ii = i + q % 3 - 1;
    if (jj < 0 || jj >= nyv || ii < 0 || ii >= nxv) continue;
    const V2 xn = x[vst(jj, ii, nxv)];
    bmv_sub(J[q * ps + st], xn.x, xn.y, r0, r1);
  }
}

// One Gauss-Seidel pass over the vertices of colour (ci, cj):
//   x_v = C_v^{-1} (b_v - sum_{nb != v} A_nb x_nb).
// MODE 0 (the first pass from x = 0): launched over all vertices; the
// colour-(0, 0) vertices get C^{-1} b (their neighbours are all zero) and
// every other vertex is set to 0.  MODE 2: x = 0 everywhere (no smoothing).
template <typename T, int MODE>
__global__ void __launch_bounds__(TPB) k_vc_sweep(int B, VcLevelArgs L, int ci, int cj,
                                                  const typename VT<T>::b4* __restrict__ J,
                                                  const typename VT<T>::v2* __restrict__ b,
                                                  typename VT<T>::v2* __restrict__ x, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int nxv = L.nx + 1, nyv = L.ny + 1, NV = nxv * nyv;
  const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
  int s, j, i, st;
  if (MODE == 1) {
    const int nr = vc_colour_rows(nyv, cj), nc = vc_colour_cols(nxv, ci), per = nr * nc;
    if (t >= (int64_t)B * per) return;
    s = (int)(t / per);
    const int u = (int)(t - (int64_t)s * per), r = u / nc;
    j = cj + 2 * r;
    i = ci + 2 * (u - r * nc);
    st = vst(j, i, nxv);
  } else {
    if (t >= (int64_t)B * NV) return;
    s = (int)(t / NV);
    st = (int)(t - (int64_t)s * NV);
    vxy(st, nxv, j, i);
  }
  if (!active[s]) return;
  const int64_t base = (int64_t)s * L.stride;
  if (MODE == 2 || (MODE == 0 && ((i & 1) || (j & 1)))) {
    x[base + st] = mk2<V2>((T)0, (T)0);
    return;
  }
  const V2 bb = b[base + st];
  T r0 = bb.x, r1 = bb.y;
  if (MODE == 1) vc_offdiag<T>(nxv, nyv, j, i, st, J + base, L.plane, x + base, r0, r1, false);
  T y0, y1;
  bmv(J[9 * L.plane + base + st], r0, r1, y0, y1);
  x[base + st] = mk2<V2>(y0, y1);
}

// r = b - A x on every vertex of a level.
template <typename T>
__global__ void __launch_bounds__(TPB) k_vc_residual(int B, VcLevelArgs L, const typename VT<T>::b4* __restrict__ J,
                                                     const typename VT<T>::v2* __restrict__ b,
                                                     const typename VT<T>::v2* __restrict__ x,
                                                     typename VT<T>::v2* __restrict__ r, const int* __restrict__ active) {
  const int nxv = L.nx + 1, nyv = L.ny + 1, NV = nxv * nyv;
  const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (t >= (int64_t)B * NV) return;
  const int s = (int)(t / NV);
  if (!active[s]) return;
  const int st = (int)(t - (int64_t)s * NV);
  int j, i;
  vxy(st, nxv, j, i);
  const int64_t base = (int64_t)s * L.stride;
  const typename VT<T>::v2 bb = b[base + st];
  T r0 = bb.x, r1 = bb.y;
  vc_offdiag<T>(nxv, nyv, j, i, st, J + base, L.plane, x + base, r0, r1, true);
  r[base + st] = mk2<typename VT<T>::v2>(r0, r1);
}

// Full weighting (the transpose of bilinear prolongation): coarse vertex
// (J, I) gathers the fine residuals of vertices (2J + a, 2I + b), a, b in
// {-1, 0, 1}, with weights (1 - |a| / 2)(1 - |b| / 2); the entries of
// Dirichlet equations (p and c at x = Lx, c at x = 0) are set to zero.
template <typename T>
__global__ void __launch_bounds__(TPB) k_vc_restrict(int B, VcLevelArgs Lf, VcLevelArgs Lc,
                                                     const typename VT<T>::v2* __restrict__ rf,
                                                     typename VT<T>::v2* __restrict__ bc, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int ncxv = Lc.nx + 1, NVc = ncxv * (Lc.ny + 1), nfxv = Lf.nx + 1, nfyv = Lf.ny + 1;
  const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (t >= (int64_t)B * NVc) return;
  const int s = (int)(t / NVc);
  if (!active[s]) return;
  const int stc = (int)(t - (int64_t)s * NVc);
  int J, I;
  vxy(stc, ncxv, J, I);
  const V2* r = rf + (int64_t)s * Lf.stride;
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int a = -1; a <= 1; ++a)
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int j = 2 * J + a, i = 2 * I + b;
      if (j < 0 || j >= nfyv || i < 0 || i >= nfxv) continue;
      const T w = (T)((a == 0 ? 1.0 : 0.5) * (b == 0 ? 1.0 : 0.5));
      const V2 v = r[vst(j, i, nfxv)];
      s0 = fma_(w, v.x, s0);
      s1 = fma_(w, v.y, s1);
    }
  if (I == Lc.nx) s0 = s1 = (T)0;
  if (I == 0) s1 = (T)0;
  bc[(int64_t)s * Lc.stride + stc] = mk2<V2>(s0, s1);
}

// x_f += P x_c (bilinear interpolation from the coarse vertices).
template <typename T>
__global__ void __launch_bounds__(TPB) k_vc_prolong_add(int B, VcLevelArgs Lf, VcLevelArgs Lc,
                                                        typename VT<T>::v2* __restrict__ xf,
                                                        const typename VT<T>::v2* __restrict__ xc,
                                                        const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int nfxv = Lf.nx + 1, NVf = nfxv * (Lf.ny + 1), ncxv = Lc.nx + 1;
  const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (t >= (int64_t)B * NVf) return;
  const int s = (int)(t / NVf);
  if (!active[s]) return;
  const int st = (int)(t - (int64_t)s * NVf);
  int j, i;
  vxy(st, nfxv, j, i);
  const V2* c = xc + (int64_t)s * Lc.stride;
  // the coarse vertices around (j, i): (J0 | J1) x (I0 | I1), with J1 = J0
  // when j is even and I1 = I0 when i is even; weights 1, 1/2 or 1/4
  const int J0 = j >> 1, I0 = i >> 1, J1 = J0 + (j & 1), I1 = I0 + (i & 1);
  V2 sum = c[vst(J0, I0, ncxv)];
  if (i & 1) {
    const V2 e = c[vst(J0, I1, ncxv)];
    sum.x += e.x;
    sum.y += e.y;
  }
  if (j & 1) {
    const V2 n = c[vst(J1, I0, ncxv)];
    sum.x += n.x;
    sum.y += n.y;
    if (i & 1) {
      const V2 ne = c[vst(J1, I1, ncxv)];
      sum.x += ne.x;
      sum.y += ne.y;
    }
  }
  const T w = (T)(((j & 1) ? 0.5 : 1.0) * ((i & 1) ? 0.5 : 1.0));
  V2 v = xf[(int64_t)s * Lf.stride + st];
  v.x = fma_(w, sum.x, v.x);
  v.y = fma_(w, sum.y, v.y);
  xf[(int64_t)s * Lf.stride + st] = v;
}

// Coarsest grid (2 x 1 elements, 3 x 2 vertices, 12 unknowns u = 2 (j 3 + i)
// + var): the dense matrix from the 9-point blocks, inverted per sample by
// Gauss-Jordan elimination with partial pivoting in FP64; Ainv[s][12][12].
template <typename T>
__global__ void k_vc_coarse_inverse(int B, VcLevelArgs L, const typename VT<T>::b4* __restrict__ J,
                                    T* __restrict__ Ainv, const int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  constexpr int n = VC_COARSE_N;
  double M[n][2 * n];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) M[r][c] = (c - n == r) ? 1.0 : 0.0;
  const int64_t base = (int64_t)s * L.stride;
  for (int j = 0; j < 2; ++j)
    for (int i = 0; i < 3; ++i) {
      const int st = vst(j, i, 3), row = 2 * (j * 3 + i);
      for (int q = 0; q < 9; ++q) {
        const int jj = j + q / 3 - 1, ii = i + q % 3 - 1;
        if (jj < 0 || jj >= 2 || ii < 0 || ii >= 3) continue;
        const auto blk = J[q * L.plane + base + st];
        const int col = 2 * (jj * 3 + ii);
        M[row][col] = (double)blk.a00;
        M[row][col + 1] = (double)blk.a01;
        M[row + 1][col] = (double)blk.a10;
        M[row + 1][col + 1] = (double)blk.a11;
      }
    }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        const double tt = M[col][c];
        M[col][c] = M[piv][c];
        M[piv][c] = tt;
      }
    const double inv = 1.0 / M[col][col];
    for (int c = 0; c < 2 * n; ++c) M[col][c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      if (f != 0.0)
        for (int c = 0; c < 2 * n; ++c) M[r][c] -= f * M[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[(int64_t)s * n * n + r * n + c] = (T)M[r][n + c];
}

template <typename T>
__global__ void k_vc_coarse_solve(int B, VcLevelArgs L, const T* __restrict__ Ainv,
                                  const typename VT<T>::v2* __restrict__ b, typename VT<T>::v2* __restrict__ x,
                                  const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  constexpr int n = VC_COARSE_N;
  const int64_t base = (int64_t)s * L.stride;
  T v[n];
  for (int u = 0; u < 6; ++u) {
    const V2 bb = b[base + vst(u / 3, u % 3, 3)];
    v[2 * u] = bb.x;
    v[2 * u + 1] = bb.y;
  }
  const T* M = Ainv + (int64_t)s * n * n;
  for (int u = 0; u < 6; ++u) {
    T o[2];
    for (int h = 0; h < 2; ++h) {
      T acc = (T)0;
      for (int c = 0; c < n; ++c) acc = fma_(M[(2 * u + h) * n + c], v[c], acc);
      o[h] = acc;
    }
    x[base + vst(u / 3, u % 3, 3)] = mk2<V2>(o[0], o[1]);
  }
}

// y = A x on the fine level (stride a multiple of TPB; padding entries of y
// set to zero) with per-CTA partial dot products like k_spmv:
//   NDOT 1: <w1, y>;  NDOT 2: <w1, y>, <y, y>.
template <typename T, int NDOT>
__global__ void __launch_bounds__(TPB) k_vc_spmv(int B, VcLevelArgs L, const typename VT<T>::b4* __restrict__ J,
                                                 const typename VT<T>::v2* __restrict__ x,
                                                 typename VT<T>::v2* __restrict__ y,
                                                 const typename VT<T>::v2* __restrict__ w1, double* __restrict__ part,
                                                 int slot1, int slot2, const int* __restrict__ active) {
  typedef typename VT<T>::v2 V2;
  __shared__ double sh[TPB + 1];
  const int nxv = L.nx + 1, nyv = L.ny + 1, NV = nxv * nyv, nct = L.stride / TPB;
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  const int s = (int)(e / L.stride);
  if (!active[s]) return;  // uniform over the CTA
  const int st = (int)(e - (int64_t)s * L.stride);
  T r0 = (T)0, r1 = (T)0;
  if (st < NV) {
    int j, i;
    vxy(st, nxv, j, i);
    const int64_t base = (int64_t)s * L.stride;
    vc_offdiag<T>(nxv, nyv, j, i, st, J + base, L.plane, x + base, r0, r1, true);
    r0 = -r0;
    r1 = -r1;
  }
  const V2 yy = mk2<V2>(r0, r1);
  y[e] = yy;
  if (NDOT >= 1 && part) {
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

// Initial state: c = 0 and fresh-water hydrostatic p, except the x = Lx
// vertices, which hold their Dirichlet values (brine hydrostatic p, c = 1).
__global__ void __launch_bounds__(TPB) k_vc_init_state(int B, int nx, int ny, int stride, double h, double rho0g,
                                                       double rho1g, double Ly, double2* __restrict__ x) {
  const int nxv = nx + 1, NV = nxv * (ny + 1);
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * stride) return;
  const int s = (int)(e / stride);
  const int st = (int)(e - (int64_t)s * stride);
  if (st >= NV) {
    x[e] = make_double2(0.0, 0.0);
    return;
  }
  int j, i;
  vxy(st, nxv, j, i);
  const double y = j * h;
  x[e] = i == nx ? make_double2(rho1g * (Ly - y), 1.0) : make_double2(rho0g * (Ly - y), 0.0);
}

// QoIs of one sample per CTA: [0] the lumped salt mass sum_v phi |CV_v|
// rho(c_v) c_v, [1] c at the vertex (ip, jp); NaN for failed samples.
__global__ void __launch_bounds__(TPB) k_vc_qoi(int B, int nx, int ny, int stride, double h, double rho0,
                                                double drho, int ip, int jp, const Coef* __restrict__ coef,
                                                const double2* __restrict__ x, const int* __restrict__ status,
                                                double* __restrict__ qoi) {
  __shared__ double sh[40];
  const int s = blockIdx.x;
  if (s >= B) return;
  const int nxv = nx + 1, NV = nxv * (ny + 1);
  const double2* xs = x + (int64_t)s * stride;
  double acc = 0.0;
  for (int st = threadIdx.x; st < NV; st += blockDim.x) {
    int j, i;
    vxy(st, nxv, j, i);
    const int nel = (i > 0 && j > 0) + (i < nx && j > 0) + (i > 0 && j < ny) + (i < nx && j < ny);
    const double c = xs[st].y;
    acc += nel * (rho0 + drho * c) * c;
  }
  const double tot = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) {
    const bool bad = status[s] != 0;
    qoi[2 * (int64_t)s] = bad ? NAN : coef[s].phi * 0.25 * h * h * tot;
    qoi[2 * (int64_t)s + 1] = bad ? NAN : xs[vst(jp, ip, nxv)].y;
  }
}

// Natural [B][ny + 1][nx + 1] <-> storage [B][stride] order.
template <typename V2>
__global__ void __launch_bounds__(TPB) k_vc_to_storage(int B, int nx, int ny, int stride, const double2* __restrict__ in,
                                                       V2* __restrict__ out) {
  const int nxv = nx + 1, NV = nxv * (ny + 1);
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * NV) return;
  const int64_t s = e / NV;
  const int nat = (int)(e - s * NV);
  const int j = nat / nxv, i = nat - j * nxv;
  const double2 v = in[e];
  out[s * stride + vst(j, i, nxv)] = mk2<V2>(v.x, v.y);
}
template <typename V2>
__global__ void __launch_bounds__(TPB) k_vc_from_storage(int B, int nx, int ny, int stride, const V2* __restrict__ in,
                                                         double2* __restrict__ out) {
  const int nxv = nx + 1, NV = nxv * (ny + 1);
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * NV) return;
  const int64_t s = e / NV;
  const int nat = (int)(e - s * NV);
  const int j = nat / nxv, i = nat - j * nxv;
  const V2 v = in[s * stride + vst(j, i, nxv)];
  out[e] = make_double2((double)v.x, (double)v.y);
}

}  // namespace hk

namespace hk {

// Jacobian planes -> natural [B][ny + 1][nx + 1][9][2][2] FP64.
template <typename B4>
__global__ void __launch_bounds__(TPB) k_vc_blocks_out(int B, int nx, int ny, int stride, const B4* __restrict__ J,
                                                       int64_t plane, double* __restrict__ out) {
  const int nxv = nx + 1, NV = nxv * (ny + 1);
  const int64_t e = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (e >= (int64_t)B * NV) return;
  const int64_t s = e / NV;
  const int nat = (int)(e - s * NV);
  const int j = nat / nxv, i = nat - j * nxv;
  const int64_t src = s * stride + vst(j, i, nxv);
  for (int q = 0; q < 9; ++q) {
    const B4 b = J[q * plane + src];
    double* o = out + e * 36 + 4 * q;
    o[0] = (double)b.a00;
    o[1] = (double)b.a01;
    o[2] = (double)b.a10;
    o[3] = (double)b.a11;
  }
}

}  // namespace hk
