// Vertex-centred finite volumes for the Henry problem, the paper's own
// discretisation (Sec. 2.3: two unknowns (p, c) per grid vertex, a
// "consistent velocity" for Darcy's law, partial upwinding of the convective
// terms).  This file holds the per-vertex residual and 9-point 2x2-block
// Jacobian; the kernel that maps one thread to each (sample, vertex) is in
// henry_engine.cu.
//
// The scheme, as assembled here:
//  * vertices (j, i) at (i h, j h); the control volume of a vertex is the
//    union of the quarter-squares of its elements (lumped storage
//    phi h^2/4 per quarter);
//  * inside an element with corners 0 (bottom-left), 1 (bottom-right),
//    2 (top-left), 3 (top-right) and local coordinates (xi, eta), four faces
//    of length h/2 join the element centre to the edge midpoints:
//      face 0: corner 0 -> 1, normal +x, at (1/2, 1/4)
//      face 1: corner 2 -> 3, normal +x, at (1/2, 3/4)
//      face 2: corner 0 -> 2, normal +y, at (1/4, 1/2)
//      face 3: corner 1 -> 3, normal +y, at (3/4, 1/2);
//  * gradients of the bilinear interpolants; Darcy flux through a face
//    q.n = -(K/mu)(grad p . n + rho_g g n_y), where the gravity density
//    rho_g(xi) interpolates the mean densities of the element's two vertical
//    edges linearly in x, so that a pressure in trapezoidal hydrostatic
//    balance along the vertical grid lines has no vertical flux;
//  * mass flux F = rho_ip (q.n) h/2 with the bilinear density at the face
//    point; salt flux G = F c_f - rho_ip phi Dm (grad c . n) h/2 with the
//    partial upwind value c_f = (c_a + c_b)/2 + s sgn(F)(c_a - c_b)/2,
//    s = max(0, 1 - rho_ip phi Dm / (2 |F|));
//  * x = Lx: Dirichlet p = rho1 g (Ly - y), c = 1; x = 0: Dirichlet c = 0 and
//    the inflow rho0 q_in over each vertex's share of the boundary (h, h/2 at
//    the corners); y = 0, Ly: no flux (Sec. 2.1).  A Dirichlet equation is
//    (value - boundary value) x rho0 h^2/tau, with p in units of rho0 g Ly.
//
// Derivatives are forward-mode: every quantity of an element carries its
// derivatives with respect to the element's 8 unknowns (p0..p3, c0..c3).
// Upwind choices are taken on the values.
//
// The functions are plain arithmetic with __host__ __device__ qualifiers, so
// the same code also compiles as host C++.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

struct VcParams {
  int nx, ny;  // elements; the vertex grid is (ny + 1) x (nx + 1)
  double h, tau;
  double rho0, drho, rho1, g, Ly;
};

struct VcCoef {
  double phi, kmu, PD, qin;  // porosity, K / mu, phi Dm, inflow velocity
};

// A value with its derivatives with respect to the element's unknowns
// (slot k: p of corner k; slot 4 + k: c of corner k).
struct VcDual {
  double v;
  double d[8];
};

__host__ __device__ inline VcDual vd_zero() {
  VcDual r;
  r.v = 0.0;
  for (int k = 0; k < 8; ++k) r.d[k] = 0.0;
  return r;
}

__host__ __device__ inline VcDual vd_add(const VcDual& a, const VcDual& b) {
  VcDual r;
  r.v = a.v + b.v;
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}

__host__ __device__ inline VcDual vd_sub(const VcDual& a, const VcDual& b) {
  VcDual r;
  r.v = a.v - b.v;
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}

__host__ __device__ inline VcDual vd_scale(const VcDual& a, double s) {
  VcDual r;
  r.v = a.v * s;
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * s;
  return r;
}

__host__ __device__ inline VcDual vd_mul(const VcDual& a, const VcDual& b) {
  VcDual r;
  r.v = a.v * b.v;
  for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}

__host__ __device__ inline VcDual vd_div(const VcDual& a, const VcDual& b) {
  VcDual r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
  for (int k = 0; k < 8; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}

// w0 u0 + w1 u1 + w2 u2 + w3 u3
__host__ __device__ inline VcDual vd_lin4(const VcDual* u, double w0, double w1, double w2, double w3) {
  VcDual r = vd_scale(u[0], w0);
  r = vd_add(r, vd_scale(u[1], w1));
  r = vd_add(r, vd_scale(u[2], w2));
  return vd_add(r, vd_scale(u[3], w3));
}

// Mass and salt flux through face f of an element, from its corner a to its
// corner b, given the corners' p, c and rho.
__host__ __device__ inline void vc_face(const VcParams& P, const VcCoef& C, const VcDual* p, const VcDual* c,
                                        const VcDual* rho, int f, VcDual* F, VcDual* G) {
  const int a = (f == 1) ? 2 : ((f == 3) ? 1 : 0);
  const int b = (f == 0) ? 1 : ((f == 2) ? 2 : 3);
  const double xi = (f == 2) ? 0.25 : ((f == 3) ? 0.75 : 0.5);
  const double eta = (f == 0) ? 0.25 : ((f == 1) ? 0.75 : 0.5);
  const double ih = 1.0 / P.h;
  VcDual dp, dc, grav;
  if (f < 2) {  // normal +x
    dp = vd_scale(vd_lin4(p, -(1.0 - eta), 1.0 - eta, -eta, eta), ih);
    dc = vd_scale(vd_lin4(c, -(1.0 - eta), 1.0 - eta, -eta, eta), ih);
    grav = vd_zero();
  } else {  // normal +y
    dp = vd_scale(vd_lin4(p, -(1.0 - xi), -xi, 1.0 - xi, xi), ih);
    dc = vd_scale(vd_lin4(c, -(1.0 - xi), -xi, 1.0 - xi, xi), ih);
    grav = vd_scale(vd_lin4(rho, 0.5 * (1.0 - xi), 0.5 * xi, 0.5 * (1.0 - xi), 0.5 * xi), P.g);
  }
  const VcDual qn = vd_scale(vd_add(dp, grav), -C.kmu);
  const VcDual rho_ip = vd_lin4(rho, (1.0 - xi) * (1.0 - eta), xi * (1.0 - eta), (1.0 - xi) * eta, xi * eta);
  *F = vd_scale(vd_mul(rho_ip, qn), 0.5 * P.h);
  const VcDual Dc = vd_scale(rho_ip, C.PD);
  const bool pos = F->v >= 0.0;
  const VcDual absF = pos ? *F : vd_scale(*F, -1.0);
  VcDual s = vd_zero();
  if (Dc.v < 2.0 * absF.v) {
    s = vd_sub(vd_zero(), vd_div(Dc, vd_scale(absF, 2.0)));
    s.v += 1.0;
  }
  const double sg = pos ? 1.0 : -1.0;
  const VcDual cf = vd_add(vd_scale(vd_add(c[a], c[b]), 0.5), vd_scale(vd_mul(s, vd_sub(c[a], c[b])), 0.5 * sg));
  *G = vd_sub(vd_mul(*F, cf), vd_scale(vd_mul(Dc, dc), 0.5 * P.h));
}

// Vertex (j, i) -> index of its (p, c) pair in a sample's state array.
struct VcNaturalIndex {  // [ny + 1][nx + 1] row-major
  int nx1;
  __host__ __device__ int operator()(int j, int i) const { return j * nx1 + i; }
};

// Residual (R^m, R^s) of vertex (j, i) of one sample and, if J is not NULL,
// its Jacobian row blocks J[(dj + 1) * 3 + (di + 1)][eq][var] with respect to
// (p, c) of vertex (j + dj, i + di) (36 doubles; zero for neighbours outside
// the grid).  x, xo: the sample's states, pairs (p, c) at idx(j, i)
// (vc_vertex: natural order [ny + 1][nx + 1][2]).
template <typename IDX>
__host__ __device__ inline void vc_vertex_at(const VcParams& P, const VcCoef& C, const double* x, const double* xo,
                                             int j, int i, double* R, double* J, IDX idx) {
  double Rm = 0.0, Rs = 0.0;
  double Jm[9][2], Js[9][2];
  for (int q = 0; q < 9; ++q) Jm[q][0] = Jm[q][1] = Js[q][0] = Js[q][1] = 0.0;

  // lumped storage
  const double cv = x[2 * idx(j, i) + 1], cvo = xo[2 * idx(j, i) + 1];
  const double rho = P.rho0 + P.drho * cv, rho_o = P.rho0 + P.drho * cvo;
  const int nel = (i > 0 && j > 0) + (i < P.nx && j > 0) + (i > 0 && j < P.ny) + (i < P.nx && j < P.ny);
  const double w = C.phi * nel * (0.25 * P.h * P.h);
  Rm += w * (rho - rho_o) / P.tau;
  Jm[4][1] += w * P.drho / P.tau;
  Rs += w * (rho * cv - rho_o * cvo) / P.tau;
  Js[4][1] += w * (rho + P.drho * cv) / P.tau;

  // the faces of the (up to four) elements this vertex is a corner of
  for (int kv = 0; kv < 4; ++kv) {
    const int ey = j - (kv >> 1), ex = i - (kv & 1);
    if (ey < 0 || ey >= P.ny || ex < 0 || ex >= P.nx) continue;
    VcDual p[4], c[4], r[4];
    for (int k = 0; k < 4; ++k) {
      const int vk = idx(ey + (k >> 1), ex + (k & 1));
      p[k] = vd_zero();
      p[k].v = x[2 * vk];
      p[k].d[k] = 1.0;
      c[k] = vd_zero();
      c[k].v = x[2 * vk + 1];
      c[k].d[4 + k] = 1.0;
      r[k] = vd_zero();
      r[k].v = P.rho0 + P.drho * c[k].v;
      r[k].d[4 + k] = P.drho;
    }
    for (int f = 0; f < 4; ++f) {
      const int a = (f == 1) ? 2 : ((f == 3) ? 1 : 0);
      const int b = (f == 0) ? 1 : ((f == 2) ? 2 : 3);
      if (a != kv && b != kv) continue;
      VcDual F, G;
      vc_face(P, C, p, c, r, f, &F, &G);
      const double sgn = (a == kv) ? 1.0 : -1.0;  // out of this vertex's volume
      Rm += sgn * F.v;
      Rs += sgn * G.v;
      for (int k = 0; k < 4; ++k) {
        const int q = (ey + (k >> 1) - j + 1) * 3 + (ex + (k & 1) - i + 1);
        Jm[q][0] += sgn * F.d[k];
        Jm[q][1] += sgn * F.d[4 + k];
        Js[q][0] += sgn * G.d[k];
        Js[q][1] += sgn * G.d[4 + k];
      }
    }
  }

  // inflow of fresh water through x = 0
  if (i == 0) Rm -= P.rho0 * C.qin * ((j == 0 || j == P.ny) ? 0.5 * P.h : P.h);

  // Dirichlet equations
  const double sc = P.rho0 * P.h * P.h / P.tau;
  if (i == P.nx) {
    const double pb = P.rho1 * P.g * (P.Ly - j * P.h);
    const double pscale = P.rho0 * P.g * P.Ly;
    Rm = sc * (x[2 * idx(j, i)] - pb) / pscale;
    Rs = sc * (cv - 1.0);
    for (int q = 0; q < 9; ++q) Jm[q][0] = Jm[q][1] = Js[q][0] = Js[q][1] = 0.0;
    Jm[4][0] = sc / pscale;
    Js[4][1] = sc;
  } else if (i == 0) {
    Rs = sc * cv;
    for (int q = 0; q < 9; ++q) Js[q][0] = Js[q][1] = 0.0;
    Js[4][1] = sc;
  }

  R[0] = Rm;
  R[1] = Rs;
  if (J) {
    for (int q = 0; q < 9; ++q) {
      J[q * 4 + 0] = Jm[q][0];
      J[q * 4 + 1] = Jm[q][1];
      J[q * 4 + 2] = Js[q][0];
      J[q * 4 + 3] = Js[q][1];
    }
  }
}

__host__ __device__ inline void vc_vertex(const VcParams& P, const VcCoef& C, const double* x, const double* xo,
                                          int j, int i, double* R, double* J) {
  vc_vertex_at(P, C, x, xo, j, i, R, J, VcNaturalIndex{P.nx + 1});
}
