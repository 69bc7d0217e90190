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
// Derivatives are exact: each face's fluxes are differentiated by hand with
// respect to the element's 8 unknowns (p0..p3, c0..c3), the chain rule
// written out for the bilinear gradients, the interpolated densities and the
// partial-upwind share.  Upwind choices are taken on the values.
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

// Mass and salt flux through face f of an element, from its corner a to its
// corner b, and their derivatives with respect to the element's unknowns
// (slot k: p of corner k, slot 4 + k: c of corner k), given the corners'
// p and c; ih = 1 / h.  (Divisions are few: on GPUs with few FP64 units a
// division is a long sequence of FP64 instructions.)  JAC = false: F and G
// alone (the same arithmetic for the values; dF, dG untouched).
template <bool JAC = true>
__host__ __device__ inline void vc_face(const VcParams& P, const VcCoef& C, const double* p, const double* c, int f,
                                        double ih, double& F, double* dF, double& G, double* dG) {
  const int a = (f == 1) ? 2 : ((f == 3) ? 1 : 0);
  const int b = (f == 0) ? 1 : ((f == 2) ? 2 : 3);
  const double xi = (f == 2) ? 0.25 : ((f == 3) ? 0.75 : 0.5);
  const double eta = (f == 0) ? 0.25 : ((f == 1) ? 0.75 : 0.5);
  const double hh = 0.5 * P.h;
  // gradient weights (normal component, 1/h included), bilinear weights at
  // the face point, weights of the gravity density (y faces only)
  double gw[4], w[4], rg[4];
  if (f < 2) {  // normal +x
    gw[0] = -(1.0 - eta) * ih; gw[1] = (1.0 - eta) * ih; gw[2] = -eta * ih; gw[3] = eta * ih;
    rg[0] = rg[1] = rg[2] = rg[3] = 0.0;
  } else {  // normal +y
    gw[0] = -(1.0 - xi) * ih; gw[1] = -xi * ih; gw[2] = (1.0 - xi) * ih; gw[3] = xi * ih;
    rg[0] = rg[2] = 0.5 * (1.0 - xi); rg[1] = rg[3] = 0.5 * xi;
  }
  w[0] = (1.0 - xi) * (1.0 - eta); w[1] = xi * (1.0 - eta); w[2] = (1.0 - xi) * eta; w[3] = xi * eta;
  double dp = 0.0, dc = 0.0, grav = 0.0, rip = 0.0;
  for (int k = 0; k < 4; ++k) {
    const double rho = P.rho0 + P.drho * c[k];
    dp += gw[k] * p[k];
    dc += gw[k] * c[k];
    grav += rg[k] * rho;
    rip += w[k] * rho;
  }
  grav *= P.g;
  const double qn = -C.kmu * (dp + grav);
  F = rip * qn * hh;
  if (!JAC) {
    const double Dc = rip * C.PD;
    const bool pos = F >= 0.0;
    const double sg = pos ? 1.0 : -1.0, A = pos ? F : -F;
    double s = 0.0;
    if (Dc < 2.0 * A) s = 1.0 - Dc * (0.5 / A);
    const double cab = c[a] - c[b];
    const double cf = 0.5 * (c[a] + c[b]) + 0.5 * sg * s * cab;
    G = F * cf - Dc * dc * hh;
    return;
  }
  double dDc[8], ddc[8];
  for (int k = 0; k < 4; ++k) {
    dF[k] = rip * (-C.kmu * gw[k]) * hh;                                    // d/dp_k
    dF[4 + k] = (w[k] * P.drho * qn + rip * (-C.kmu * P.g * rg[k] * P.drho)) * hh;  // d/dc_k
    dDc[k] = 0.0;
    dDc[4 + k] = w[k] * P.drho * C.PD;
    ddc[k] = 0.0;
    ddc[4 + k] = gw[k];
  }
  const double Dc = rip * C.PD;
  // partial upwind share s = max(0, 1 - Dc / (2 |F|)), its sign from F
  const bool pos = F >= 0.0;
  const double sg = pos ? 1.0 : -1.0, A = pos ? F : -F;
  double s = 0.0, ds[8];
  for (int j = 0; j < 8; ++j) ds[j] = 0.0;
  if (Dc < 2.0 * A) {
    const double i2A = 0.5 / A;  // 1 / (2 |F|)
    s = 1.0 - Dc * i2A;
    const double u = Dc * sg * (2.0 * i2A);  // Dc sgn(F) / |F|
    for (int j = 0; j < 8; ++j) ds[j] = (u * dF[j] - dDc[j]) * i2A;
  }
  const double cab = c[a] - c[b];
  const double cf = 0.5 * (c[a] + c[b]) + 0.5 * sg * s * cab;
  G = F * cf - Dc * dc * hh;
  for (int j = 0; j < 8; ++j) {
    double dcf = 0.5 * sg * cab * ds[j];
    if (j == 4 + a) dcf += 0.5 + 0.5 * sg * s;
    if (j == 4 + b) dcf += 0.5 - 0.5 * sg * s;
    dG[j] = dF[j] * cf + F * dcf - (dDc[j] * dc + Dc * ddc[j]) * hh;
  }
}

// Vertex (j, i) -> index of its (p, c) pair in a sample's state array.
struct VcNaturalIndex {  // [ny + 1][nx + 1] row-major
  int nx1;
  __host__ __device__ int operator()(int j, int i) const { return j * nx1 + i; }
};

// The pieces of a vertex's residual row, in the order vc_vertex_at adds
// them (the face-once tile kernel adds the same pieces in the same order).
// Rows are Jm[q][var] (mass) and Js[q][var] (salt), q = (dj + 1) 3 + (di + 1)
// the neighbour (j + dj, i + di), var 0: p, 1: c.

// Lumped storage phi |CV| (rho c^k - rho_old c_old^k) / tau of vertex (j, i)
// (k = 0: mass, 1: salt) with cv, cvo its c and old c.
template <bool JAC = true>
__host__ __device__ inline void vc_storage(const VcParams& P, const VcCoef& C, double cv, double cvo, int j, int i,
                                           double& Rm, double& Rs, double Jm[9][2], double Js[9][2]) {
  const double rho = P.rho0 + P.drho * cv, rho_o = P.rho0 + P.drho * cvo;
  const int nel = (i > 0 && j > 0) + (i < P.nx && j > 0) + (i > 0 && j < P.ny) + (i < P.nx && j < P.ny);
  const double wt = C.phi * nel * (0.25 * P.h * P.h) / P.tau;  // lumped phi |CV| / tau
  Rm += wt * (rho - rho_o);
  Rs += wt * (rho * cv - rho_o * cvo);
  if (JAC) {
    Jm[4][1] += wt * P.drho;
    Js[4][1] += wt * (rho + P.drho * cv);
  }
}

// A face's fluxes out of the vertex's volume (sgn +1 when the vertex is the
// face's source corner, -1 when it is the target) and their derivatives with
// respect to the element's corners; q0 is the row slot of the element's
// corner 0.
template <bool JAC = true>
__host__ __device__ inline void vc_add_face(double sgn, int q0, double F, const double* dF, double G,
                                            const double* dG, double& Rm, double& Rs, double Jm[9][2],
                                            double Js[9][2]) {
  Rm += sgn * F;
  Rs += sgn * G;
  if (!JAC) return;
  for (int k = 0; k < 4; ++k) {
    const int q = q0 + (k >> 1) * 3 + (k & 1);
    Jm[q][0] += sgn * dF[k];
    Jm[q][1] += sgn * dF[4 + k];
    Js[q][0] += sgn * dG[k];
    Js[q][1] += sgn * dG[4 + k];
  }
}

// Inflow of fresh water through x = 0 and the Dirichlet rows (x = Lx: both
// equations; x = 0: salt); pv, cv the vertex's p and c.
template <bool JAC = true>
__host__ __device__ inline void vc_boundary(const VcParams& P, const VcCoef& C, double pv, double cv, int j, int i,
                                            double& Rm, double& Rs, double Jm[9][2], double Js[9][2]) {
  if (i == 0) Rm -= P.rho0 * C.qin * ((j == 0 || j == P.ny) ? 0.5 * P.h : P.h);
  const double sc = P.rho0 * P.h * P.h / P.tau;
  if (i == P.nx) {
    const double pb = P.rho1 * P.g * (P.Ly - j * P.h);
    const double pscale = P.rho0 * P.g * P.Ly;
    Rm = sc * (pv - pb) / pscale;
    Rs = sc * (cv - 1.0);
    if (JAC) {
      for (int q = 0; q < 9; ++q) Jm[q][0] = Jm[q][1] = Js[q][0] = Js[q][1] = 0.0;
      Jm[4][0] = sc / pscale;
      Js[4][1] = sc;
    }
  } else if (i == 0) {
    Rs = sc * cv;
    if (JAC) {
      for (int q = 0; q < 9; ++q) Js[q][0] = Js[q][1] = 0.0;
      Js[4][1] = sc;
    }
  }
}

// Residual (R^m, R^s) of vertex (j, i) of one sample and, if J is not NULL,
// its Jacobian row blocks J[(dj + 1) * 3 + (di + 1)][eq][var] with respect to
// (p, c) of vertex (j + dj, i + di) (36 doubles; zero for neighbours outside
// the grid).  x, xo: the sample's states, pairs (p, c) at idx(j, i)
// (vc_vertex: natural order [ny + 1][nx + 1][2]).
// JAC = false: the residual alone (J is ignored; the residual's arithmetic is
// the same as with JAC = true).
template <typename IDX, bool JAC = true>
__host__ __device__ inline void vc_vertex_at(const VcParams& P, const VcCoef& C, const double* x, const double* xo,
                                             int j, int i, double* R, double* J, IDX idx) {
  double Rm = 0.0, Rs = 0.0;
  double Jm[9][2], Js[9][2];
  for (int q = 0; q < 9; ++q) Jm[q][0] = Jm[q][1] = Js[q][0] = Js[q][1] = 0.0;
  const double cv = x[2 * idx(j, i) + 1], cvo = xo[2 * idx(j, i) + 1];
  vc_storage<JAC>(P, C, cv, cvo, j, i, Rm, Rs, Jm, Js);
  const double ih = 1.0 / P.h;

  // the faces of the (up to four) elements this vertex is a corner of
  for (int kv = 0; kv < 4; ++kv) {
    const int ey = j - (kv >> 1), ex = i - (kv & 1);
    if (ey < 0 || ey >= P.ny || ex < 0 || ex >= P.nx) continue;
    double p[4], c[4];
    for (int k = 0; k < 4; ++k) {
      const int vk = idx(ey + (k >> 1), ex + (k & 1));
      p[k] = x[2 * vk];
      c[k] = x[2 * vk + 1];
    }
    for (int f = 0; f < 4; ++f) {
      const int a = (f == 1) ? 2 : ((f == 3) ? 1 : 0);
      const int b = (f == 0) ? 1 : ((f == 2) ? 2 : 3);
      if (a != kv && b != kv) continue;
      double F, G, dF[8], dG[8];
      vc_face<JAC>(P, C, p, c, f, ih, F, dF, G, dG);
      const double sgn = (a == kv) ? 1.0 : -1.0;  // out of this vertex's volume
      vc_add_face<JAC>(sgn, (ey - j + 1) * 3 + (ex - i + 1), F, dF, G, dG, Rm, Rs, Jm, Js);
    }
  }
  vc_boundary<JAC>(P, C, x[2 * idx(j, i)], cv, j, i, Rm, Rs, Jm, Js);

  R[0] = Rm;
  R[1] = Rs;
  if (JAC && J) {
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
