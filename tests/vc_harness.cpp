// Host build of the vertex-centred assembly of the CUDA path (henry_vc.cuh,
// plain arithmetic under __host__ __device__) for a CPU test: the same
// per-vertex function the kernel calls, looped over the grid of one sample.
#include "../paper_2302_07804_gb300/csrc/henry_vc.cuh"

extern "C" void vc_assemble_host(int nx, int ny, double h, double tau, double rho0, double rho1, double g,
                                 double Ly, double phi, double kmu, double PD, double qin, const double* x,
                                 const double* xo, double* R, double* J) {
  const VcParams P{nx, ny, h, tau, rho0, rho1 - rho0, rho1, g, Ly};
  const VcCoef C{phi, kmu, PD, qin};
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      const int v = j * (nx + 1) + i;
      vc_vertex(P, C, x, xo, j, i, R + 2 * v, J + 36 * v);
    }
}
