// Host-side set-up of the library: geometry and mortar maps (Section 3.1,
// Section 3.3), KL eigenpairs (Section 2.1, Eq. 6.1) and collocation grids
// (Section 4). Pure FP64 host arithmetic that runs once per problem; the
// per-realization work all runs in the CUDA kernels.
#pragma once

#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

namespace sfb {

struct HostIface {
  int kind;            // 0 Stokes-Darcy, 1 vertical Darcy-Darcy, 2 horizontal Darcy-Darcy
  double s0, s1;       // segment along its coordinate (x for horizontal, y for vertical)
  int n_el, deg;
  int sub_a, side_a;   // first side (sub = -1: Stokes)
  int sub_b, side_b;
  int64_t off;         // first global mortar DOF
  int n_dof;
};

struct HostSub {
  int nx, ny;
  double x0, x1, y0, y1, hx, hy;
  int side_type[4];
  double side_val[4];
  int side_iface[4];          // interface index per side or -1
  std::vector<int64_t> dofs;  // local -> global mortar DOF (increasing)
  double source;
  // KL
  int n_term = 0;
  double sigma2 = 0, eta1 = 0, eta2 = 0, mean_y = 0;
  std::vector<double> slam;   // sqrt(lambda_j)
  std::vector<double> lam;    // lambda_j
  std::vector<double> fx, fy; // [nt][nx], [nt][ny] at cell centres
  // dense face projections per side: [faces][R]
  std::vector<double> proj[4];
  std::vector<int> dofinfo;   // per local DOF: side, first face, end face
};

// Exact face averages (1/|f|) int_f xi ds of the mortar basis functions of
// one interface on the faces [f0 + i h, f0 + (i+1) h), i < n_faces; writes
// columns (local DOF positions) `cols` of a [n_faces][ld] array.
void face_projection(const HostIface& itf, double f0, double h, int n_faces,
                     const std::vector<int>& cols, int ld, double* out);

// Integral of the mortar basis functions of `itf` times a quadratic Lagrange
// shape on [xa, xb] (node q = 0, 1, 2 at xa, midpoint, xb): out[n_dof].
void mortar_times_p2(const HostIface& itf, double xa, double xb, int q, double* out);

// 1-D KL of exp(-|x - x'| / eta) on a segment of length L: the n largest
// eigenvalues with their angular frequencies and parities (0 even, 1 odd).
void kl_1d_host(double L, double eta, int n, std::vector<double>& omega,
                std::vector<double>& lam, std::vector<int>& parity);
double kl_1d_eval_host(double x, double L, double omega, int parity);

// Probabilists' Gauss-Hermite rule (nodes ascending, weights summing to 1).
void gauss_hermite_host(int m, std::vector<double>& x, std::vector<double>& w);

struct Grid {
  int n_dim = 0;
  std::vector<double> y;  // [n_pts][n_dim]
  std::vector<double> w;
  int64_t n_pts() const { return n_dim ? (int64_t)w.size() : 0; }
};

void tensor_grid_host(const std::vector<int>& ms, Grid& out);
void smolyak_grid_host(int n_dim, int lmax, const std::vector<int>& rule, Grid& out);
int rule_size_host(int p, const std::vector<int>& rule);

// Quantised coordinate key shared by the grid builders and the device lookup.
inline int64_t qkey(double v) {
  double r = v * 1e12;
  int64_t k = (int64_t)(r < 0 ? r - 0.5 : r + 0.5);
  return k;
}

}  // namespace sfb
