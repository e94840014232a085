// Method S1 (Section 5.2): the interface operator applied by subdomain
// solves. Every CG iteration applies, for every global point l and every
// Darcy subdomain i, the Dirichlet-to-Neumann map of the point's own
// realization to the current direction: the mortar data R_i p_l enter as
// Dirichlet data (Eqs. 5.5-5.6), one subdomain solve gives the pressure, and
// the flux functional of its boundary fluxes, Phi_i^l (R_i p_l) = -<u.n, xi>,
// is written to the per-unit products Y, where the CG's update gathers it as
// it gathers the products of the stored bases in Method S3. The solve uses
// the point's block factor (FP64 block inverses G_b of the scaled 5-point
// matrix, built once per point by the basis kernel in its factor-only mode):
// z_b = G_b (s_b u_b + D_{b-1} z_{b-1}), d_b = z_b + G_b (D_b d_{b+1}),
// x_b = s_b d_b. The recovery applies the same solve to lambda plus the
// particular data (the source and outer Dirichlet data, Eqs. 5.7-5.8) and
// writes the pressure field.
#include <algorithm>

#include "basis_dev.cuh"
#include "sfb_ctx.h"

namespace sfb {

namespace {

constexpr int kDtnThreads = 256;

struct DtnArgs {
  const SubDev* subs;
  const double* proj;
  const int* dofinfo;
  const ItemOff* off;
  const int64_t* gdof;
  const int64_t* ybase;
  const int* kmap;
  const int* pstat;
  const double* T;
  const double* G;
  const double* S;    // FP64 diagonal scalings
  const double* DL;   // FP64 scaled couplings to the row below
  const double* vin;  // [n_pts][n_lambda]: the CG direction, or lambda (recovery)
  double* Y;          // [n_pts][NY] per-unit products (product mode)
  double* field;      // [cnt][len_d] Darcy entries of points p0.. (recovery mode)
  const int64_t* cell_off;
  const int64_t* face_off;
  int64_t p0, n_lambda, NY, len_d, off_f;
  int ns;
  int recovery;
};

// z = G u for the np x np block G (FP64, symmetric, so row r is read as
// column r and consecutive threads read consecutive entries), u and z in
// shared memory; the threads split the sum into parts, added up in `part`.
__device__ __forceinline__ void block_matvec(const double* __restrict__ G, const double* u, double* z, int np,
                                             double* part) {
  const int t = threadIdx.x;
  if (np > kDtnThreads / 2) {   // one thread per row
    for (int r = t; r < np; r += blockDim.x) {
      double acc = 0.0;
      for (int k = 0; k < np; ++k) acc = fma(G[(int64_t)k * np + r], u[k], acc);
      z[r] = acc;
    }
    __syncthreads();
    return;
  }
  const int parts = kDtnThreads / np;   // >= 2
  const int r = t % np, q = t / np;
  if (q < parts) {
    const int k0 = q * np / parts, k1 = (q + 1) * np / parts;
    double acc = 0.0;
    for (int k = k0; k < k1; ++k) acc = fma(G[(int64_t)k * np + r], u[k], acc);
    part[q * np + r] = acc;
  }
  __syncthreads();
  for (int rr = t; rr < np; rr += blockDim.x) {
    double acc = 0.0;
    for (int qq = 0; qq < parts; ++qq) acc += part[qq * np + rr];
    z[rr] = acc;
  }
  __syncthreads();
}

// One CTA per (point p0 + blockIdx.x, Darcy subdomain blockIdx.y).
__global__ void __launch_bounds__(kDtnThreads) dtn_kernel(DtnArgs a) {
  extern __shared__ __align__(16) double dsm[];
  const int64_t l = a.p0 + blockIdx.x;
  const int sub = blockIdx.y;
  // product mode: the points still iterating; recovery: every point
  if (!a.recovery && a.pstat[l] != 0) return;
  const SubDev S = a.subs[sub];
  const int k = a.kmap[l * a.ns + sub];
  if (k < 0) return;
  const ItemOff off = a.off[S.item0 + k];
  const int nx = S.nx, ny = S.ny, R = S.R;
  const int np = (nx + kPanel - 1) & ~(kPanel - 1);
  Geo g;
  g.nx = nx; g.ny = ny; g.R = R; g.C = R + 1; g.Cp = (R + 4) & ~3; g.nc = nx * ny;
  g.Tx = a.T + off.t;
  g.Ty = g.Tx + (int64_t)ny * (nx + 1);
  const double* Gi = a.G + off.g;
  const double* Sg = a.S + off.sc;
  const double* DLg = a.DL + off.sc;
  // shared memory: z rows [ny][np] | c [R] | u [np] | d [np] | v [np] | parts | boundary x
  double* Z = dsm;
  double* c = Z + (int64_t)ny * np;
  double* u = c + ((R + 1) & ~1);
  double* d = u + np;
  double* v = d + np;
  double* part = v + np;
  double* xb = part + kDtnThreads;   // x on the bottom, right, top, left cells: nx, ny, nx, ny
  const int64_t* gd = a.gdof + S.gdof_off;
  for (int j = threadIdx.x; j < R; j += blockDim.x) c[j] = a.vin[l * a.n_lambda + gd[j]];
  __syncthreads();
  // forward sweep: z_b = G_b (s_b r_b + D_{b-1} z_{b-1}), r = B c (+ the particular data)
  for (int b = 0; b < ny; ++b) {
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      double ui = 0.0;
      if (i < nx) {
        double rhs = 0.0;
        if (b == 0 || b == ny - 1 || i == 0 || i == nx - 1)
          for (int j = 0; j < R; ++j) rhs = fma(c[j], rhs_entry(S, g, a.proj, b, i, j), rhs);
        if (a.recovery) rhs += rhs_entry(S, g, a.proj, b, i, R);
        ui = Sg[b * nx + i] * rhs;
        if (b > 0) ui = fma(DLg[b * nx + i], Z[(int64_t)(b - 1) * np + i], ui);
      }
      u[i] = ui;
    }
    __syncthreads();
    block_matvec(Gi + (int64_t)b * np * np, u, Z + (int64_t)b * np, np, part);
  }
  // backward sweep: d_b = z_b + G_b (D_b d_{b+1}), x_b = s_b d_b (d holds d_{b+1})
  double* fld = a.recovery ? a.field + (int64_t)blockIdx.x * a.len_d : nullptr;
  for (int b = ny - 1; b >= 0; --b) {
    if (b < ny - 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) v[i] = i < nx ? DLg[(b + 1) * nx + i] * d[i] : 0.0;
      __syncthreads();
      block_matvec(Gi + (int64_t)b * np * np, v, u, np, part);
    }
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      const double di = Z[(int64_t)b * np + i] + (b < ny - 1 ? u[i] : 0.0);
      d[i] = di;
      if (i < nx) {
        const double x = Sg[b * nx + i] * di;
        if (fld) fld[a.cell_off[sub] + (int64_t)b * nx + i] = x;
        if (b == 0) xb[i] = x;
        if (i == nx - 1) xb[nx + b] = x;
        if (b == ny - 1) xb[nx + ny + i] = x;
        if (i == 0) xb[2 * nx + ny + b] = x;
      }
    }
    __syncthreads();
  }
  if (a.recovery) {
    // normal velocities of every face (the Darcy flux field's layout: x-faces
    // [ny][nx+1], then y-faces [ny+1][nx], oriented +x / +y); on a mortar side
    // the outer value is the mortar pressure sum_j c_j <xi_j>_e, on an outer
    // Dirichlet side its data, on a no-flow side the flux is zero
    const double* P = fld + a.cell_off[sub];   // the pressures just written
    double* F = fld + a.off_f + a.face_off[sub];
    const double ihx = 1.0 / S.hx, ihy = 1.0 / S.hy;
    const int nxf = ny * (nx + 1), nf = nxf + (ny + 1) * nx;
    for (int e = threadIdx.x; e < nf; e += blockDim.x) {
      double val;
      if (e < nxf) {
        const int r = e / (nx + 1), ix = e - r * (nx + 1);
        const double t = g.Tx[e] * ihy;
        if (ix > 0 && ix < nx) {
          val = t * (P[r * nx + ix - 1] - P[r * nx + ix]);
        } else {
          const int side = ix == 0 ? 3 : 1;
          double gb = S.side_val[side];
          if (S.side_type[side] == SIDE_IFACE) {
            gb = 0.0;
            for (int j = 0; j < R; ++j) gb = fma(a.proj[S.proj_off[side] + (int64_t)r * R + j], c[j], gb);
          }
          const double fo = t * (P[r * nx + (ix == 0 ? 0 : nx - 1)] - gb);
          val = S.side_type[side] == SIDE_NOFLOW ? 0.0 : (ix == 0 ? -fo : fo);
        }
      } else {
        const int f = e - nxf, jr = f / nx, ix = f - jr * nx;
        const double t = g.Ty[f] * ihx;
        if (jr > 0 && jr < ny) {
          val = t * (P[(jr - 1) * nx + ix] - P[jr * nx + ix]);
        } else {
          const int side = jr == 0 ? 0 : 2;
          double gb = S.side_val[side];
          if (S.side_type[side] == SIDE_IFACE) {
            gb = 0.0;
            for (int j = 0; j < R; ++j) gb = fma(a.proj[S.proj_off[side] + (int64_t)ix * R + j], c[j], gb);
          }
          const double fo = t * (P[(jr == 0 ? 0 : ny - 1) * nx + ix] - gb);
          val = S.side_type[side] == SIDE_NOFLOW ? 0.0 : (jr == 0 ? -fo : fo);
        }
      }
      F[e] = val;
    }
    return;
  }
  // Phi c = -(flux functional of x less the mortar data), per local DOF
  const int* info = a.dofinfo + S.dofinfo_off;
  for (int ll = threadIdx.x; ll < R; ll += blockDim.x) {
    const int side = info[3 * ll], f0 = info[3 * ll + 1], f1 = info[3 * ll + 2];
    const double* Pj = a.proj + S.proj_off[side];
    double acc = 0.0;
    for (int f = f0; f < f1; ++f) {
      double t, xc;
      if (side == 0) { t = g.Ty[f]; xc = xb[f]; }
      else if (side == 1) { t = g.Tx[f * (nx + 1) + nx]; xc = xb[nx + f]; }
      else if (side == 2) { t = g.Ty[ny * nx + f]; xc = xb[nx + ny + f]; }
      else { t = g.Tx[f * (nx + 1)]; xc = xb[2 * nx + ny + f]; }
      double pc = 0.0;
      for (int j = 0; j < R; ++j) pc = fma(Pj[(int64_t)f * R + j], c[j], pc);
      acc = fma(Pj[(int64_t)f * R + ll] * t, xc - pc, acc);
    }
    a.Y[l * a.NY + a.ybase[sub] + ll] = -acc;
  }
}

// Weighted shifted sums of the recovered Darcy entries of cnt points (rows of
// field), added to S1 and S2; the first batch after a reset takes its first
// point's values as the shift.
__global__ void s1_moments_kernel(const double* __restrict__ field, int64_t cnt, int64_t len,
                                  const double* __restrict__ w, int first, double* shift, double* S1, double* S2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    const double sh = first ? field[e] : shift[e];
    double a1 = 0.0, a2 = 0.0;
    for (int64_t q = 0; q < cnt; ++q) {
      const double dv = field[q * len + e] - sh;
      a1 = fma(w[q], dv, a1);
      a2 = fma(w[q] * dv, dv, a2);
    }
    if (first) shift[e] = sh;
    S1[e] += a1;
    S2[e] += a2;
  }
}

}  // namespace

size_t dtn_smem_bytes(int max_nx, int max_ny, int max_R) {
  const int np = (max_nx + kPanel - 1) / kPanel * kPanel;
  return sizeof(double) * ((size_t)max_ny * np + ((max_R + 1) & ~1) + 3 * (size_t)np + kDtnThreads +
                           2 * (size_t)max_nx + 2 * (size_t)max_ny);
}

// Product mode (recovery = 0): Y (Darcy units) of the iterating points among
// p0 .. p0 + cnt - 1 = the subdomain solves' flux functionals of vin.
// Recovery mode: the Darcy entries (pressures, then normal velocities) of
// every one of those points for lambda = vin, as rows of field.
cudaError_t launch_dtn(sfb_ctx* c, const double* vin, int64_t p0, int64_t cnt, int recovery, double* field,
                       cudaStream_t st) {
  Dev& d = c->dev;
  DtnArgs a;
  a.subs = d.subs; a.proj = d.proj; a.dofinfo = d.dofinfo; a.off = d.off; a.gdof = d.gdof; a.ybase = d.ybase;
  a.kmap = d.kmap; a.pstat = d.pstat; a.T = d.T;
  a.G = reinterpret_cast<const double*>(d.G);
  a.S = reinterpret_cast<const double*>(d.S);
  a.DL = reinterpret_cast<const double*>(d.DL);
  a.vin = vin; a.Y = d.Y; a.field = field; a.cell_off = d.cell_off; a.face_off = d.face_off;
  a.p0 = p0; a.n_lambda = c->n_lambda; a.NY = c->NY; a.ns = (int)c->subs.size();
  a.len_d = c->mom_len[0] + c->mom_len[1];
  a.off_f = c->mom_len[0];
  a.recovery = recovery;
  int mnx = 1, mny = 1, mR = 1;
  for (const HostSub& H : c->subs) {
    mnx = std::max(mnx, H.nx);
    mny = std::max(mny, H.ny);
    mR = std::max(mR, (int)H.dofs.size());
  }
  const size_t smem = dtn_smem_bytes(mnx, mny, mR);
  cudaError_t e = cudaFuncSetAttribute(dtn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess || cnt == 0) return e;
  dtn_kernel<<<dim3((unsigned)cnt, (unsigned)a.ns), kDtnThreads, smem, st>>>(a);
  ++c->launches;
  return cudaGetLastError();
}

cudaError_t launch_s1_moments(sfb_ctx* c, const double* field, int64_t p0, int64_t cnt, int first,
                              cudaStream_t st) {
  Dev& d = c->dev;
  const int64_t len = c->mom_len[0] + c->mom_len[1];
  if (cnt == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((len + 255) / 256, 4 * 152);
  s1_moments_kernel<<<blocks, 256, 0, st>>>(field, cnt, len, d.w + p0, first, d.mom, d.mom + len, d.mom + 2 * len);
  ++c->launches;
  return cudaGetLastError();
}

}  // namespace sfb
