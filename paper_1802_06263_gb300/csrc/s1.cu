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

// Partial sums of z = G u for the np x np block G (FP64, symmetric, so row r
// is read as column r and consecutive threads read consecutive entries):
// part[q][r] = sum over the q-th of `parts` slices of k of G[k][r] u[k].
__device__ __forceinline__ void block_partials(const double* __restrict__ G, const double* u, int np, int parts,
                                               double* part) {
  for (int idx = threadIdx.x; idx < parts * np; idx += blockDim.x) {
    const int q = idx / np, r = idx - q * np;
    const int k0 = q * np / parts, k1 = (q + 1) * np / parts;
    double a0 = 0.0, a1 = 0.0;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      a0 = fma(G[(int64_t)k * np + r], u[k], a0);
      a1 = fma(G[(int64_t)(k + 1) * np + r], u[k + 1], a1);
    }
    if (k < k1) a0 = fma(G[(int64_t)k * np + r], u[k], a0);
    part[idx] = a0 + a1;
  }
}

// One CTA per (point p0 + blockIdx.x, Darcy subdomain blockIdx.y). Each block
// row costs two barriers: one after the partial products, one after the
// threads r < np have summed row r and formed their entry of the next row's
// right-hand side.
__global__ void __launch_bounds__(kDtnThreads, 4) dtn_kernel(DtnArgs a) {
  extern __shared__ __align__(16) double dsm[];
  const int64_t l = a.p0 + blockIdx.x;
  const int sub = blockIdx.y;
  // product mode: the points still iterating; recovery: every point
  if (!a.recovery && a.pstat[l] != 0) return;
  const SubDev& S = a.subs[sub];
  const int k = a.kmap[l * a.ns + sub];
  if (k < 0) return;
  const ItemOff off = a.off[S.item0 + k];
  const int nx = S.nx, ny = S.ny, R = S.R;
  const int np = (nx + kPanel - 1) & ~(kPanel - 1);
  const int parts = max(1, kDtnThreads / np);
  const int nb = 2 * nx + 2 * ny;   // boundary faces: bottom nx, right ny, top nx, left ny
  Geo g;
  g.nx = nx; g.ny = ny; g.R = R; g.C = R + 1; g.Cp = (R + 4) & ~3; g.nc = nx * ny;
  g.src = S.source * S.hx * S.hy;
  g.Tx = a.T + off.t;
  g.Ty = g.Tx + (int64_t)ny * (nx + 1);
  const double* Gi = a.G + off.g;
  const double* Sg = a.S + off.sc;
  const double* DLg = a.DL + off.sc;
  // shared memory: z rows [ny][np] | c [R] | u [np] | part | mortar values gf [nb] | boundary x [nb]
  double* Z = dsm;
  double* c = Z + (int64_t)ny * np;
  double* u = c + ((R + 1) & ~1);
  double* part = u + np;
  double* gf = part + max(kDtnThreads, np);
  double* xb = gf + nb;
  const int64_t* gd = a.gdof + S.gdof_off;
  for (int j = threadIdx.x; j < R; j += blockDim.x) c[j] = a.vin[l * a.n_lambda + gd[j]];
  __syncthreads();
  // mortar pressure on every boundary face of an interface side, sum_j c_j <xi_j>_f
  for (int e = threadIdx.x; e < nb; e += blockDim.x) {
    const int side = e < nx ? 0 : e < nx + ny ? 1 : e < 2 * nx + ny ? 2 : 3;
    const int f = side == 0 ? e : side == 1 ? e - nx : side == 2 ? e - nx - ny : e - 2 * nx - ny;
    double v = 0.0;
    if (S.side_type[side] == SIDE_IFACE) {
      const double* P = a.proj + S.proj_off[side] + (int64_t)f * R;
      for (int j = 0; j < R; ++j) v = fma(P[j], c[j], v);
    }
    gf[e] = v;
  }
  __syncthreads();
  // entry r of row b of s (B c + particular data) + D_{b-1} z_{b-1}
  auto urow = [&](int b, int r, double zprev) -> double {
    if (r >= nx) return 0.0;
    double rhs = 0.0;
    if (b == 0) rhs = fma(g.Ty[r], gf[r], rhs);
    if (b == ny - 1) rhs = fma(g.Ty[ny * nx + r], gf[nx + ny + r], rhs);
    if (r == 0) rhs = fma(g.Tx[b * (nx + 1)], gf[2 * nx + ny + b], rhs);
    if (r == nx - 1) rhs = fma(g.Tx[b * (nx + 1) + nx], gf[nx + b], rhs);
    if (a.recovery) rhs += rhs_entry(S, g, a.proj, b, r, R);
    double v = Sg[b * nx + r] * rhs;
    if (b > 0) v = fma(DLg[b * nx + r], zprev, v);
    return v;
  };
  // forward sweep: z_b = G_b (s_b r_b + D_{b-1} z_{b-1})
  for (int r = threadIdx.x; r < np; r += blockDim.x) u[r] = urow(0, r, 0.0);
  __syncthreads();
  for (int b = 0; b < ny; ++b) {
    block_partials(Gi + (int64_t)b * np * np, u, np, parts, part);
    __syncthreads();
    for (int r = threadIdx.x; r < np; r += blockDim.x) {
      double z = 0.0;
      for (int q = 0; q < parts; ++q) z += part[q * np + r];
      Z[(int64_t)b * np + r] = z;
      if (b + 1 < ny) u[r] = urow(b + 1, r, z);
    }
    __syncthreads();
  }
  // backward sweep: d_b = z_b + G_b (D_{b+1} d_{b+1}), x_b = s_b d_b; u holds D_{b+1} d_{b+1}
  double* fld = a.recovery ? a.field + (int64_t)blockIdx.x * a.len_d : nullptr;
  auto emit = [&](int b, int r, double dv) {
    const double x = Sg[b * nx + r] * dv;
    if (fld) fld[a.cell_off[sub] + (int64_t)b * nx + r] = x;
    if (b == 0) xb[r] = x;
    if (r == nx - 1) xb[nx + b] = x;
    if (b == ny - 1) xb[nx + ny + r] = x;
    if (r == 0) xb[2 * nx + ny + b] = x;
  };
  for (int r = threadIdx.x; r < np; r += blockDim.x) {
    const double dv = Z[(int64_t)(ny - 1) * np + r];
    if (r < nx) emit(ny - 1, r, dv);
    u[r] = (ny > 1 && r < nx) ? DLg[(ny - 1) * nx + r] * dv : 0.0;
  }
  __syncthreads();
  for (int b = ny - 2; b >= 0; --b) {
    block_partials(Gi + (int64_t)b * np * np, u, np, parts, part);
    __syncthreads();
    for (int r = threadIdx.x; r < np; r += blockDim.x) {
      double dv = Z[(int64_t)b * np + r];
      for (int q = 0; q < parts; ++q) dv += part[q * np + r];
      if (r < nx) emit(b, r, dv);
      u[r] = (b > 0 && r < nx) ? DLg[b * nx + r] * dv : 0.0;
    }
    __syncthreads();
  }
  if (a.recovery) {
    // normal velocities of every face (the Darcy flux field's layout: x-faces
    // [ny][nx+1], then y-faces [ny+1][nx], oriented +x / +y); outside a
    // boundary face the value is the mortar pressure on an interface side,
    // the data on an outer Dirichlet side; a no-flow face carries no flux
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
          const double gb = S.side_type[side] == SIDE_IFACE ? gf[ix == 0 ? 2 * nx + ny + r : nx + r]
                                                             : S.side_val[side];
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
          const double gb = S.side_type[side] == SIDE_IFACE ? gf[jr == 0 ? ix : nx + ny + ix] : S.side_val[side];
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
    const int base = side == 0 ? 0 : side == 1 ? nx : side == 2 ? nx + ny : 2 * nx + ny;
    double acc = 0.0;
    for (int f = f0; f < f1; ++f) {
      const double t = side == 0 ? g.Ty[f] : side == 1 ? g.Tx[f * (nx + 1) + nx]
                     : side == 2 ? g.Ty[ny * nx + f] : g.Tx[f * (nx + 1)];
      acc = fma(Pj[(int64_t)f * R + ll] * t, xb[base + f] - gf[base + f], acc);
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
  const size_t np = (max_nx + kPanel - 1) / kPanel * kPanel;
  return sizeof(double) * ((size_t)max_ny * np + ((max_R + 1) & ~1) + np + std::max<size_t>(kDtnThreads, np) +
                           4 * ((size_t)max_nx + max_ny));
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
