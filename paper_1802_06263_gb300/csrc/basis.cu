// Stochastic multiscale flux basis: one CTA per (Darcy subdomain, local
// realization) item (Section 5.4, pre-computation loop, Steps 1-2).
//
// Per item the kernel
//  1. evaluates the truncated local KL expansion at the cell centres,
//     K = exp(E[Y] + sum_j sqrt(lambda_j) y_j f_j) (Eq. 2.13), and the face
//     transmissibilities of the cell-centred form of lowest-order RT with the
//     trapezoidal rule (harmonic means inside, half-cell values on Dirichlet
//     faces, zero on no-flow faces);
//  2. factors the 5-point matrix A, which is block tridiagonal with nx x nx
//     tridiagonal diagonal blocks and diagonal couplings between grid rows,
//     by the block LDL^T recurrence S_b = A_bb - D_{b-1} S_{b-1}^{-1} D_{b-1};
//     each S_b is inverted in place by the symmetric sweep operator and
//     G_b = S_b^{-1} is stored. Everything is applied to the diagonally
//     scaled matrix diag(A)^{-1/2} A diag(A)^{-1/2};
//  3. solves A X = B for the R + 1 right-hand sides at once: one column per
//     mortar DOF (Dirichlet data = the face averages of xi_j, Eqs. 5.5-5.6)
//     and one particular column (source and outer data, Eqs. 5.7-5.8), by a
//     forward sweep z_b = G_b (B_b + D_{b-1} z_{b-1}) and a backward sweep
//     x_b = z_b + G_b D_b x_{b+1};
//  4. in the mixed form (factor type float) refines X with FP64 residuals
//     r = B - A X of the 5-point stencil: X += A_32^{-1} r until
//     ||r||_F <= tol ||B||_F, stagnation, or the step limit.
// The flux-basis epilogue then projects the boundary fluxes of X back onto the
// mortar space (Section 5.2 step 3): Phi[l][j] = -<u(xi_j).n, xi_l>.
#include <math.h>

#include "sfb_internal.h"

namespace sfb {

namespace {

constexpr int kThreads = 256;

struct Geo {
  int nx, ny, R, C, Cp;
  const double* Tx;  // [ny][nx+1]
  const double* Ty;  // [ny+1][nx]
};

__device__ __forceinline__ double diag_of(const Geo& g, int b, int i) {
  return g.Tx[b * (g.nx + 1) + i] + g.Tx[b * (g.nx + 1) + i + 1] + g.Ty[b * g.nx + i] +
         g.Ty[(b + 1) * g.nx + i];
}

// Right-hand side entry B[(b, i)][c]: interface columns c < R carry
// T_e * P_side[face][c] on interface faces; column R carries the source and
// the outer Dirichlet data.
__device__ __forceinline__ double rhs_entry(const SubDev& S, const Geo& g, const double* proj,
                                            int b, int i, int c) {
  const int nx = g.nx, ny = g.ny;
  double v = 0.0;
  if (c < g.R) {
    if (b == 0 && S.side_type[0] == SIDE_IFACE) v += g.Ty[i] * proj[S.proj_off[0] + (int64_t)i * g.R + c];
    if (b == ny - 1 && S.side_type[2] == SIDE_IFACE)
      v += g.Ty[ny * nx + i] * proj[S.proj_off[2] + (int64_t)i * g.R + c];
    if (i == 0 && S.side_type[3] == SIDE_IFACE)
      v += g.Tx[b * (nx + 1)] * proj[S.proj_off[3] + (int64_t)b * g.R + c];
    if (i == nx - 1 && S.side_type[1] == SIDE_IFACE)
      v += g.Tx[b * (nx + 1) + nx] * proj[S.proj_off[1] + (int64_t)b * g.R + c];
  } else {
    v = S.source * S.hx * S.hy;
    if (b == 0 && S.side_type[0] == SIDE_DIRICHLET) v += g.Ty[i] * S.side_val[0];
    if (b == ny - 1 && S.side_type[2] == SIDE_DIRICHLET) v += g.Ty[ny * nx + i] * S.side_val[2];
    if (i == 0 && S.side_type[3] == SIDE_DIRICHLET) v += g.Tx[b * (nx + 1)] * S.side_val[3];
    if (i == nx - 1 && S.side_type[1] == SIDE_DIRICHLET) v += g.Tx[b * (nx + 1) + nx] * S.side_val[1];
  }
  return v;
}

// out[i][c] = base[i][c] + sum_k G[i][k] Y[k][c] for i < n, c < C; smem
// operands with row pitch n (G) and Cp (Y, out). `base` may alias `out`.
template <typename T>
__device__ __forceinline__ void gemm_acc(const T* __restrict__ G, const T* __restrict__ Y, T* out,
                                         const T* base, int n, int C, int Cp) {
  const int nct = (C + 3) >> 2;
  const int ntile = ((n + 3) >> 2) * nct;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
    const int i0 = (t / nct) * 4, c0 = (t % nct) * 4;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][q] = T(0);
    for (int k = 0; k < n; ++k) {
      T gv[4], yv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) gv[a] = (i0 + a < n) ? G[(i0 + a) * n + k] : T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) yv[q] = Y[k * Cp + c0 + q];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = fma(gv[a], yv[q], acc[a][q]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i0 + a < n && c0 + q < C) {
          T b0 = base ? base[(i0 + a) * Cp + c0 + q] : T(0);
          out[(i0 + a) * Cp + c0 + q] = b0 + acc[a][q];
        }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// In-place inversion of the SPD matrix in A (n x n, row pitch n) by the
// symmetric sweep operator: sweeping pivot k maps a_kk -> -1/a_kk,
// a_ik -> a_ik / a_kk, a_ij -> a_ij - a_ik a_kj / a_kk; after all pivots A
// holds -S^{-1}, negated at the end. Pivots of an SPD matrix stay positive;
// a non-positive pivot sets *bad.
template <typename T>
__device__ void sweep_invert(T* A, int n, T* vk, int* bad) {
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) vk[i] = A[i * n + k];
    __syncthreads();
    T piv = vk[k];
    if (!(piv > T(0))) {
      if (threadIdx.x == 0) *bad = 1;
      piv = T(1);
    }
    const T inv = T(1) / piv;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      T v;
      if (i == k && j == k) v = -inv;
      else if (i == k) v = vk[j] * inv;
      else if (j == k) v = vk[i] * inv;
      else v = A[e] - vk[i] * (vk[j] * inv);
      A[e] = v;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = -A[e];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) basis_kernel(BasisArgs a, int refine) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int bad_spd;
  const int item = blockIdx.x;
  if (item >= a.n_items) return;
  const int s = a.item_sub[item], kk = a.item_k[item];
  const SubDev S = a.subs[s];
  const int id = (int)S.item0 + kk;
  const ItemOff off = a.off[id];
  const int nx = S.nx, ny = S.ny, nc = nx * ny;
  Geo g;
  g.nx = nx; g.ny = ny; g.R = S.R; g.C = S.R + 1; g.Cp = (g.C + 3) & ~3;
  double* Tx = a.T + off.t;
  double* Ty = Tx + (int64_t)ny * (nx + 1);
  g.Tx = Tx; g.Ty = Ty;
  double* X = a.X + off.x;
  double* Dg = a.D + off.diag;
  T* Gg = reinterpret_cast<T*>(a.G) + off.g;
  T* Zg = reinterpret_cast<T*>(a.Z) + off.z;
  const int C = g.C, Cp = g.Cp;

  // smem: sc[nx] | scp[nx] (double) | Gs[nx*nx] | Ys[nx*Cp] | Zs[nx*Cp] | vk[nx] (T)
  double* sc = reinterpret_cast<double*>(smem_raw);
  double* scp = sc + nx;
  T* Gs = reinterpret_cast<T*>(scp + nx);
  T* Ys = Gs + nx * nx;
  T* Zs = Ys + nx * Cp;
  T* vk = Zs + nx * Cp;

  if (threadIdx.x == 0) bad_spd = 0;
  int st = 0;

  // ---- 1. permeability and transmissibilities ---------------------------
  {
    const int nt = S.n_term;
    const double* slam = a.kl + S.kl_off;
    const double* fx = slam + nt;
    const double* fy = fx + (int64_t)nt * nx;
    const double* yl = a.yloc + S.yloc_off + (int64_t)kk * nt;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int ix = c % nx, iy = c / nx;
      double Y = S.mean_y;
      for (int j = 0; j < nt; ++j) Y += slam[j] * yl[j] * fx[j * nx + ix] * fy[j * ny + iy];
      const double K = exp(Y);
      if (!(K > 0.0) || !isfinite(K)) st |= ST_NONFINITE;
      X[c] = K;  // scratch: X is written only after the factorization
    }
    __syncthreads();
    const double nu = S.nu;
    for (int f = threadIdx.x; f < ny * (nx + 1); f += blockDim.x) {
      const int iy = f / (nx + 1), ix = f - iy * (nx + 1);
      double t;
      if (ix == 0) t = S.side_type[3] != SIDE_NOFLOW ? 2.0 * X[iy * nx] * S.hy / (nu * S.hx) : 0.0;
      else if (ix == nx)
        t = S.side_type[1] != SIDE_NOFLOW ? 2.0 * X[iy * nx + nx - 1] * S.hy / (nu * S.hx) : 0.0;
      else {
        const double ka = X[iy * nx + ix - 1], kb = X[iy * nx + ix];
        t = (S.hy / S.hx) * 2.0 * ka * kb / (nu * (ka + kb));
      }
      Tx[f] = t;
    }
    for (int f = threadIdx.x; f < (ny + 1) * nx; f += blockDim.x) {
      const int iy = f / nx, ix = f - iy * nx;
      double t;
      if (iy == 0) t = S.side_type[0] != SIDE_NOFLOW ? 2.0 * X[ix] * S.hx / (nu * S.hy) : 0.0;
      else if (iy == ny)
        t = S.side_type[2] != SIDE_NOFLOW ? 2.0 * X[(ny - 1) * nx + ix] * S.hx / (nu * S.hy) : 0.0;
      else {
        const double ka = X[(iy - 1) * nx + ix], kb = X[iy * nx + ix];
        t = (S.hx / S.hy) * 2.0 * ka * kb / (nu * (ka + kb));
      }
      Ty[f] = t;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) Dg[c] = diag_of(g, c / nx, c % nx);
    __syncthreads();
  }

  // ---- 2. block LDL^T factorization of the scaled matrix -------------------
  for (int b = 0; b < ny; ++b) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      if (b > 0) scp[i] = sc[i];
      sc[i] = 1.0 / sqrt(Dg[b * nx + i]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
      const int i = e / nx, j = e - i * nx;
      double v = 0.0;
      if (i == j) v = 1.0;
      else if (j == i + 1) v = -Tx[b * (nx + 1) + j] * sc[i] * sc[j];
      else if (j == i - 1) v = -Tx[b * (nx + 1) + i] * sc[i] * sc[j];
      T w = T(v);
      if (b > 0) {
        const double di = scp[i] * Ty[b * nx + i] * sc[i];
        const double dj = scp[j] * Ty[b * nx + j] * sc[j];
        w = T(v - di * (double)Gs[e] * dj);
      }
      Gs[e] = w;
    }
    __syncthreads();
    sweep_invert<T>(Gs, nx, vk, &bad_spd);
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) Gg[(int64_t)b * nx * nx + e] = Gs[e];
    __syncthreads();
  }

  // ---- 3./4. solve, then refine with FP64 residuals --------------------------
  double bnorm2 = 0.0, rprev = 0.0;
  int it = 0;
  for (; it <= refine; ++it) {
    // forward sweep: r_b = B_b - (A x)_b; u_b = s_b r_b + dhat_{b-1} z_{b-1}; z_b = G_b u_b
    double rr = 0.0;
    for (int b = 0; b < ny; ++b) {
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        if (b > 0) scp[i] = sc[i];
        sc[i] = 1.0 / sqrt(Dg[b * nx + i]);
      }
      const T* Grow = Gg + (int64_t)b * nx * nx;
      for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) Gs[e] = Grow[e];
      __syncthreads();
      for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
        const int i = e / C, c = e - i * C;
        double r = rhs_entry(S, g, a.proj, b, i, c);
        if (it == 0) {
          bnorm2 += r * r;
        } else {
          const int64_t cell = (int64_t)b * nx + i;
          double ax = Dg[cell] * X[cell * C + c];
          if (i > 0) ax -= Tx[b * (nx + 1) + i] * X[(cell - 1) * C + c];
          if (i < nx - 1) ax -= Tx[b * (nx + 1) + i + 1] * X[(cell + 1) * C + c];
          if (b > 0) ax -= Ty[b * nx + i] * X[(cell - nx) * C + c];
          if (b < ny - 1) ax -= Ty[(b + 1) * nx + i] * X[(cell + nx) * C + c];
          r -= ax;
          rr += r * r;
        }
        double u = sc[i] * r;
        if (b > 0) u += scp[i] * Ty[b * nx + i] * sc[i] * (double)Zs[i * Cp + c];
        Ys[i * Cp + c] = T(u);
      }
      __syncthreads();
      gemm_acc<T>(Gs, Ys, Zs, nullptr, nx, C, Cp);
      __syncthreads();
      for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
        const int i = e / C, c = e - i * C;
        Zg[((int64_t)b * nx + i) * C + c] = Zs[i * Cp + c];
      }
    }
    if (it == 0) {
      bnorm2 = block_sum(bnorm2, red);
    } else {
      rr = block_sum(rr, red);
      const double rel = sqrt(rr / fmax(bnorm2, 1e-300));
      if (threadIdx.x == 0) a.resid[id] = rel;
      if (rel <= a.refine_tol) break;                      // converged: keep X
      if (it >= 2 && rel > 0.5 * rprev) { st |= ST_NOT_CONVERGED; break; }  // stagnated
      if (it == refine) { st |= ST_NOT_CONVERGED; break; }  // step limit: keep X
      rprev = rel;
    }
    __syncthreads();
    // backward sweep: d_b = z_b + G_b (dhat_b .* d_{b+1}); x_b += s_b d_b
    double dn2 = 0.0, xn2 = 0.0;
    for (int b = ny - 1; b >= 0; --b) {
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        sc[i] = 1.0 / sqrt(Dg[b * nx + i]);
        if (b < ny - 1) scp[i] = 1.0 / sqrt(Dg[(b + 1) * nx + i]);
      }
      const T* Grow = Gg + (int64_t)b * nx * nx;
      for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) Gs[e] = Grow[e];
      __syncthreads();
      if (b < ny - 1) {
        for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
          const int i = e / C, c = e - i * C;
          const double dh = sc[i] * Ty[(b + 1) * nx + i] * scp[i];
          Ys[i * Cp + c] = T(dh * (double)Zs[i * Cp + c]);
        }
        for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
          const int i = e / C, c = e - i * C;
          Zs[i * Cp + c] = Zg[((int64_t)b * nx + i) * C + c];
        }
        __syncthreads();
        gemm_acc<T>(Gs, Ys, Zs, Zs, nx, C, Cp);
      } else {
        for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
          const int i = e / C, c = e - i * C;
          Zs[i * Cp + c] = Zg[((int64_t)b * nx + i) * C + c];
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nx * C; e += blockDim.x) {
        const int i = e / C, c = e - i * C;
        const int64_t idx = ((int64_t)b * nx + i) * C + c;
        const double d = sc[i] * (double)Zs[i * Cp + c];
        if (it == 0) {
          X[idx] = d;
        } else {
          const double xo = X[idx];
          X[idx] = xo + d;
          if (it == 1) { dn2 += d * d; xn2 += (xo + d) * (xo + d); }
        }
      }
      __syncthreads();
    }
    if (it == 1) {
      dn2 = block_sum(dn2, red);
      xn2 = block_sum(xn2, red);
      if (threadIdx.x == 0) a.corr1[id] = sqrt(dn2 / fmax(xn2, 1e-300));
    }
  }
  if (threadIdx.x == 0) a.nref[id] = it > refine ? refine : it;
  // NaN check on the result
  for (int e = threadIdx.x; e < nc * C; e += blockDim.x)
    if (!isfinite(X[e])) st |= ST_NONFINITE;
  __syncthreads();
  if (bad_spd) st |= ST_NOT_SPD;
  if (st) atomicOr(&a.status[id], st);
}

// Phi[l][j] = -sum_e P[e][l] T_e (X[c_e][j] - P[e][j]) (j < R) and
// g[l] = sum_e P[e][l] T_e X[c_e][R], the sum running over the faces e of the
// side that carries mortar DOF l and lying in the support of xi_l.
__global__ void flux_epilogue_kernel(BasisArgs a) {
  const int item = blockIdx.x;
  if (item >= a.n_items) return;
  const int s = a.item_sub[item], kk = a.item_k[item];
  const SubDev S = a.subs[s];
  const int id = (int)S.item0 + kk;
  const ItemOff off = a.off[id];
  const int nx = S.nx, ny = S.ny, R = S.R, C = R + 1;
  const double* Tx = a.T + off.t;
  const double* Ty = Tx + (int64_t)ny * (nx + 1);
  const double* X = a.X + off.x;
  double* phi = a.phi + off.phi;
  const int* info = a.dofinfo + S.dofinfo_off;
  for (int e2 = threadIdx.x; e2 < R * C; e2 += blockDim.x) {
    const int l = e2 / C, j = e2 - l * C;
    const int side = info[3 * l], f0 = info[3 * l + 1], f1 = info[3 * l + 2];
    const double* P = a.proj + S.proj_off[side];
    double acc = 0.0;
    for (int f = f0; f < f1; ++f) {
      int cell;
      double t;
      if (side == 0) { cell = f; t = Ty[f]; }
      else if (side == 2) { cell = (ny - 1) * nx + f; t = Ty[ny * nx + f]; }
      else if (side == 3) { cell = f * nx; t = Tx[f * (nx + 1)]; }
      else { cell = f * nx + nx - 1; t = Tx[f * (nx + 1) + nx]; }
      const double pl = P[(int64_t)f * R + l];
      const double pj = (j < R) ? P[(int64_t)f * R + j] : 0.0;
      acc += pl * t * (X[(int64_t)cell * C + j] - pj);
    }
    if (j < R) phi[l * R + j] = -acc;
    else phi[R * R + l] = acc;
  }
}

template <typename T>
size_t basis_smem(int max_nx, int max_cols) {
  const int cp = (max_cols + 3) & ~3;
  return sizeof(double) * 2 * max_nx + sizeof(T) * ((size_t)max_nx * max_nx + 2 * (size_t)max_nx * cp + max_nx);
}

template <typename T>
cudaError_t launch_basis(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st) {
  const size_t smem = basis_smem<T>(max_nx, max_cols);
  cudaError_t e = cudaFuncSetAttribute(basis_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  basis_kernel<T><<<a.n_items, kThreads, smem, st>>>(a, refine);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_basis_fp64(const BasisArgs& a, int max_nx, int max_cols, cudaStream_t st) {
  return launch_basis<double>(a, max_nx, max_cols, 0, st);
}

cudaError_t launch_basis_mixed(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st) {
  return launch_basis<float>(a, max_nx, max_cols, refine, st);
}

cudaError_t launch_flux_epilogue(const BasisArgs& a, int /*max_R*/, cudaStream_t st) {
  flux_epilogue_kernel<<<a.n_items, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

size_t basis_smem_bytes(int prec_fp64, int max_nx, int max_cols) {
  return prec_fp64 ? basis_smem<double>(max_nx, max_cols) : basis_smem<float>(max_nx, max_cols);
}

}  // namespace sfb
