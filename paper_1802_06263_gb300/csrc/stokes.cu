// Deterministic Stokes subdomain basis on the GPU (Section 5.4: N_real = 1
// for Stokes subdomains). The Taylor-Hood saddle-point system assembled on
// the host (stokes_host.cpp) is scattered into a dense FP64 matrix, factored
// by a blocked right-looking LU with partial pivoting, and solved for the
// R_s + 1 right-hand sides (one normal-stress load per mortar DOF, Eqs.
// 5.1-5.2, and the inflow-driven particular problem, Eqs. 5.3-5.4). The flux
// basis is Phi_s[l][j] = -<u(xi_j).n, xi_l>, g_s[l] = <u_bar.n, xi_l>.
#include <algorithm>

#include "sfb_ctx.h"

namespace sfb {

namespace {

constexpr int kNB = 64;

__global__ void scatter_triplets(double* A, int n, const int* r, const int* c, const double* v, int64_t nnz) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
    A[(int64_t)r[t] * n + c[t]] = v[t];
}

// Factor the panel A[j0:n, j0:j0+jb] with partial pivoting (one CTA).
__global__ void __launch_bounds__(1024) lu_panel(double* A, int n, int j0, int jb, int* piv, int* status) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int prow;
  for (int j = j0; j < j0 + jb; ++j) {
    // pivot search: largest |A[i][j]|, i >= j (smallest index on ties)
    double best = -1.0;
    int bi = j;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      const double a = fabs(A[(int64_t)i * n + j]);
      if (a > best) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int nw = blockDim.x >> 5;
      best = threadIdx.x < nw ? sv[threadIdx.x] : -1.0;
      bi = threadIdx.x < nw ? si[threadIdx.x] : n;
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        prow = bi;
        piv[j] = bi;
        if (!(best > 0.0)) atomicOr(status, 2);
      }
    }
    __syncthreads();
    const int p = prow;
    if (p != j)
      for (int k = j0 + threadIdx.x; k < j0 + jb; k += blockDim.x) {
        const double t = A[(int64_t)j * n + k];
        A[(int64_t)j * n + k] = A[(int64_t)p * n + k];
        A[(int64_t)p * n + k] = t;
      }
    __syncthreads();
    const double d = A[(int64_t)j * n + j];
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    // scale the column and update the rest of the panel (rank-1)
    const int ncol = j0 + jb - (j + 1);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double* row = A + (int64_t)i * n;
      const double l = row[j] * inv;
      row[j] = l;
      const double* urow = A + (int64_t)j * n;
      for (int k = 0; k < ncol; ++k) row[j + 1 + k] -= l * urow[j + 1 + k];
    }
    __syncthreads();
  }
}

// Apply the panel's row interchanges to the columns outside the panel.
__global__ void lu_swap(double* A, int n, int j0, int jb, const int* piv) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n || (col >= j0 && col < j0 + jb)) return;
  for (int j = j0; j < j0 + jb; ++j) {
    const int p = piv[j];
    if (p != j) {
      const double t = A[(int64_t)j * n + col];
      A[(int64_t)j * n + col] = A[(int64_t)p * n + col];
      A[(int64_t)p * n + col] = t;
    }
  }
}

// A12 <- L11^{-1} A12 with L11 unit lower triangular (one thread per column).
__global__ void trsm_unit_lower(const double* L, int ldl, double* B, int ldb, int jb, int ncols) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  for (int i = 0; i < jb; ++i) {
    double v = B[(int64_t)i * ldb + col];
    for (int k = 0; k < i; ++k) v -= L[(int64_t)i * ldl + k] * B[(int64_t)k * ldb + col];
    B[(int64_t)i * ldb + col] = v;
  }
}

// B <- U11^{-1} B with U11 upper triangular (one thread per column).
__global__ void trsm_upper(const double* U, int ldu, double* B, int ldb, int jb, int ncols) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  for (int i = jb - 1; i >= 0; --i) {
    double v = B[(int64_t)i * ldb + col];
    for (int k = i + 1; k < jb; ++k) v -= U[(int64_t)i * ldu + k] * B[(int64_t)k * ldb + col];
    B[(int64_t)i * ldb + col] = v / U[(int64_t)i * ldu + i];
  }
}

// C[M x N] -= A[M x K] B[K x N], K <= 64, row-major with leading dims;
// 64 x 64 output tile per CTA, K in chunks of 32.
__global__ void __launch_bounds__(256) gemm_sub(const double* A, int lda, const double* B, int ldb, double* C,
                                                int ldc, int M, int N, int K) {
  __shared__ double As[64][33];
  __shared__ double Bs[32][65];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;  // 16 x 16 threads, 4 x 4 outputs each
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
      const int r = e / 32, q = e % 32;
      As[r][q] = (m0 + r < M && k0 + q < K) ? A[(int64_t)(m0 + r) * lda + k0 + q] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
      const int r = e / 64, q = e % 64;
      Bs[r][q] = (k0 + r < K && n0 + q < N) ? B[(int64_t)(k0 + r) * ldb + n0 + q] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < 32; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[tr * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + tr * 4 + i, q = n0 + tc + 16 * j;
      if (r < M && q < N) C[(int64_t)r * ldc + q] -= acc[i][j];
    }
}

__global__ void apply_pivots(double* B, int ldb, int n, int ncols, const int* piv) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  for (int j = 0; j < n; ++j) {
    const int p = piv[j];
    if (p != j) {
      const double t = B[(int64_t)j * ldb + col];
      B[(int64_t)j * ldb + col] = B[(int64_t)p * ldb + col];
      B[(int64_t)p * ldb + col] = t;
    }
  }
}

__global__ void expand_solution(const double* sol, int Cs, int n_free, const int* free_to_full, int n_u,
                                const double* dir, double* U, double* P, int n_p) {
  // Dirichlet rows: zero for the basis columns, the data for the particular one
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n_u * Cs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(e % Cs);
    U[e] = col == Cs - 1 ? dir[e / Cs] : 0.0;
  }
}

__global__ void expand_free(const double* sol, int Cs, int n_free, const int* free_to_full, int n_u, double* U,
                            double* P) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n_free * Cs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / Cs), col = (int)(e % Cs);
    const int d = free_to_full[f];
    if (d < n_u) U[(int64_t)d * Cs + col] = sol[e];
    else P[(int64_t)(d - n_u) * Cs + col] = sol[e];
  }
}

// Phi_s[l][j] = -sum_b nb[b][l] U[(y, node_b)][j], g_s[l] = sum_b nb[b][l] U[(y, node_b)][Rs]
__global__ void stokes_flux(const double* nb, const int* nb_node, int nbn, int Rs, const double* U, int n_nodes,
                            double* phi, float* phi32) {
  const int Cs = Rs + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Rs * Cs; e += gridDim.x * blockDim.x) {
    const int l = e / Cs, j = e % Cs;
    double acc = 0.0;
    for (int b = 0; b < nbn; ++b) acc += nb[b * Rs + l] * U[(int64_t)(n_nodes + nb_node[b]) * Cs + j];
    const int o = j < Rs ? l * Rs + j : Rs * Rs + l;
    const double v = j < Rs ? -acc : acc;
    phi[o] = v;
    phi32[o] = (float)v;
  }
}

}  // namespace

cudaError_t stokes_solve_device(sfb_ctx* c) {
  const StokesHost& S = c->stokes;
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  const int n = S.n_free, Rs = (int)S.dofs.size(), Cs = Rs + 1;
  cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  CK(cudaMemsetAsync(d.s_mat, 0, sizeof(double) * (size_t)n * n, st));
  CK(cudaMemsetAsync(d.s_status, 0, sizeof(int) * 4, st));
  CK(cudaMemcpyAsync(d.s_tr_row, S.tr_row.data(), sizeof(int) * S.tr_row.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_tr_col, S.tr_col.data(), sizeof(int) * S.tr_col.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_tr_val, S.tr_val.data(), sizeof(double) * S.tr_val.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_rhs, S.rhs.data(), sizeof(double) * S.rhs.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_dir, S.dir_val.data(), sizeof(double) * S.dir_val.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_nb, S.nb.data(), sizeof(double) * S.nb.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_nb_node, S.nb_node.data(), sizeof(int) * S.nb_node.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_free_to_full, S.free_to_full.data(), sizeof(int) * S.free_to_full.size(),
                     cudaMemcpyHostToDevice, st));
  const int64_t nnz = (int64_t)S.tr_val.size();
  scatter_triplets<<<(int)std::min<int64_t>((nnz + 255) / 256, 4096), 256, 0, st>>>(d.s_mat, n, d.s_tr_row,
                                                                                    d.s_tr_col, d.s_tr_val, nnz);
  ++c->launches;
  CK(cudaGetLastError());
  for (int j0 = 0; j0 < n; j0 += kNB) {
    const int jb = std::min(kNB, n - j0);
    lu_panel<<<1, 1024, 0, st>>>(d.s_mat, n, j0, jb, d.s_piv, d.s_status);
    ++c->launches;
    lu_swap<<<(n + 255) / 256, 256, 0, st>>>(d.s_mat, n, j0, jb, d.s_piv);
    ++c->launches;
    const int rest = n - j0 - jb;
    if (rest > 0) {
      double* A11 = d.s_mat + (int64_t)j0 * n + j0;
      trsm_unit_lower<<<(rest + 127) / 128, 128, 0, st>>>(A11, n, A11 + jb, n, jb, rest);
      ++c->launches;
      dim3 grid((rest + 63) / 64, (rest + 63) / 64);
      gemm_sub<<<grid, 256, 0, st>>>(A11 + (int64_t)jb * n, n, A11 + jb, n, A11 + (int64_t)jb * n + jb, n, rest,
                                      rest, jb);
      ++c->launches;
    }
    CK(cudaGetLastError());
  }
  // solve: P L U X = B
  apply_pivots<<<(Cs + 63) / 64, 64, 0, st>>>(d.s_rhs, Cs, n, Cs, d.s_piv);
  ++c->launches;
  for (int j0 = 0; j0 < n; j0 += kNB) {
    const int jb = std::min(kNB, n - j0);
    double* A11 = d.s_mat + (int64_t)j0 * n + j0;
    double* B1 = d.s_rhs + (int64_t)j0 * Cs;
    trsm_unit_lower<<<(Cs + 63) / 64, 64, 0, st>>>(A11, n, B1, Cs, jb, Cs);
    ++c->launches;
    const int rest = n - j0 - jb;
    if (rest > 0) {
      dim3 grid((Cs + 63) / 64, (rest + 63) / 64);
      gemm_sub<<<grid, 256, 0, st>>>(A11 + (int64_t)jb * n, n, B1, Cs, B1 + (int64_t)jb * Cs, Cs, rest, Cs, jb);
      ++c->launches;
    }
  }
  for (int j0 = ((n - 1) / kNB) * kNB; j0 >= 0; j0 -= kNB) {
    const int jb = std::min(kNB, n - j0);
    double* A11 = d.s_mat + (int64_t)j0 * n + j0;
    double* B1 = d.s_rhs + (int64_t)j0 * Cs;
    trsm_upper<<<(Cs + 63) / 64, 64, 0, st>>>(A11, n, B1, Cs, jb, Cs);
    ++c->launches;
    if (j0 > 0) {
      dim3 grid((Cs + 63) / 64, (j0 + 63) / 64);
      gemm_sub<<<grid, 256, 0, st>>>(d.s_mat + j0, n, B1, Cs, d.s_rhs, Cs, j0, Cs, jb);
      ++c->launches;
    }
  }
  CK(cudaGetLastError());
  expand_solution<<<256, 256, 0, st>>>(d.s_rhs, Cs, n, d.s_free_to_full, S.n_u, d.s_dir, d.s_U, d.s_P, S.n_p);
  ++c->launches;
  expand_free<<<256, 256, 0, st>>>(d.s_rhs, Cs, n, d.s_free_to_full, S.n_u, d.s_U, d.s_P);
  ++c->launches;
  stokes_flux<<<64, 256, 0, st>>>(d.s_nb, d.s_nb_node, (int)S.nb_node.size(), Rs, d.s_U, S.n_nodes, d.s_phi,
                                 d.s_phi32);
  ++c->launches;
  CK(cudaGetLastError());
#undef CK
  return cudaSuccess;
}

}  // namespace sfb
