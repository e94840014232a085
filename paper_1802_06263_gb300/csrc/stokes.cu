// Deterministic Stokes subdomain basis on the GPU (Section 5.4: N_real = 1
// for Stokes subdomains). The Taylor-Hood saddle-point system assembled on
// the host (stokes_host.cpp), with its unknowns in band order, is scattered
// into band storage, factored by a blocked right-looking band LU with partial
// pivoting, and solved for the R_s + 1 right-hand sides (one normal-stress
// load per mortar DOF, Eqs. 5.1-5.2, and the inflow-driven particular
// problem, Eqs. 5.3-5.4). The flux basis is Phi_s[l][j] = -<u(xi_j).n, xi_l>,
// g_s[l] = <u_bar.n, xi_l>.
//
// Band storage: row i holds columns i - kl .. i + kl + ku (the kl + ku upper
// diagonals leave room for the fill of row interchanges) at
// a[i * ld + j + kl], ld = 2 kl + ku: a row-major array of leading dimension
// ld whose rows shift by one column each. Pivots of column k are sought in
// rows k .. k + kl, the only ones where column k has entries; the row
// interchanges are recorded and applied to the right-hand sides column by
// column in the forward solve (L is kept as its columns were when formed).
#include <algorithm>

#include "sfb_ctx.h"

namespace sfb {

namespace {

struct Band {
  double* a;
  int n, kl, ku;
  int64_t ld;
  __device__ __forceinline__ double& at(int i, int j) const { return a[(int64_t)i * ld + j + kl]; }
  __device__ __forceinline__ bool in(int i, int j) const { return j >= i - kl && j <= i + kl + ku; }
};

__global__ void band_scatter(Band B, const int* r, const int* c, const double* v, int64_t nnz) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
    B.at(r[t], c[t]) = v[t];
}

// Block-wide argmax of |value| (smallest index on ties); every thread gets it.
__device__ __forceinline__ int block_argmax(double best, int bi, double* sv, int* si, int* out, double* outv) {
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
    bi = threadIdx.x < nw ? si[threadIdx.x] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (threadIdx.x == 0) { *out = bi; *outv = best; }
  }
  __syncthreads();
  return *out;
}

// Panel k0 .. k0 + jb - 1 (one CTA): per column the pivot among rows
// k .. k + kl, the interchange inside the panel's columns, the multipliers
// and the rank-1 update of the panel's remaining columns. The band keeps each
// multiplier column as it was formed (later interchanges do not move it), the
// order the forward solve applies them in; the trailing update needs them in
// the final row order, so the panel also keeps a dense copy PL [(jb + kl) x
// kPlW] (row r - k0, column k - k0) whose rows follow every interchange.
constexpr int kPlW = 32;
__global__ void __launch_bounds__(1024) band_panel(Band B, int k0, int jb, int* piv, double* PL, int* status) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int prow;
  __shared__ double pval;
  const int cend = k0 + jb - 1;
  const int ph = jb + B.kl;   // rows of PL
  for (int e = threadIdx.x; e < ph * kPlW; e += blockDim.x) PL[e] = 0.0;
  __syncthreads();
  for (int k = k0; k <= cend; ++k) {
    const int kk = k - k0;
    const int rend = min(B.n - 1, k + B.kl);
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i <= rend; i += blockDim.x) {
      const double a = fabs(B.at(i, k));
      if (a > best) { best = a; bi = i; }
    }
    const int p = block_argmax(best, bi, sv, si, &prow, &pval);
    if (threadIdx.x == 0) {
      piv[k] = p;
      if (!(pval > 0.0)) atomicOr(status, 2);
    }
    if (p != k) {
      for (int j = k + threadIdx.x; j <= cend; j += blockDim.x) {
        const double t = B.at(k, j);
        B.at(k, j) = B.at(p, j);
        B.at(p, j) = t;
      }
      for (int q = threadIdx.x; q < kk; q += blockDim.x) {   // the copy's earlier columns follow
        const double t = PL[kk * kPlW + q];
        PL[kk * kPlW + q] = PL[(p - k0) * kPlW + q];
        PL[(p - k0) * kPlW + q] = t;
      }
    }
    __syncthreads();
    const double d = B.at(k, k);
    const double inv = d != 0.0 ? 1.0 / d : 0.0;
    for (int i = k + 1 + threadIdx.x; i <= rend; i += blockDim.x) {
      const double l = B.at(i, k) * inv;
      B.at(i, k) = l;
      PL[(i - k0) * kPlW + kk] = l;
    }
    __syncthreads();
    const int m = rend - k, nc = cend - k;
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
      const int i = k + 1 + e / nc, j = k + 1 + e % nc;
      B.at(i, j) -= B.at(i, k) * B.at(k, j);
    }
    __syncthreads();
  }
}

// The panel's interchanges on the trailing columns k0 + jb .. jend (one thread
// per column); a row's entries beyond column k + kl + ku are zero by the band
// invariant, so the interchange there has nothing to move.
__global__ void band_swap(Band B, int k0, int jb, int jend, const int* piv) {
  const int j = k0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (j > jend) return;
  for (int k = k0; k < k0 + jb; ++k) {
    const int p = piv[k];
    if (p != k && j <= k + B.kl + B.ku) {
      const double t = B.at(k, j);
      B.at(k, j) = B.at(p, j);
      B.at(p, j) = t;
    }
  }
}

// U12 = L11^{-1} A12 for the trailing columns (one thread per column), L11
// unit lower triangular from the panel's final-order copy PL; entries of A12
// outside the band are zero.
__global__ void band_trsm(Band B, int k0, int jb, int jend, const double* PL) {
  const int j = k0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (j > jend) return;
  for (int r = k0; r < k0 + jb; ++r) {
    if (!B.in(r, j)) continue;
    double v = B.at(r, j);
    for (int q = k0; q < r; ++q)
      if (B.in(q, j)) v -= PL[(r - k0) * kPlW + (q - k0)] * B.at(q, j);
    B.at(r, j) = v;
  }
}

// A22 -= L21 U12 over rows k0 + jb .. iend and columns k0 + jb .. jend, the
// panel's jb <= 32 columns as the inner dimension, L21 from the final-order
// copy PL; U12 entries outside the band are read as zero. 64 x 64 output tile
// per CTA, 4 x 4 per thread.
__global__ void __launch_bounds__(256) band_gemm(Band B, int k0, int jb, int iend, int jend, const double* PL) {
  __shared__ double Ls[64][33];
  __shared__ double Us[32][65];
  const int r0 = k0 + jb + blockIdx.y * 64, c0 = k0 + jb + blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    const int r = e / 32, q = e % 32;
    const int i = r0 + r, kq = k0 + q;
    Ls[r][q] = (i <= iend && q < jb) ? PL[(i - k0) * kPlW + q] : 0.0;
  }
  for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
    const int q = e / 64, c = e % 64;
    const int kq = k0 + q, j = c0 + c;
    Us[q][c] = (q < jb && j <= jend && B.in(kq, j)) ? B.at(kq, j) : 0.0;
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  double acc[4][4] = {};
  for (int q = 0; q < 32; ++q) {
    double l[4], u[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) l[a] = Ls[tr * 4 + a][q];
#pragma unroll
    for (int b = 0; b < 4; ++b) u[b] = Us[q][tc + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = r0 + tr * 4 + a, j = c0 + tc + 16 * b;
      if (i <= iend && j <= jend) B.at(i, j) -= acc[a][b];
    }
}

// Forward solve P L y = b for right-hand-side columns c0 .. c0 + 3 of X
// ([n][Cs] row-major): per column k of L, the recorded interchange, then
// rows k + 1 .. k + kl less L[r][k] y_k.
constexpr int kSolveCols = 4;
__global__ void __launch_bounds__(256) band_fwd(Band B, const int* piv, double* X, int Cs) {
  const int c0 = blockIdx.x * kSolveCols;
  for (int k = 0; k < B.n; ++k) {
    const int p = piv[k];
    if (p != k && threadIdx.x < kSolveCols && c0 + threadIdx.x < Cs) {
      const double t = X[(int64_t)k * Cs + c0 + threadIdx.x];
      X[(int64_t)k * Cs + c0 + threadIdx.x] = X[(int64_t)p * Cs + c0 + threadIdx.x];
      X[(int64_t)p * Cs + c0 + threadIdx.x] = t;
    }
    __syncthreads();
    const int rend = min(B.n - 1, k + B.kl);
    const int m = rend - k;
    for (int e = threadIdx.x; e < m * kSolveCols; e += blockDim.x) {
      const int r = k + 1 + e / kSolveCols, c = c0 + e % kSolveCols;
      if (c < Cs) X[(int64_t)r * Cs + c] -= B.at(r, k) * X[(int64_t)k * Cs + c];
    }
    __syncthreads();
  }
}

// Backward solve U x = y: x_k = y_k / U[k][k], then rows k - kl - ku .. k - 1
// less U[r][k] x_k.
__global__ void __launch_bounds__(256) band_bwd(Band B, double* X, int Cs, int* status) {
  const int c0 = blockIdx.x * kSolveCols;
  for (int k = B.n - 1; k >= 0; --k) {
    if (threadIdx.x < kSolveCols && c0 + threadIdx.x < Cs) {
      const double d = B.at(k, k);
      if (d == 0.0) atomicOr(status, 2);
      X[(int64_t)k * Cs + c0 + threadIdx.x] /= (d != 0.0 ? d : 1.0);
    }
    __syncthreads();
    const int rbeg = max(0, k - B.kl - B.ku);
    const int m = k - rbeg;
    for (int e = threadIdx.x; e < m * kSolveCols; e += blockDim.x) {
      const int r = rbeg + e / kSolveCols, c = c0 + e % kSolveCols;
      if (c < Cs) X[(int64_t)r * Cs + c] -= B.at(r, k) * X[(int64_t)k * Cs + c];
    }
    __syncthreads();
  }
}

// R = B - A X for every right-hand side (one thread per row and column; the
// row's entries in ascending column order), the residual of one FP64
// refinement pass of the band LU solution.
__global__ void stokes_residual(int n, int Cs, const int* row_ptr, const int* col, const double* val,
                                const double* B, const double* X, double* R) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * Cs;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Cs), c = (int)(e % Cs);
    double acc = B[e];
    for (int t = row_ptr[r]; t < row_ptr[r + 1]; ++t) acc = fma(-val[t], X[(int64_t)col[t] * Cs + c], acc);
    R[e] = acc;
  }
}

__global__ void add_correction(int64_t n, double* X, const double* D) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    X[e] += D[e];
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
  Band B;
  B.a = d.s_mat;
  B.n = n;
  B.kl = S.kl;
  B.ku = S.ku;
  B.ld = 2 * (int64_t)S.kl + S.ku;
  cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  CK(cudaMemsetAsync(d.s_mat, 0, sizeof(double) * ((size_t)n * (B.ld + 1) + 8), st));
  CK(cudaMemsetAsync(d.s_status, 0, sizeof(int) * 4, st));
  CK(cudaMemcpyAsync(d.s_tr_row, S.tr_row.data(), sizeof(int) * S.tr_row.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_tr_col, S.tr_col.data(), sizeof(int) * S.tr_col.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_tr_val, S.tr_val.data(), sizeof(double) * S.tr_val.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_rhs, S.rhs.data(), sizeof(double) * S.rhs.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_b, S.rhs.data(), sizeof(double) * S.rhs.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_row_ptr, S.row_ptr.data(), sizeof(int) * S.row_ptr.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_dir, S.dir_val.data(), sizeof(double) * S.dir_val.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_nb, S.nb.data(), sizeof(double) * S.nb.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_nb_node, S.nb_node.data(), sizeof(int) * S.nb_node.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.s_free_to_full, S.free_to_full.data(), sizeof(int) * S.free_to_full.size(),
                     cudaMemcpyHostToDevice, st));
  const int64_t nnz = (int64_t)S.tr_val.size();
  band_scatter<<<(int)std::min<int64_t>((nnz + 255) / 256, 4096), 256, 0, st>>>(B, d.s_tr_row, d.s_tr_col,
                                                                                d.s_tr_val, nnz);
  ++c->launches;
  CK(cudaGetLastError());
  // panels no wider than the band, so a panel row's columns stay inside it
  const int nb = std::max(1, std::min(kPlW, S.kl + S.ku + 1));
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int jb = std::min(nb, n - k0);
    band_panel<<<1, 1024, 0, st>>>(B, k0, jb, d.s_piv, d.s_pl, d.s_status);
    ++c->launches;
    const int jend = std::min(n - 1, k0 + jb - 1 + S.kl + S.ku);
    const int iend = std::min(n - 1, k0 + jb - 1 + S.kl);
    const int ncol = jend - (k0 + jb) + 1, nrow = iend - (k0 + jb) + 1;
    if (ncol > 0) {
      band_swap<<<(ncol + 127) / 128, 128, 0, st>>>(B, k0, jb, jend, d.s_piv);
      band_trsm<<<(ncol + 127) / 128, 128, 0, st>>>(B, k0, jb, jend, d.s_pl);
      c->launches += 2;
      if (nrow > 0) {
        band_gemm<<<dim3((ncol + 63) / 64, (nrow + 63) / 64), 256, 0, st>>>(B, k0, jb, iend, jend, d.s_pl);
        ++c->launches;
      }
    }
    CK(cudaGetLastError());
  }
  // solve P L U X = B, right-hand-side columns in groups of kSolveCols per CTA
  const int ng = (Cs + kSolveCols - 1) / kSolveCols;
  band_fwd<<<ng, 256, 0, st>>>(B, d.s_piv, d.s_rhs, Cs);
  band_bwd<<<ng, 256, 0, st>>>(B, d.s_rhs, Cs, d.s_status);
  c->launches += 2;
  CK(cudaGetLastError());
  // one pass of FP64 iterative refinement: R = B - A X from the assembled
  // rows, the correction by the same factors (the saddle-point system's
  // pivoted band LU leaves errors of about cond * 1e-16; the pass takes them
  // to round-off)
  const int64_t nel = (int64_t)n * Cs;
  const int rg = (int)std::min<int64_t>((nel + 255) / 256, 8192);
  stokes_residual<<<rg, 256, 0, st>>>(n, Cs, d.s_row_ptr, d.s_tr_col, d.s_tr_val, d.s_b, d.s_rhs, d.s_res);
  band_fwd<<<ng, 256, 0, st>>>(B, d.s_piv, d.s_res, Cs);
  band_bwd<<<ng, 256, 0, st>>>(B, d.s_res, Cs, d.s_status);
  add_correction<<<rg, 256, 0, st>>>(nel, d.s_rhs, d.s_res);
  c->launches += 4;
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
