// Stochastic multiscale flux basis: one CTA per (Darcy subdomain, local
// realization) item (Section 5.4, pre-computation loop, Steps 1-2).
//
// Per item the kernel
//  1. evaluates the truncated local KL expansion at the cell centres,
//     K = exp(E[Y] + sum_j sqrt(lambda_j) y_j f_j) (Eq. 2.13), and the face
//     transmissibilities of the cell-centred form of lowest-order RT with the
//     trapezoidal rule (harmonic means inside, half-cell values on Dirichlet
//     faces, zero on no-flow faces);
//  2. factors the diagonally scaled 5-point matrix
//     Ahat = diag(A)^{-1/2} A diag(A)^{-1/2}, block tridiagonal with nx x nx
//     tridiagonal diagonal blocks and diagonal couplings between grid rows,
//     by the block LDL^T recurrence S_b = Ahat_bb - D_{b-1} S_{b-1}^{-1} D_{b-1}.
//     Each S_b is inverted in registers by the symmetric sweep operator (one
//     barrier per pivot) and G_b = S_b^{-1} is stored;
//  3. solves A X = B for R + 1 right-hand sides at once: one column per mortar
//     DOF (Dirichlet data = face averages of xi_j, Eqs. 5.5-5.6) and one
//     particular column (source and outer data, Eqs. 5.7-5.8), by a forward
//     sweep z_b = G_b (s_b r_b + D_{b-1} z_{b-1}) and a backward sweep
//     d_b = z_b + G_b D_b d_{b+1}, x_b += s_b d_b;
//  4. in the mixed form (factor type float) refines X with FP64 residuals
//     r = B - A X of the 5-point stencil, stopping when the contraction of the
//     corrections predicts a relative error below tol (or on stagnation or the
//     step limit).
// The flux-basis epilogue projects the boundary fluxes of X back onto the
// mortar space (Section 5.2 step 3): Phi[l][j] = -<u(xi_j).n, xi_l>.
//
// Layouts: X is column-major per item ([R+1][n_cells]); a block row of the
// right-hand sides, in shared memory and in the Z store alike, is column-major
// [Cp][np] (Cp = R+1 rounded up to 4, np = nx padded to 16), so the row loops
// give a warp 32 consecutive cells of one column and the products G_b U read
// 16-byte pieces of G_b (symmetric) rows and of U columns.
#include <math.h>

#include <algorithm>

#include "basis_dev.cuh"

namespace sfb {

namespace {

// The same blocked sweep with the kP x kP pivot-block inverse done once, by
// warp 0 in shared memory, and W formed by the threads j < np: the FP64 form,
// where a redundant inverse in every warp would multiply the scarce FP64 work.
template <typename T, int MT, int NT, int kP>
__device__ __forceinline__ void blocked_sweep_w0(T (&areg)[MT][4][4], int np, int ntr, T* VT, T* W, T* Ablk,
                                                 int* bad) {
  for (int k0 = 0; k0 < np; k0 += kP) {
    // (a) panel columns: VT[p][i] = A[i][k0 + p]
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int t = threadIdx.x + m * NT;
      if (t >= ntr * ntr) break;
      const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
      if (j0 >= k0 && j0 < k0 + kP)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) VT[(j0 + q - k0) * np + i0 + a] = areg[m][a][q];
    }
    __syncthreads();
    // (b) warp 0: sweep of the kP x kP block A_KK (Ablk = -A_KK^{-1})
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int e = lane; e < kP * kP; e += 32) {
        const int p = e / kP, q = e % kP;
        Ablk[e] = VT[q * np + k0 + p];
      }
      __syncwarp();
      for (int kk = 0; kk < kP; ++kk) {
        T piv = Ablk[kk * kP + kk];
        if (!(piv > T(0))) {
          if (lane == 0) *bad = 1;
          piv = T(1);
        }
        const T inv = rcp_rn(piv);
        T nv[(kP * kP + 31) / 32];
#pragma unroll
        for (int r = 0; r < (kP * kP + 31) / 32; ++r) {
          const int e = lane + 32 * r;
          const int p = e / kP, q = e % kP;
          const T own = Ablk[e], rowk = Ablk[kk * kP + q], colk = Ablk[p * kP + kk];
          T v;
          if (p == kk && q == kk) v = -inv;
          else if (p == kk) v = rowk * inv;
          else if (q == kk) v = colk * inv;
          else v = fma(-colk, rowk * inv, own);
          nv[r] = v;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < (kP * kP + 31) / 32; ++r) Ablk[lane + 32 * r] = nv[r];
        __syncwarp();
      }
    }
    __syncthreads();
    // (c) W[p][j] = sum_q A_KK^{-1}[p][q] VT[q][j]
    for (int j = threadIdx.x; j < np; j += NT) {
      T col[kP];
#pragma unroll
      for (int q = 0; q < kP; ++q) col[q] = VT[q * np + j];
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        T w = T(0);
#pragma unroll
        for (int q = 0; q < kP; ++q) w = fma(-Ablk[p * kP + q], col[q], w);
        W[p * np + j] = w;
      }
    }
    __syncthreads();
    // (d) update the register tiles
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int t = threadIdx.x + m * NT;
      if (t >= ntr * ntr) break;
      const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
      const bool rk = i0 >= k0 && i0 < k0 + kP, ck = j0 >= k0 && j0 < k0 + kP;
      if (!rk && !ck) {
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          T v4[4], w4[4];
          load4(VT + p * np + i0, v4);
          load4(W + p * np + j0, w4);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) areg[m][a][q] = fma(-v4[a], w4[q], areg[m][a][q]);
        }
      } else if (rk && !ck) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) areg[m][a][q] = W[(i0 + a - k0) * np + j0 + q];
      } else if (!rk && ck) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) areg[m][a][q] = W[(j0 + q - k0) * np + i0 + a];
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) areg[m][a][q] = Ablk[(i0 + a - k0) * kP + (j0 + q - k0)];
      }
    }
    __syncthreads();
  }
}

// MODE 0: one CTA per item does everything; MODE 1: one CTA per item does
// phases 1-2 only (KL, assembly, factor: G_b, S, D_{b-1}, T and diag(A) to
// global memory); MODE 2: one CTA per column chunk of an item runs phases 3-4
// for its columns on the stored factor, the first solve as a forward sweep on
// x = 0. Splitting an item's solves over several CTAs shortens the longest
// dependent chain per CTA and gives the scheduler several times more, smaller
// work units than there are items.
// The work of one CTA on item `item` (an index into a.item_sub / a.item_k)
// and, in MODE 2, on its columns c0 .. c0 + ccount - 1; statistics go to slot
// wid_in (the item's id when negative). The shared-memory state comes from
// the calling kernel.
template <typename T, int MT, int NT, int GB, int MODE>
__device__ __forceinline__ void basis_body(const BasisArgs& a, int refine, int item, int c0, int ccount, int wid_in,
                                           unsigned char* smem_raw, double* red, int& bad_spd, uint64_t* gbar,
                                           uint64_t& zbar) {
  const int s = a.item_sub[item], kk = a.item_k[item];
  const SubDev S = a.subs[s];
  const int id = (int)S.item0 + kk;
  // statistics slot: the item, or (MODE 2) the chunk after all items
  const int wid = wid_in >= 0 ? wid_in : id;
  const ItemOff off = a.off[id];
  Geo g;
  // all R + 1 right-hand sides, or (Method S1's set-up) only the particular
  // one, column R of the right-hand side and of X, or (MODE 2) the chunk's
  // columns; none in MODE 1
  const int coff = MODE == 2 ? c0 : (a.particular_only ? S.R : 0);
  g.nx = S.nx; g.ny = S.ny; g.R = S.R;
  g.src = S.source * S.hx * S.hy;
  g.C = MODE == 2 ? ccount : MODE == 1 ? 0 : (a.particular_only ? 1 : S.R + 1);
  g.Cp = (g.C + 3) & ~3;
  g.nc = S.nx * S.ny;
  const int nx = g.nx, ny = g.ny, nc = g.nc, C = g.C, Cp = g.Cp;
  constexpr int kP = panel_of<T>();
  const int np = (nx + kPanel - 1) & ~(kPanel - 1);  // identity-padded block size
  const int ntr = np >> 2;
  const uint32_t gbytes = (uint32_t)(np * np * sizeof(T));
  const uint32_t zbytes = (uint32_t)(np * Cp * sizeof(T));
  double* Tx = a.T + off.t;
  double* Ty = Tx + (int64_t)ny * (nx + 1);
  g.Tx = Tx; g.Ty = Ty;
  double* X = a.X + off.x + (int64_t)coff * S.nx * S.ny;
  double* Dg = a.D + off.diag;
  T* Sg = reinterpret_cast<T*>(a.S) + off.sc;
  T* DLg = reinterpret_cast<T*>(a.DL) + off.sc;  // [ny][nx] scaled couplings to the row below
  T* Gg = reinterpret_cast<T*>(a.G) + off.g;   // [ny][np][np]
  // [ny][np][Cp], the shared-memory image of a row block; a chunk's own block
  // starts after the earlier chunks' (their column counts are multiples of 4)
  T* Zg = reinterpret_cast<T*>(a.Z) + off.z + (MODE == 2 ? (int64_t)ny * np * c0 : 0);

  // smem: Gs[GB][np*np] | U region | Zs[Cp][np] | sc | dlo | dup | txh | rbs,
  // the U region holding Us[Cp][np] in the solves and VT[kP*np] | W[kP*np] |
  // Ablk[kP*kP] during the block inversions (never both at once); rbs (FP64,
  // [2][Cp]) the right-hand sides of a row's two end cells in the solves
  const int ureg = MODE == 2 ? np * Cp : max(np * Cp, 2 * kP * np + kP * kP);
  T* Gs0 = reinterpret_cast<T*>(smem_raw);
  T* Us = Gs0 + GB * np * np;
  T* VT = Us;
  T* W = VT + kP * np;
  T* Ablk = W + kP * np;
  T* Zs = Us + ureg;
  T* sc = Zs + np * Cp;
  T* dlo = sc + np;
  T* dup = dlo + np;
  T* txh = dup + np;
  double* rbs = reinterpret_cast<double*>(txh + np);
  uint32_t gph[2] = {0u, 0u}, zph = 0u;

  if (threadIdx.x == 0) {
    bad_spd = 0;
    mbar_init(&gbar[0], 1);
    mbar_init(&gbar[1], 1);
    mbar_init(&zbar, 1);
    fence_barrier_init();
  }
  int st = 0;
  long long* cyc = a.cycles + kCycSlots * (int64_t)wid;
  // thread 0's clocks, kept in shared memory so that they take no registers
  // of the other threads: [0, 12) the sub-phases of the factor, forward and
  // backward row steps (slots 4-15 of the per-item cycle record), then the
  // forward and backward totals, the phase mark and the sub-phase mark
  __shared__ long long clk[16];
  constexpr int kFwd = 12, kBwd = 13, kMark = 14, kSub = 15;
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    for (int q = 0; q < kMark; ++q) clk[q] = 0;
    clk[kMark] = t0;
    clk[kSub] = t0;
  }
#define SFB_MARK(k)                                          \
  do {                                                       \
    if (threadIdx.x == 0) {                                  \
      const long long t_ = clock64();                        \
      clk[k] += t_ - clk[kSub];                              \
      clk[kSub] = t_;                                        \
    }                                                        \
  } while (0)
  for (int e = threadIdx.x; e < np * Cp; e += blockDim.x) { Us[e] = T(0); Zs[e] = T(0); }
  for (int e = threadIdx.x; e < np; e += blockDim.x) { sc[e] = T(0); dlo[e] = T(0); dup[e] = T(0); txh[e] = T(0); }
  __syncthreads();

  // ---- 1. permeability, transmissibilities, diagonal and scaling ------------
  if constexpr (MODE != 2) {
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
    // the diagonal scaling s = D^{-1/2}: any positive scaling serves (the
    // factor, the solves and x += s d all read the same s), so the FP32 factor
    // takes it from the FP32 reciprocal square root and keeps its FP64 pipe for
    // the transmissibilities; the FP64 factor keeps it in FP64
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int b = c / nx, i = c - b * nx;
      const double d = Tx[b * (nx + 1) + i] + Tx[b * (nx + 1) + i + 1] + Ty[b * nx + i] + Ty[(b + 1) * nx + i];
      Dg[c] = d;
      if constexpr (sizeof(T) == 4) Sg[c] = rsqrtf(f64_to_f32_bits(d));
      else Sg[c] = T(1.0 / sqrt(d));
    }
    __syncthreads();
    // D_{b-1} of the scaled matrix: s_{b-1,i} Ty[b][i] s_{b,i} (zero for row 0)
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int b = c / nx, i = c - b * nx;
      if constexpr (sizeof(T) == 4)
        DLg[c] = b > 0 ? f64_to_f32_bits(Ty[b * nx + i]) * Sg[c] * Sg[c - nx] : T(0);
      else
        DLg[c] = b > 0 ? T(Ty[b * nx + i] / sqrt(Dg[c] * Dg[c - nx])) : T(0);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { const long long t = clock64(); cyc[0] = t - clk[kMark]; clk[kMark] = t; }

  // ---- 2. factorization, fused with the first forward solve ------------------
  // G_b and z_b leave through bulk stores from shared memory.
  T areg[MT][4][4];
  for (int b = 0; b < (MODE == 2 ? 0 : ny); ++b) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double si = (double)Sg[b * nx + i];
      sc[i] = T(si);
      txh[i] = i > 0 ? T(-Tx[b * (nx + 1) + i] * si * (double)Sg[b * nx + i - 1]) : T(0);
      dlo[i] = DLg[b * nx + i];
    }
    __syncthreads();
    SFB_MARK(0);
    form_block<T, MT, NT>(areg, b, nx, ntr, txh, dlo);
    if constexpr (sizeof(T) == 4) blocked_sweep<T, MT, NT, panel_of<T>()>(areg, np, ntr, VT, W, Ablk, &bad_spd);
    else blocked_sweep_w0<T, MT, NT, panel_of<T>()>(areg, np, ntr, VT, W, Ablk, &bad_spd);
    SFB_MARK(1);
    // G_b in shared memory (bulk-stored below), or straight to global memory
    // when the shape keeps no G buffer (GB == 0: the 128-wide FP64 blocks)
    T* Gs = GB == 0 ? Gg + (int64_t)b * np * np : Gs0 + (b % (GB == 0 ? 1 : GB)) * np * np;
    if (threadIdx.x == 0) bulk_wait_read();   // the store that last read Gs / Zs is done
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int t = threadIdx.x + m * NT;
      if (t >= ntr * ntr) break;
      const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
        for (int q = 0; q < 4; ++q) Gs[(i0 + a2) * np + j0 + q] = -areg[m][a2][q];
    }
    // first forward solve row: u_b = s_b B_b + dlo_b z_{b-1}
    if constexpr (MODE == 0)
      for (int e = threadIdx.x; e < np * C; e += blockDim.x) {
        const int c = e / np, i = e - c * np;
        if (i >= nx) continue;
        T u = sc[i] * from_f64<T>(rhs_entry(S, g, a.proj, b, i, c + coff));
        if (b > 0) u = fma(dlo[i], Zs[c * np + i], u);
        Us[c * np + i] = u;
      }
    fence_async_shared();
    __syncthreads();
    SFB_MARK(2);
    if (GB > 0 && threadIdx.x == 0) bulk_store(Gg + (int64_t)b * np * np, Gs, gbytes);
    if constexpr (MODE == 0) {
      gemm_g<T>(Gs, Us, Zs, false, np, C);
      fence_async_shared();
      __syncthreads();
      SFB_MARK(3);
      if (threadIdx.x == 0) bulk_store(Zg + (int64_t)b * np * Cp, Zs, zbytes);
    }
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    fence_async_global();
  }
  __syncthreads();
  if (threadIdx.x == 0) { const long long t = clock64(); cyc[1] = t - clk[kMark]; clk[kMark] = t; clk[kSub] = t; }
  if constexpr (MODE == 1) {
    // the factor alone: its status, and the sub-phase clocks of its rows
    if (threadIdx.x == 0) {
      cyc[2] = 0;
      cyc[3] = 0;
      for (int q = 0; q < 12; ++q) cyc[4 + q] = clk[q];
    }
    if (bad_spd) st |= ST_NOT_SPD;
    if (st) atomicOr(&a.status[id], st);
    return;
  }

  // ---- 3./4. backward sweep, then refine with FP64 residuals --------------------------
  // Row loops over the nx x C entries of a block row: the 32 lanes of a warp
  // take 32 consecutive cells of one column (a 256-byte run of an X column,
  // consecutive words of the column-major shared-memory blocks) and the warps
  // the (cell segment, column) tasks in turn, task k = (k mod nseg, k / nseg).
  // When the segments divide the warps (nx <= 32, or 64 with an even number
  // of warps, ...) a lane keeps one cell for the whole row and loads the
  // cell's coefficients once.
  const int lane = (int)(threadIdx.x & 31);
  const int nseg = (nx + 31) >> 5, nwarp = (int)(blockDim.x >> 5), wrp = (int)(threadIdx.x >> 5);
  const int seg0 = wrp % nseg, col0 = wrp / nseg;       // the warp's first task
  const int dseg = nwarp % nseg, dcol = nwarp / nseg;   // the step between its tasks
  // the two end cells of a row (rows 1 .. ny-2): their right-hand sides come
  // from rbs, prefetched a row ahead as the operands of T_face * value
  const int rbt = (int)threadIdx.x;
  const int rb_side = rbt < 2 * C ? rbt / C : 0, rb_col = rbt < 2 * C ? rbt - rb_side * C : 0;
  auto edge_operands = [&](int bb, double& t, double& v) {
    const int sd = rb_side ? 1 : 3, cg = rb_col + coff;
    t = Tx[bb * (nx + 1) + (rb_side ? nx : 0)];
    v = 0.0;
    if (cg < S.R) {
      if (S.side_type[sd] == SIDE_IFACE) v = a.proj[S.proj_off[sd] + (int64_t)bb * S.R + cg];
    } else if (S.side_type[sd] == SIDE_DIRICHLET) {
      v = S.side_val[sd];
    }
  };
  // the bulk copies of the solves are issued (and their groups waited on) by
  // lane 0 of the last warp, which holds no product tile and no row set-up
  // work in the chunk shapes, so that the copies start while the other
  // threads set up the next row
  const unsigned tma = blockDim.x - 32;
  double xref2 = 0.0, prev_corr = 0.0, est = 1.0, bnorm2 = 0.0;
  int n_done = 0;
  bool timeout = false, nonfinite = false;
  for (int it = 0; it <= refine && !timeout; ++it) {
    float rr = 0.f;
    // x = 0 before a chunk's first forward sweep (MODE 2): r = B
    const bool xzero = MODE == 2 && it == 0;
    if (it > 0 || MODE == 2) {
      // forward sweep: r_b = B_b - (A x)_b in FP64; u_b = s_b r_b + dlo_b z_{b-1}
      if (GB > 0 && threadIdx.x == tma) { fence_async_shared(); bulk_load(Gs0, Gg, gbytes, &gbar[0]); }
      // row scalings of the next row travel in registers while a row runs
      T nsc = threadIdx.x < nx ? Sg[threadIdx.x] : T(0), ndl = threadIdx.x < nx ? DLg[threadIdx.x] : T(0);
      if (!xzero) {
        prefetch_x_row(X, nc, nx, 0, C);
        if (ny > 1) prefetch_x_row(X, nc, nx, 1, C);
      }
      const bool rb_thread = rbt < 2 * C && nx > 1;
      double rb_t = 0.0, rb_v = 0.0;
      if (rb_thread && ny > 2) edge_operands(1, rb_t, rb_v);
      for (int b = 0; b < ny; ++b) {
        const int cur = GB == 2 ? (b & 1) : 0;
        T* Gs = GB == 0 ? Gg + (int64_t)b * np * np : Gs0 + cur * np * np;
        if (threadIdx.x < nx) {
          sc[threadIdx.x] = nsc;
          dlo[threadIdx.x] = ndl;
          if (b + 1 < ny) { nsc = Sg[(b + 1) * nx + threadIdx.x]; ndl = DLg[(b + 1) * nx + threadIdx.x]; }
        }
        if (b + 2 < ny && !xzero) prefetch_x_row(X, nc, nx, b + 2, C);   // the residual of row b + 1 reads it
        if (rb_thread && b >= 1 && b <= ny - 2) {
          // an end cell's right-hand side: T_face * value (+ the source in column R)
          rbs[rb_side * Cp + rb_col] = rb_col + coff < S.R ? rb_t * rb_v : fma(rb_t, rb_v, g.src);
          if (b + 1 <= ny - 2) edge_operands(b + 1, rb_t, rb_v);
        }
        __syncthreads();
        SFB_MARK(4);
        if (GB == 2 && threadIdx.x == tma && b + 1 < ny) {
          fence_async_shared();
          bulk_load(Gs0 + (cur ^ 1) * np * np, Gg + (int64_t)(b + 1) * np * np, gbytes, &gbar[cur ^ 1]);
        }
        {
          // rows 1 .. ny-2 (and nx > 1): every cell's five stencil FMAs without
          // a branch, the end cells' right-hand sides from rbs and their
          // missing neighbour's coefficient zero (its load then reads the end
          // cell of an adjacent row, in bounds, times zero); rows 0 and ny-1
          // take the general right-hand side and guarded neighbours
          const bool edge_row = b == 0 || b == ny - 1 || nx == 1;
          const double* Tb = Tx + b * (nx + 1);
          const double* xb = X + (int64_t)b * nx;
          auto coeffs = [&](int i, double& dd, double& tw, double& te, double& ts, double& tn) {
            dd = Dg[(int64_t)b * nx + i];
            tw = i > 0 ? Tb[i] : 0.0;
            te = i < nx - 1 ? Tb[i + 1] : 0.0;
            ts = b > 0 ? Ty[b * nx + i] : 0.0;
            tn = b < ny - 1 ? Ty[(b + 1) * nx + i] : 0.0;
          };
          auto entry = [&](int i, int c, double dd, double tw, double te, double ts, double tn, T sci, T dli) {
            const double* xp = xb + (int64_t)c * nc + i;
            double r;
            // r = B - A x as five FP64 FMAs: B - D x, then + T x over the neighbours
            if (!edge_row) {
              r = (i == 0 || i == nx - 1) ? rbs[(i == 0 ? 0 : Cp) + c] : (c + coff < g.R ? 0.0 : g.src);
              if (!xzero) {
                r = fma(-dd, xp[0], r);
                r = fma(tw, xp[-1], r);
                r = fma(te, xp[1], r);
                r = fma(ts, xp[-nx], r);
                r = fma(tn, xp[nx], r);
              }
            } else {
              r = rhs_boundary(S, g, a.proj, b, i, c + coff);
              if (!xzero) {
                r = fma(-dd, xp[0], r);
                if (i > 0) r = fma(tw, xp[-1], r);
                if (i < nx - 1) r = fma(te, xp[1], r);
                if (b > 0) r = fma(ts, xp[-nx], r);
                if (b < ny - 1) r = fma(tn, xp[nx], r);
              }
            }
            const T rt = from_f64<T>(r);
            const float rf = to_f32(rt);
            rr = fmaf(rf, rf, rr);
            T u = sci * rt;
            if (b > 0) u = fma(dli, Zs[c * np + i], u);
            Us[c * np + i] = u;
          };
          double dd = 0.0, tw = 0.0, te = 0.0, ts = 0.0, tn = 0.0;
          if (dseg == 0) {
            const int i = seg0 * 32 + lane;
            if (i < nx) {
              if (!xzero) coeffs(i, dd, tw, te, ts, tn);
              const T sci = sc[i], dli = dlo[i];
              if (edge_row) {
                for (int c = col0; c < C; c += dcol) entry(i, c, dd, tw, te, ts, tn, sci, dli);
              } else {
                // the uniform conditions hoisted: an end cell reads its right-hand
                // side from rbs, the others the column's constant (every lane
                // loads from rbs, in bounds, and selects)
                const bool end_cell = i == 0 || i == nx - 1;
                const double* rbp = rbs + (i == nx - 1 ? Cp : 0);
                const double* xp = xb + (int64_t)col0 * nc + i;
                const int64_t xs = (int64_t)dcol * nc;
                int zo = col0 * np + i;
                const int zs = dcol * np;
                if (xzero) {
                  for (int c = col0; c < C; c += dcol, zo += zs) {
                    const double rbv = rbp[c];
                    const double r = end_cell ? rbv : (c + coff < g.R ? 0.0 : g.src);
                    const T rt = from_f64<T>(r);
                    const float rf = to_f32(rt);
                    rr = fmaf(rf, rf, rr);
                    Us[zo] = fma(dli, Zs[zo], sci * rt);
                  }
                } else {
#pragma unroll 2
                  for (int c = col0; c < C; c += dcol, xp += xs, zo += zs) {
                    const double rbv = rbp[c];
                    double r = end_cell ? rbv : (c + coff < g.R ? 0.0 : g.src);
                    // r = B - A x as five FP64 FMAs: B - D x, then + T x over the neighbours
                    r = fma(-dd, xp[0], r);
                    r = fma(tw, xp[-1], r);
                    r = fma(te, xp[1], r);
                    r = fma(ts, xp[-nx], r);
                    r = fma(tn, xp[nx], r);
                    const T rt = from_f64<T>(r);
                    const float rf = to_f32(rt);
                    rr = fmaf(rf, rf, rr);
                    Us[zo] = fma(dli, Zs[zo], sci * rt);
                  }
                }
              }
            }
          } else {
            int sg = seg0, c = col0, scur = -1, i = 0;
            T sci = T(0), dli = T(0);
            while (c < C) {
              if (sg != scur) {
                scur = sg;
                i = sg * 32 + lane;
                if (i < nx) {
                  if (!xzero) coeffs(i, dd, tw, te, ts, tn);
                  sci = sc[i];
                  dli = dlo[i];
                }
              }
              if (i < nx) entry(i, c, dd, tw, te, ts, tn, sci, dli);
              sg += dseg;
              c += dcol;
              if (sg >= nseg) { sg -= nseg; ++c; }
            }
          }
        }
        SFB_MARK(8);
        // G_b present, and the store that reads Zs finished
        if (threadIdx.x == tma) bulk_wait_read();
        bool ok = true;
        if (GB > 0) {
          ok = mbar_wait(&gbar[cur], gph[cur]);
          gph[cur] ^= 1u;
        }
        if (__syncthreads_or(!ok)) { timeout = true; break; }
        SFB_MARK(5);
        gemm_g<T>(Gs, Us, Zs, false, np, C);
        fence_async_shared();
        __syncthreads();
        SFB_MARK(6);
        if (threadIdx.x == tma) {
          bulk_store(Zg + (int64_t)b * np * Cp, Zs, zbytes);
          if (GB == 1 && b + 1 < ny) { fence_async_shared(); bulk_load(Gs0, Gg + (int64_t)(b + 1) * np * np, gbytes, &gbar[0]); }
        }
      }
      if (threadIdx.x == tma) {
        bulk_wait_all();
        fence_async_global();
      }
      __syncthreads();
      if (timeout) break;
      const double rnorm2 = block_sum((double)rr, red);
      if (xzero) bnorm2 = rnorm2;   // |B|^2 for the relative residual
      else if (threadIdx.x == 0) a.resid[wid] = sqrt(rnorm2 / fmax(bnorm2, 1e-300));
      if (threadIdx.x == 0) { const long long t = clock64(); clk[kFwd] += t - clk[kMark]; clk[kMark] = t; clk[kSub] = t; }
    } else {
      // |B|^2 for the relative residual
      float bb = 0.f;
      for (int e = threadIdx.x; e < nc * C; e += blockDim.x) {
        const int c = e / nc, cell = e - c * nc;
        const float v = f64_to_f32_bits(rhs_entry(S, g, a.proj, cell / nx, cell % nx, c + coff));
        bb = fmaf(v, v, bb);
      }
      bnorm2 = block_sum((double)bb, red);
    }
    // backward sweep: d_b = z_b + G_b (dup_b .* d_{b+1}); x_b += s_b d_b, with
    // dup_b .* d_{b+1} formed by the update loop of row b + 1 (dup holding the
    // coupling of that row to the one below). G_{b-1} is prefetched while row b
    // runs (two G buffers).
    float dn2f = 0.f;
    if (GB == 2 && threadIdx.x == tma && ny >= 2) {
      fence_async_shared();
      bulk_load(Gs0, Gg + (int64_t)(ny - 2) * np * np, gbytes, &gbar[0]);
    }
    T bsc = threadIdx.x < nx ? Sg[(ny - 1) * nx + threadIdx.x] : T(0);
    T bdl = threadIdx.x < nx ? DLg[(ny - 1) * nx + threadIdx.x] : T(0);
    for (int b = ny - 1; b >= 0; --b) {
      const int cur = GB == 2 ? ((ny - 2 - b) & 1) : 0;   // buffer of G_b (b <= ny-2)
      T* Gs = GB == 0 ? Gg + (int64_t)b * np * np : Gs0 + cur * np * np;
      // the previous row's loop finished with Zs and sc / dup (trailing barrier)
      if (threadIdx.x < nx) {
        sc[threadIdx.x] = bsc;
        dup[threadIdx.x] = bdl;   // coupling of row b to row b - 1 (zero for row 0)
        if (b > 0) { bsc = Sg[(b - 1) * nx + threadIdx.x]; bdl = DLg[(b - 1) * nx + threadIdx.x]; }
      }
      if (it > 0) prefetch_x_row(X, nc, nx, b, C);   // updated after the product below
      SFB_MARK(7);
      if (threadIdx.x == tma) {
        fence_async_shared();
        if (b < ny - 1) {
          if (GB == 2 && b >= 1)   // prefetch G_{b-1}
            bulk_load(Gs0 + (cur ^ 1) * np * np, Gg + (int64_t)(b - 1) * np * np, gbytes, &gbar[cur ^ 1]);
          if (GB == 1)             // G_b into the single buffer
            bulk_load(Gs0, Gg + (int64_t)b * np * np, gbytes, &gbar[0]);
        }
        bulk_load(Zs, Zg + (int64_t)b * np * Cp, zbytes, &zbar);
      }
      bool ok = mbar_wait(&zbar, zph);
      zph ^= 1u;
      if (GB > 0 && b < ny - 1) {
        ok = mbar_wait(&gbar[cur], gph[cur]) && ok;
        gph[cur] ^= 1u;
      }
      if (__syncthreads_or(!ok)) { timeout = true; break; }
      SFB_MARK(9);
      if (b < ny - 1) gemm_g<T>(Gs, Us, Zs, true, np, C);
      __syncthreads();
      SFB_MARK(10);
      // x_b += s d_b and Us = dup .* d_b for row b - 1; with a fixed cell per
      // lane the X entries of four columns are loaded before any of them is
      // stored, so that the loads overlap
      {
        double* xb = X + (int64_t)b * nx;
        auto upd = [&](int i, int c, T sci, T dpi, double xo) {
          const T z = Zs[c * np + i];
          const T dt = sci * z;
          const float df = to_f32(dt);
          dn2f = fmaf(df, df, dn2f);
          const double xn = it == 0 ? to_f64(dt) : xo + to_f64(dt);
          nonfinite |= ((__double2hiint(xn) >> 20) & 0x7ff) == 0x7ff;
          xb[(int64_t)c * nc + i] = xn;
          if (b > 0) Us[c * np + i] = dpi * z;
        };
        if (dseg == 0) {
          const int i = seg0 * 32 + lane;
          if (i < nx) {
            // dup is zero on row 0, so its product input is written there too
            const T sci = sc[i], dpi = dup[i];
            double* xp = xb + (int64_t)col0 * nc + i;
            const int64_t xs = (int64_t)dcol * nc;
            int zo = col0 * np + i;
            const int zs = dcol * np;
            for (int c = col0; c < C; c += 4 * dcol, xp += 4 * xs, zo += 4 * zs) {
              double xo[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) xo[u] = (it > 0 && c + u * dcol < C) ? xp[u * xs] : 0.0;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (c + u * dcol >= C) break;
                const T z = Zs[zo + u * zs];
                const T dt = sci * z;
                const float df = to_f32(dt);
                dn2f = fmaf(df, df, dn2f);
                const double xn = it == 0 ? to_f64(dt) : xo[u] + to_f64(dt);
                nonfinite |= ((__double2hiint(xn) >> 20) & 0x7ff) == 0x7ff;
                xp[u * xs] = xn;
                Us[zo + u * zs] = dpi * z;
              }
            }
          }
        } else {
          int sg = seg0, c = col0;
          while (c < C) {
            const int i = sg * 32 + lane;
            if (i < nx) upd(i, c, sc[i], dup[i], it > 0 ? xb[(int64_t)c * nc + i] : 0.0);
            sg += dseg;
            c += dcol;
            if (sg >= nseg) { sg -= nseg; ++c; }
          }
        }
      }
      // the reads of Zs above come before the next row's copy into it
      fence_async_shared();
      __syncthreads();
      SFB_MARK(11);
    }
    if (timeout) break;
    const double dn2 = block_sum((double)dn2f, red);
    if (threadIdx.x == 0) { const long long t = clock64(); clk[kBwd] += t - clk[kMark]; clk[kMark] = t; clk[kSub] = t; }
    if (it == 0) {
      xref2 = dn2;  // ||x_0||^2
      prev_corr = 1.0;
      est = 1.0;
    } else {
      const double corr = sqrt(dn2 / fmax(xref2, 1e-300));  // ||d_it|| / ||x||
      const double rho = corr / fmax(prev_corr, 1e-300);
      est = rho < 1.0 ? rho / (1.0 - rho) * corr : 1.0;
      if (threadIdx.x == 0 && it == 1) a.corr1[wid] = corr;
      prev_corr = corr;
      n_done = it;
      if (est <= a.refine_tol) break;
      if (rho > 0.5) {
        st |= ST_NOT_CONVERGED;
        break;
      }
      if (it == refine) st |= ST_NOT_CONVERGED;
    }
  }
  if (timeout) {
    // give the copies in flight a bounded chance to land before the CTA exits
    if (threadIdx.x == tma) {
      if (GB > 0) mbar_wait(&gbar[0], gph[0]);
      mbar_wait(&gbar[1], gph[1]);
      mbar_wait(&zbar, zph);
      bulk_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicOr(&a.status[id], ST_TIMEOUT);
    return;
  }
  if (threadIdx.x == 0) {
    bulk_wait_all();
    cyc[2] = clk[kFwd];
    cyc[3] = clk[kBwd];
    for (int q = 0; q < 12; ++q) cyc[4 + q] = clk[q];
    a.nref[wid] = n_done;
    a.errest[wid] = refine > 0 ? est : 0.0;
  }
  // non-finite entries of X (every value X took was checked when stored; a
  // non-finite entry stays non-finite under later corrections)
  if (nonfinite) st |= ST_NONFINITE;
  __syncthreads();
  if (bad_spd) st |= ST_NOT_SPD;
  if (st) atomicOr(&a.status[id], st);
#undef SFB_MARK
}

template <typename T, int MT, int NT, int MINB, int GB, int MODE = 0>
__global__ void __launch_bounds__(NT, MINB) basis_kernel(BasisArgs a, int refine) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int bad_spd;
  __shared__ __align__(8) uint64_t gbar[2];
  __shared__ __align__(8) uint64_t zbar;
  if constexpr (MODE == 2) {
    if ((int)blockIdx.x >= a.n_chunks) return;
    basis_body<T, MT, NT, GB, MODE>(a, refine, a.chunk_item[blockIdx.x], a.chunk_c0[blockIdx.x],
                                    a.chunk_cnt[blockIdx.x], a.n_items_all + a.chunk_slot0 + (int)blockIdx.x,
                                    smem_raw, red, bad_spd, gbar, zbar);
  } else {
    if ((int)blockIdx.x >= a.n_items) return;
    basis_body<T, MT, NT, GB, MODE>(a, refine, blockIdx.x, 0, 0, -1, smem_raw, red, bad_spd, gbar, zbar);
  }
}

// Persistent form of the split shapes: one launch for every item of every size
// class. Each CTA takes tasks in order from a counter: first the factor of
// every item (MODE 1), then every column chunk (MODE 2). A chunk waits for its
// item's factor flag. Every factor task is taken before any chunk task, and a
// task is only taken by a running CTA, so the factor a chunk waits for is
// already running; the wait is bounded all the same (about 4 s), after which
// the chunk's item is marked ST_TIMEOUT and the chunk skipped.
struct PersistArgs {
  int* counter;     // task counter, zero at launch
  int* flags;       // per item (build order): 1 once its factor is in global memory; zero at launch
  int n_items, n_chunks;
  int n_wide;       // the chunks' items are class-local: the wide class first
  int chunk_n0;     // chunks of the wide class
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename T, int MT, int NT, int MINB, int GB>
__global__ void __launch_bounds__(NT, MINB) basis_persistent_kernel(BasisArgs a, int refine, PersistArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int bad_spd;
  __shared__ __align__(8) uint64_t gbar[2];
  __shared__ __align__(8) uint64_t zbar;
  __shared__ int task, ready;
  const int n_tasks = p.n_items + p.n_chunks;
  for (;;) {
    __syncthreads();   // the last task's reads of `task` and of the barriers are done
    if (threadIdx.x == 0) task = atomicAdd(p.counter, 1);
    __syncthreads();
    const int t = task;
    if (t >= n_tasks) break;
    if (t < p.n_items) {
      basis_body<T, MT, NT, GB, 1>(a, refine, t, 0, 0, -1, smem_raw, red, bad_spd, gbar, zbar);
      // publish the factor: every thread's global stores, then the flag
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        fence_async_global();
        __threadfence();
        atomicExch(&p.flags[t], 1);
      }
    } else {
      const int ch = t - p.n_items;
      const int item = (ch < p.chunk_n0 ? 0 : p.n_wide) + a.chunk_item[ch];
      if (threadIdx.x == 0) {
        int ok = 0;
        for (int k = 0; k < (1 << 24); ++k) {
          if (ld_acquire(&p.flags[item]) == 1) { ok = 1; break; }
          __nanosleep(256);
        }
        fence_async_global();   // the bulk loads of the factor come after the acquire
        ready = ok;
      }
      __syncthreads();
      if (ready) {
        basis_body<T, MT, NT, GB, 2>(a, refine, item, a.chunk_c0[ch], a.chunk_cnt[ch], a.n_items_all + ch, smem_raw,
                                     red, bad_spd, gbar, zbar);
      } else if (threadIdx.x == 0) {
        const SubDev& S = a.subs[a.item_sub[item]];
        atomicOr(&a.status[S.item0 + a.item_k[item]], ST_TIMEOUT);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the body initialises them again for the next task
      mbar_inval(&gbar[0]);
      mbar_inval(&gbar[1]);
      mbar_inval(&zbar);
    }
  }
}

// Phi[l][j] = -sum_e P[e][l] T_e (X[c_e][j] - P[e][j]) (j < R) and
// g[l] = sum_e P[e][l] T_e X[c_e][R], the sum running over the faces e of the
// side that carries mortar DOF l and lying in the support of xi_l.
__global__ void flux_epilogue_kernel(BasisArgs a) {
  const int item = blockIdx.x;
  if (item >= a.n_items) return;
  const int s = a.item_sub[item], kk = a.item_k[item];
  const SubDev& S = a.subs[s];
  const int id = (int)S.item0 + kk;
  const ItemOff off = a.off[id];
  const int nx = S.nx, ny = S.ny, R = S.R, C = R + 1, nc = nx * ny;
  const double* Tx = a.T + off.t;
  const double* Ty = Tx + (int64_t)ny * (nx + 1);
  const double* X = a.X + off.x;
  double* phi = a.phi + off.phi;
  const int* info = a.dofinfo + S.dofinfo_off;
  // Method S1's set-up keeps only the particular solution (X's column R): g alone
  const int ncol = a.particular_only ? 1 : C;
  for (int e2 = threadIdx.x; e2 < R * ncol; e2 += blockDim.x) {
    const int l = e2 / ncol, j = a.particular_only ? R : e2 - l * ncol;
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
      acc += pl * t * (X[(int64_t)j * nc + cell] - pj);
    }
    const int64_t o = j < R ? (int64_t)l * R + j : (int64_t)R * R + l;
    const double v = j < R ? -acc : acc;
    phi[o] = v;
    if (a.phi32) a.phi32[off.phi + o] = (float)v;
  }
}

// G buffers: two (prefetch of the next block row) where shared memory allows,
// one where it would limit residency: the FP64 factor, and the default FP32
// shape for grids up to 64 cells wide, which runs 4 CTAs per SM instead of 3
// (648 items of 64x64 cells in 1.07 waves instead of 1.42; measured 17.8 ms
// against 18.0 ms, the lost prefetch and 64 registers included). The
// autotuner times both FP32 shapes of each size class (kShape below).
template <typename T>
size_t basis_smem(int max_nx, int max_cols, int gb, int mode = 0) {
  // mode 1 (factor alone) holds no right-hand sides; mode 2 (a chunk's
  // solves) at most kChunkCols of them and no inversion scratch
  const size_t cp = mode == 1 ? 0 : mode == 2 ? (size_t)((std::min(max_cols, kChunkCols) + 3) & ~3)
                                               : (size_t)((max_cols + 3) & ~3);
  constexpr size_t kP = panel_of<T>();
  const size_t np = (max_nx + kPanel - 1) & ~size_t(kPanel - 1);
  const size_t ureg = mode == 2 ? np * cp : std::max(np * cp, 2 * kP * np + kP * kP);
  // + the two end cells' right-hand sides of a row in the solves (FP64)
  return sizeof(T) * (gb * np * np + ureg + np * cp + 4 * np) + (mode == 1 ? 0 : 2 * cp * sizeof(double));
}

template <typename T, int MT, int NT, int MINB, int GB, int MODE = 0>
cudaError_t launch_one(const BasisArgs& a, size_t smem, int refine, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(basis_kernel<T, MT, NT, MINB, GB, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = MODE == 2 ? a.n_chunks : a.n_items;
  if (grid == 0) return cudaSuccess;
  basis_kernel<T, MT, NT, MINB, GB, MODE><<<grid, NT, smem, st>>>(a, refine);
  return cudaGetLastError();
}

// A split shape: the factor of every item (part 1), then the solves of every
// chunk (part 2); part 0 runs both on one stream.
template <typename T, int MT1, int NT1, int MINB1, int GB1, int MT2, int NT2, int MINB2, int GB2>
cudaError_t launch_split(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st, int part) {
  cudaError_t e = cudaSuccess;
  if (part != 2)
    e = launch_one<T, MT1, NT1, MINB1, GB1, 1>(a, basis_smem<T>(max_nx, max_cols, GB1, 1), refine, st);
  if (e != cudaSuccess || part == 1) return e;
  return launch_one<T, MT2, NT2, MINB2, GB2, 2>(a, basis_smem<T>(max_nx, max_cols, GB2, 2), refine, st);
}

// Thread-block shape: the register tiles of the sweep are 4 x 4; np <= 64
// gives at most 256 tiles (one per thread of 256), np <= 128 at most 1024
// (four per thread of 256 for FP32, two per thread of 512 for FP64).
template <typename T>
cudaError_t launch_basis(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (max_nx <= 64) return launch_one<T, 1, 256, 4, 1>(a, basis_smem<T>(max_nx, max_cols, 1), refine, st);
    return launch_one<T, 4, 256, 1, 2>(a, basis_smem<T>(max_nx, max_cols, 2), refine, st);
  } else {
    if (max_nx <= 64) return launch_one<T, 1, 256, 2, 1>(a, basis_smem<T>(max_nx, max_cols, 1), refine, st);
    return launch_one<T, 2, 512, 1, 1>(a, basis_smem<T>(max_nx, max_cols, 1), refine, st);
  }
}

// Launch shapes per precision and size class (wide: grids more than 64 cells
// wide), the candidates that the build's autotuner times. Shape 0 is the one
// launch_basis picks. FP32 has a second shape per class that trades the G
// prefetch buffer against resident CTAs the other way: narrow grids 3 CTAs per
// SM with two G buffers, wide grids 2 CTAs per SM with one. Its third shape,
// narrow grids only, is the tensor-core kernel of basis_tc.cu. FP64 has one
// shape per class (its shared memory already limits residency). Entries with
// zero threads do not exist.
// The split shapes (split = 1) run a factor launch (256 threads, MODE 1) and
// a solve launch over the column chunks (MODE 2); the table gives the solve
// launch's threads, CTAs per SM and G buffers.
constexpr int kShapes = 4;
constexpr BasisShape kShape[2][2][kShapes] = {
    // FP32: narrow, wide
    {{{256, 4, 1, 0, 0}, {256, 3, 2, 0, 0}, {256, 3, 1, 1, 0}, {128, 7, 1, 0, 1}},
     {{256, 1, 2, 0, 0}, {256, 2, 1, 0, 0}, {128, 2, 1, 0, 1}, {0, 0, 0, 0, 0}}},
    // FP64: narrow, wide (the second wide shape keeps G_b in global memory,
    // for blocks too large for shared memory beside the right-hand sides)
    {{{256, 2, 1, 0, 0}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}},
     {{512, 1, 1, 0, 0}, {512, 1, 0, 0, 0}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}}},
};

template <typename T, int MT, int NT, int MINB, int GB, int MODE = 0>
cudaError_t occupancy_of(size_t smem, int* ctas) {
  cudaError_t e = cudaFuncSetAttribute(basis_kernel<T, MT, NT, MINB, GB, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, basis_kernel<T, MT, NT, MINB, GB, MODE>, NT, smem);
}

// Launches (ctas == nullptr) or sizes (ctas != nullptr: resident CTAs per SM)
// one shape. The template arguments match kShape.
template <typename T>
cudaError_t shape_dispatch(const BasisArgs* a, bool wide, int shape, int max_nx, int max_cols, int refine,
                           cudaStream_t st, int* ctas, int part = 0) {
  if constexpr (sizeof(T) == 4) {
    if (!wide && shape == 0) {
      const size_t sm = basis_smem<T>(max_nx, max_cols, 1);
      return ctas ? occupancy_of<T, 1, 256, 4, 1>(sm, ctas) : launch_one<T, 1, 256, 4, 1>(*a, sm, refine, st);
    }
    if (!wide && shape == 1) {
      const size_t sm = basis_smem<T>(max_nx, max_cols, 2);
      return ctas ? occupancy_of<T, 1, 256, 3, 2>(sm, ctas) : launch_one<T, 1, 256, 3, 2>(*a, sm, refine, st);
    }
    if (wide && shape == 0) {
      const size_t sm = basis_smem<T>(max_nx, max_cols, 2);
      return ctas ? occupancy_of<T, 4, 256, 1, 2>(sm, ctas) : launch_one<T, 4, 256, 1, 2>(*a, sm, refine, st);
    }
    if (wide && shape == 1) {
      const size_t sm = basis_smem<T>(max_nx, max_cols, 1);
      return ctas ? occupancy_of<T, 4, 256, 2, 1>(sm, ctas) : launch_one<T, 4, 256, 2, 1>(*a, sm, refine, st);
    }
    if (!wide && shape == 2)
      return ctas ? basis_tc_ctas(max_nx, max_cols, ctas) : launch_basis_tc(*a, max_nx, max_cols, refine, st);
    if (!wide && shape == 3)
      return ctas ? occupancy_of<T, 1, 128, 7, 1, 2>(basis_smem<T>(max_nx, max_cols, 1, 2), ctas)
                  : launch_split<T, 2, 128, 5, 1, 1, 128, 7, 1>(*a, max_nx, max_cols, refine, st, part);
    if (wide && shape == 2)
      return ctas ? occupancy_of<T, 1, 128, 2, 1, 2>(basis_smem<T>(max_nx, max_cols, 1, 2), ctas)
                  : launch_split<T, 4, 256, 2, 1, 1, 128, 2, 1>(*a, max_nx, max_cols, refine, st, part);
  } else {
    const size_t sm = basis_smem<T>(max_nx, max_cols, 1);
    if (!wide && shape == 0)
      return ctas ? occupancy_of<T, 1, 256, 2, 1>(sm, ctas) : launch_one<T, 1, 256, 2, 1>(*a, sm, refine, st);
    if (wide && shape == 0)
      return ctas ? occupancy_of<T, 2, 512, 1, 1>(sm, ctas) : launch_one<T, 2, 512, 1, 1>(*a, sm, refine, st);
    if (wide && shape == 1) {
      const size_t sm0 = basis_smem<T>(max_nx, max_cols, 0);
      return ctas ? occupancy_of<T, 2, 512, 1, 0>(sm0, ctas) : launch_one<T, 2, 512, 1, 0>(*a, sm0, refine, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int basis_shape_count(int fp64) { return fp64 ? 2 : kShapes; }

bool basis_shape_split(int fp64, int wide, int shape) {
  BasisShape d;
  return basis_shape_desc(fp64, wide, shape, &d) && d.split;
}

bool basis_shape_desc(int fp64, int wide, int shape, BasisShape* out) {
  if (shape < 0 || shape >= basis_shape_count(fp64)) return false;
  const BasisShape& d = kShape[fp64 ? 1 : 0][wide ? 1 : 0][shape];
  if (d.threads == 0) return false;
  *out = d;
  return true;
}

cudaError_t basis_shape_ctas(int fp64, int wide, int shape, int max_nx, int max_cols, int* ctas) {
  *ctas = 0;
  BasisShape d;
  if (!basis_shape_desc(fp64, wide, shape, &d)) return cudaErrorInvalidValue;
  if ((wide != 0) != (max_nx > 64)) return cudaErrorInvalidValue;
  return fp64 ? shape_dispatch<double>(nullptr, wide, shape, max_nx, max_cols, 0, nullptr, ctas)
              : shape_dispatch<float>(nullptr, wide, shape, max_nx, max_cols, 0, nullptr, ctas);
}

cudaError_t launch_basis_shape(const BasisArgs& a, int fp64, int wide, int shape, int max_nx, int max_cols,
                               int refine, cudaStream_t st) {
  BasisShape d;
  if (!basis_shape_desc(fp64, wide, shape, &d)) return cudaErrorInvalidValue;
  if ((wide != 0) != (max_nx > 64)) return cudaErrorInvalidValue;
  return fp64 ? shape_dispatch<double>(&a, wide, shape, max_nx, max_cols, 0, st, nullptr)
              : shape_dispatch<float>(&a, wide, shape, max_nx, max_cols, refine, st, nullptr);
}

namespace {
template <typename T, int MT, int NT, int MINB, int GB>
cudaError_t persistent_one(const BasisArgs& a, const PersistArgs& p, int max_nx, int max_cols, int refine,
                           cudaStream_t st, int* ctas) {
  const size_t smem = std::max(basis_smem<T>(max_nx, max_cols, GB, 1), basis_smem<T>(max_nx, max_cols, GB, 2));
  auto fn = basis_persistent_kernel<T, MT, NT, MINB, GB>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NT, smem);
  if (e != cudaSuccess) return e;
  if (ctas) { *ctas = per; return cudaSuccess; }
  if (per < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, n_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.counter, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.flags, 0, sizeof(int) * std::max(p.n_items, 1), st);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.n_items + p.n_chunks, per * n_sm);
  if (grid == 0) return cudaSuccess;
  fn<<<grid, NT, smem, st>>>(a, refine, p);
  return cudaGetLastError();
}
}  // namespace

// One instantiation for both size classes: the wide one's register tiles (up
// to 128-wide grids) when there are wide items, else the narrow one's.
cudaError_t launch_basis_persistent(const BasisArgs& a, int* counter, int* flags, int n_wide, int chunk_n0,
                                    int max_nx, int max_cols, int refine, cudaStream_t st, int* ctas) {
  PersistArgs p;
  p.counter = counter;
  p.flags = flags;
  p.n_items = a.n_items;
  p.n_chunks = a.n_chunks;
  p.n_wide = n_wide;
  p.chunk_n0 = chunk_n0;
  if (max_nx > 128) return cudaErrorInvalidValue;
  return max_nx > 64 ? persistent_one<float, 4, 256, 2, 1>(a, p, max_nx, max_cols, refine, st, ctas)
                     : persistent_one<float, 1, 256, 4, 1>(a, p, max_nx, max_cols, refine, st, ctas);
}

cudaError_t launch_basis_part(const BasisArgs& a, int wide, int shape, int part, int max_nx, int max_cols, int refine,
                              cudaStream_t st) {
  if (!basis_shape_split(0, wide, shape) || (wide != 0) != (max_nx > 64)) return cudaErrorInvalidValue;
  return shape_dispatch<float>(&a, wide, shape, max_nx, max_cols, refine, st, nullptr, part);
}

cudaError_t launch_basis_fp64(const BasisArgs& a, int max_nx, int max_cols, cudaStream_t st) {
  return launch_basis<double>(a, max_nx, max_cols, 0, st);
}

cudaError_t launch_basis_mixed(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st) {
  return launch_basis<float>(a, max_nx, max_cols, refine, st);
}

cudaError_t launch_flux_epilogue(const BasisArgs& a, int /*max_R*/, cudaStream_t st) {
  flux_epilogue_kernel<<<a.n_items, 256, 0, st>>>(a);
  return cudaGetLastError();
}

size_t basis_smem_bytes(int prec_fp64, int max_nx, int max_cols) {
  // the largest of the launch shapes (FP32 grids wider than 64 cells keep two G buffers)
  return prec_fp64 ? basis_smem<double>(max_nx, max_cols, 1) : basis_smem<float>(max_nx, max_cols, max_nx <= 64 ? 1 : 2);
}

}  // namespace sfb
