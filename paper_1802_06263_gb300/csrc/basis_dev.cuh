// Device helpers shared by the basis kernels (basis.cu: the CUDA-core form,
// basis_tc.cu: the tensor-core form): right-hand sides of the subdomain
// problems, block reductions, bulk asynchronous copies and mbarriers, and the
// block-row factor step (the blocked symmetric sweep of one diagonal block).
#pragma once

#include <math.h>

#include "sfb_internal.h"

namespace sfb {

namespace {

struct Geo {
  int nx, ny, R, C, Cp, nc;
  const double* Tx;  // [ny][nx+1]
  const double* Ty;  // [ny+1][nx]
  double src;        // source * hx * hy, the particular column's entry of an inner cell
};

// Right-hand side entry B[(b, i)][c] in FP64: interface columns c < R carry
// T_e * P_side[face][c] on interface faces of boundary cells; column R carries
// the source and the outer Dirichlet data. The terms of the boundary cells
// sit in a function of their own, called (not inlined) from the cells of the
// grid's outer ring only: inlined, its FP64 products were issued, predicated
// off, for every entry, and the FP64 pipe runs at 1/64 of the FP32 rate.
__device__ __noinline__ double rhs_boundary(const SubDev& S, const Geo& g, const double* proj, int b, int i,
                                            int c) {
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
    v = g.src;
    if (b == 0 && S.side_type[0] == SIDE_DIRICHLET) v += g.Ty[i] * S.side_val[0];
    if (b == ny - 1 && S.side_type[2] == SIDE_DIRICHLET) v += g.Ty[ny * nx + i] * S.side_val[2];
    if (i == 0 && S.side_type[3] == SIDE_DIRICHLET) v += g.Tx[b * (nx + 1)] * S.side_val[3];
    if (i == nx - 1 && S.side_type[1] == SIDE_DIRICHLET) v += g.Tx[b * (nx + 1) + nx] * S.side_val[1];
  }
  return v;
}
__device__ __forceinline__ double rhs_entry(const SubDev& S, const Geo& g, const double* proj, int b, int i,
                                            int c) {
  if (b > 0 && b < g.ny - 1 && i > 0 && i < g.nx - 1) return c < g.R ? 0.0 : g.src;
  return rhs_boundary(S, g, proj, b, i, c);
}

// 4 consecutive values from a 16-byte aligned address (one float4 or two
// double2 shared-memory loads).
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p);
  const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// 4 consecutive values to a 16-byte aligned address.
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// out[c][i] (+)= sum_k G[i][k] U[c][k] for i < np, c < C. The right-hand-side
// blocks U and out are column-major with pitch np (entry (i, c) at c * np + i);
// G is symmetric with pitch np, so row k of G is read as its column k. np is a
// multiple of 16 and all three arrays start 16-byte aligned, so every 4-wide
// access is aligned. A thread owns a tile of 4 cells by 4 columns (cells
// fastest across threads: a warp's G reads are contiguous and its U reads
// broadcasts); the last C mod 4 columns form tiles of 4 cells by 1-3 columns.
// Per KS = 16 / sizeof(T) steps of k a thread reads KS rows of G and 4
// column pieces of U, 16 bytes each, for 16 KS FMAs.
// 1 / x correctly rounded (the value of the IEEE division 1 / x), by the
// reciprocal intrinsics rather than the division sequence.
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// KS consecutive values (one 16-byte load) from a 16-byte aligned address.
__device__ __forceinline__ void load_ks(const float* p, float (&v)[4]) { load4(p, v); }
__device__ __forceinline__ void load_ks(const double* p, double (&v)[2]) {
  const double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x; v[1] = q.y;
}

// One thread's tile of the product: cells i0..i0+3 of columns c0..c0+NQ-1.
// NP > 0 fixes np at compile time, so every shared-memory offset inside the
// k loop is an immediate.
template <typename T, int NQ, int NP>
__device__ __forceinline__ void gemm_tile(const T* __restrict__ G, const T* __restrict__ U, T* out, bool add_base,
                                          int np_rt, int i0, int c0) {
  constexpr int KS = 16 / (int)sizeof(T);   // steps of k per 16-byte piece of a U column
  const int np = NP > 0 ? NP : np_rt;
  T acc[NQ][4];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[q][a] = T(0);
  const T* gp = G + i0;
  const T* up = U + c0 * np;
#pragma unroll 2
  for (int k = 0; k < np; k += KS) {
    T gv[KS][4];
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) load4(gp + kk * np, gv[kk]);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T uv[KS];
      load_ks(up + q * np, uv);
#pragma unroll
      for (int kk = 0; kk < KS; ++kk)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[q][a] = fma(gv[kk][a], uv[kk], acc[q][a]);
    }
    gp += KS * np;
    up += KS;
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T* o = out + (c0 + q) * np + i0;
    if (add_base) {
      T base[4];
      load4(o, base);
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[q][a] += base[a];
    }
    store4(o, acc[q]);
  }
}

template <typename T, int NP>
__device__ __forceinline__ void gemm_g_np(const T* __restrict__ G, const T* __restrict__ U, T* out, bool add_base,
                                          int np, int C) {
  const int nrt = (NP > 0 ? NP : np) >> 2;
  const int Cm = C & ~3;
  const int nmain = nrt * (Cm >> 2);
  const int rc = C - Cm;
  const int ntot = nmain + (rc ? nrt : 0);
  for (int t = threadIdx.x; t < ntot; t += blockDim.x) {
    if (t < nmain) {
      const int ct = t / nrt;
      gemm_tile<T, 4, NP>(G, U, out, add_base, np, (t - ct * nrt) * 4, ct * 4);
    } else {
      const int i0 = (t - nmain) * 4;
      if (rc == 1) gemm_tile<T, 1, NP>(G, U, out, add_base, np, i0, Cm);
      else if (rc == 2) gemm_tile<T, 2, NP>(G, U, out, add_base, np, i0, Cm);
      else gemm_tile<T, 3, NP>(G, U, out, add_base, np, i0, Cm);
    }
  }
}

template <typename T>
__device__ __forceinline__ void gemm_g(const T* __restrict__ G, const T* __restrict__ U, T* out, bool add_base,
                                       int np, int C) {
  if (np == 64) gemm_g_np<T, 64>(G, U, out, add_base, np, C);
  else if (np == 128) gemm_g_np<T, 128>(G, U, out, add_base, np, C);
  else if (np == 32) gemm_g_np<T, 32>(G, U, out, add_base, np, C);
  else if (np == 96) gemm_g_np<T, 96>(G, U, out, add_base, np, C);
  else gemm_g_np<T, 0>(G, U, out, add_base, np, C);
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

// ---- bulk asynchronous copies (TMA engine) and mbarriers ---------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// global -> shared bulk copy completing on `bar` (issued by one thread)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// shared -> global bulk copy in the thread's bulk group (issued by one thread)
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar`; false after the iteration limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Pivots per panel of the blocked sweep: 16 in the FP32 factor (register-resident
// pivot-block inverse in every warp), 8 in the FP64 one (one inverse by warp 0).
template <typename T>
__host__ __device__ constexpr int panel_of() { return sizeof(T) == 4 ? 16 : 8; }

// L2 prefetch of grid row b of all C columns of X (column-major, nx doubles
// per row segment): one 128-byte line per thread.
__device__ __forceinline__ void prefetch_x_row(const double* X, int64_t nc, int nx, int b, int C) {
  const int lines = (nx * 8 + 127) >> 7;
  for (int t = threadIdx.x; t < lines * C; t += blockDim.x) {
    const int c = t / lines, q = t - c * lines;
    const double* p = X + (int64_t)c * nc + (int64_t)b * nx + q * 16;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

// Block row b of the scaled matrix into the register tiles of the sweep:
// S_b = Ahat_bb - D_{b-1} G_{b-1} D_{b-1}; on entry the tiles hold -G_{b-1}.
// Rows / columns nx..np-1 are an identity padding.
template <typename T, int MT, int NT>
__device__ __forceinline__ void form_block(T (&areg)[MT][4][4], int b, int nx, int ntr, const T* txh,
                                           const T* dlo) {
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    const int t = threadIdx.x + m * NT;
    if (t >= ntr * ntr) break;
    const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + a, j = j0 + q;
        T v;
        if (i >= nx || j >= nx) {
          v = (i == j) ? T(1) : T(0);
        } else {
          v = (i == j) ? T(1) : (j == i + 1 ? txh[j] : (j == i - 1 ? txh[i] : T(0)));
          if (b > 0) v = fma(dlo[i] * areg[m][a][q], dlo[j], v);
        }
        areg[m][a][q] = v;
      }
  }
}

// Blocked symmetric sweep of the np x np SPD matrix held in register tiles:
// for each panel K of kP pivots, A_KK -> -A_KK^{-1}, A_KJ -> A_KK^{-1} A_KJ,
// A_JK -> A_JK A_KK^{-1}, A_JJ -> A_JJ - A_JK A_KK^{-1} A_KJ (the composition
// of kP single-pivot sweeps). On exit the tiles hold -S^{-1}.
// Per panel: (a) the panel columns go to VT; (b) every warp sweeps the kP x kP
// pivot block in registers (lane p % kP holds row p; the pivot row arrives
// by shuffles) and forms its share of W = A_KK^{-1} A_K* from VT; (c) the
// register tiles take the rank-kP update. Three barriers per panel.
template <typename T, int MT, int NT, int kP>
__device__ __forceinline__ void blocked_sweep(T (&areg)[MT][4][4], int np, int ntr, T* VT, T* W, T* Ablk,
                                              int* bad) {
  static_assert(kP == 16, "the pivot-block layout puts one row per half-warp lane");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nwarp = NT / 32;
  const int p = lane & (kP - 1), half = lane >> 4;
  for (int k0 = 0; k0 < np; k0 += kP) {
    // (a) panel columns: VT[q][i] = A[i][k0 + q]
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
    // (b) row p of the pivot block, A_KK[p][q] = A[k0 + q][k0 + p], swept in
    // registers to row p of -A_KK^{-1}
    T row[kP];
#pragma unroll
    for (int q = 0; q < kP; ++q) row[q] = VT[q * np + k0 + p];
#pragma unroll
    for (int kk = 0; kk < kP; ++kk) {
      T piv = __shfl_sync(0xffffffffu, row[kk], kk);
      if (!(piv > T(0))) {
        if (lane == 0 && warp == 0) *bad = 1;
        piv = T(1);
      }
      const T inv = rcp_rn(piv);
      const T colk = row[kk];
#pragma unroll
      for (int q = 0; q < kP; ++q) {
        const T rowk = __shfl_sync(0xffffffffu, row[q], kk);
        T v;
        if (p == kk) v = q == kk ? -inv : rowk * inv;
        else v = q == kk ? colk * inv : fma(-colk, rowk * inv, row[q]);
        row[q] = v;
      }
    }
    if (warp == 0 && half == 0)
#pragma unroll
      for (int q = 0; q < kP; ++q) Ablk[p * kP + q] = row[q];
    // W[p][j] = sum_q A_KK^{-1}[p][q] A[k0 + q][j] for this warp's columns j
    const int cpw = np / nwarp;
    for (int j = warp * cpw + half; j < (warp + 1) * cpw; j += 2) {
      T w = T(0);
#pragma unroll
      for (int q = 0; q < kP; ++q) w = fma(-row[q], VT[q * np + j], w);
      W[p * np + j] = w;
    }
    __syncthreads();
    // (c) update the register tiles
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int t = threadIdx.x + m * NT;
      if (t >= ntr * ntr) break;
      const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
      const bool rk = i0 >= k0 && i0 < k0 + kP, ck = j0 >= k0 && j0 < k0 + kP;
      if (!rk && !ck) {
#pragma unroll
        for (int pp = 0; pp < kP; ++pp) {
          T v4[4], w4[4];
          load4(VT + pp * np + i0, v4);
          load4(W + pp * np + j0, w4);
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

}  // namespace

}  // namespace sfb
