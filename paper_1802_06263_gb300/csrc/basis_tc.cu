// Stochastic multiscale flux basis, mixed form, with the block-row products on
// the fifth-generation tensor cores (Section 5.4, pre-computation loop, Steps
// 1-2; Section 5.3: one subdomain solve per mortar DOF).
//
// The method per item is the one of basis.cu: KL permeability (Eq. 2.13),
// cell-centred RT0 operator, block LDL^T recurrence of the diagonally scaled
// 5-point matrix with explicit block inverses G_b = S_b^{-1} (FP32 on the CUDA
// cores), the R + 1 right-hand sides by a forward sweep
// z_b = G_b (s_b r_b + D_{b-1} z_{b-1}) and a backward sweep
// d_b = z_b + G_b (D_b d_{b+1}), x_b += s_b d_b, and refinement with FP64
// residuals r = B - A X of the 5-point stencil. What changes is where the
// products G_b U run:
//  - each product is one group of tcgen05.mma kind::tf32 instructions of shape
//    M = 64 (the block rows, identity-padded to np <= 64), N = R + 1 rounded up
//    to 8, K = np, issued by one thread with the FP32 accumulator in tensor
//    memory (TMEM);
//  - both operands are split into TF32 pairs, x = hi + lo with
//    hi = rna_tf32(x), lo = rna_tf32(x - hi), and the product is
//    A_lo B_hi + A_hi B_lo + A_hi B_hi (three passes, FP32 accumulation): the
//    accuracy of an FP32 product (about 2^-21 relative per term) from a unit
//    that rounds its inputs to 10 fraction bits;
//  - the block inverses are written row-major to global memory (hi and lo
//    arrays) by the factor and come back in each sweep by 2-D TMA tensor
//    copies (cp.async.bulk.tensor, box {4 columns, np rows}) that land them in
//    the no-swizzle K-major core-matrix layout the MMA reads;
//  - the right-hand-side block is written by the threads in the same layout.
// The accumulator of M = 64 occupies TMEM lanes 0-15 of each 32-lane quadrant
// (row i in lane 32 (i / 16) + i % 16); warp w reads quadrant w % 4 and the
// column chunks j with j % 2 == w / 4, so threads with lane < 16 own one row
// and half the column chunks.
//
// Shared memory: A tiles (hi, lo) 16 KB each: K-chunk kc of 4 columns at
// kc * 1024 bytes, row i at i * 16 bytes within it (LBO 1024, SBO 128); B tiles
// (hi, lo): column n, row k at (n / 8) * 32 np + (k / 4) * 128 + (n % 8) * 16 +
// (k % 4) * 4 bytes (LBO 128, SBO 32 np). The block inversion's scratch shares
// the B-lo tile; the stage of D z (the previous row's contribution) shares the
// B-hi tile.
//
// Every wait is bounded (mbarrier polls); a wait that runs out sets
// ST_TIMEOUT, waits (bounded) for the copies and products in flight, frees
// the tensor memory and returns.
#include <cuda.h>

#include <algorithm>

#include "basis_dev.cuh"

namespace sfb {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 64;         // MMA M: block rows (identity-padded np <= 64)
constexpr uint32_t kTmemCols = 128; // accumulator columns (N <= 72 used)
constexpr int kTcMinCtas = 3;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo with both parts TF32 (10 fraction bits)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  const uint32_t h = tf32_rna(x);
  hi = __uint_as_float(h);
  lo = __uint_as_float(tf32_rna(x - hi));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading and
// stride byte offsets (all >> 4), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__device__ __forceinline__ uint32_t umma_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrives on `bar` once every tcgen05 operation this thread issued is complete
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 8 columns of 32 bits: thread t of the warp gets lane (base + t)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
// 2-D tensor copy global -> shared completing on `bar` (one thread)
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Offsets (floats) in the core-matrix layouts of the A tiles (row i, column k)
// and the B tiles (column n, row k; K extent np).
__device__ __forceinline__ int a_off(int i, int k) { return (k >> 2) * (kTcRows * 4) + i * 4 + (k & 3); }
__device__ __forceinline__ int b_off(int n, int k, int np) { return (n >> 3) * (np * 8) + (k >> 2) * 32 + (n & 7) * 4 + (k & 3); }

// Loads G_b (hi and lo) into the A tiles: np / 4 boxes of {4, np} per part.
__device__ __forceinline__ void load_g(float* Ahi, float* Alo, const void* map, int b, int np, int ny, uint64_t* bar) {
  const uint32_t bytes = 2u * np * np * 4u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  for (int kc = 0; kc < np / 4; ++kc) {
    tma_load_2d(Ahi + kc * kTcRows * 4, map, kc * 4, b * np, bar);
    tma_load_2d(Alo + kc * kTcRows * 4, map, kc * 4, (ny + b) * np, bar);
  }
}

// D (TMEM) = G (A tiles) times U (B tiles) in three TF32 passes.
__device__ __forceinline__ void issue_product(uint32_t tmem, const float* Ahi, const float* Alo, const float* Bhi,
                                              const float* Blo, int np, uint32_t idesc) {
  const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
  const uint32_t sbo_b = (uint32_t)np * 32u;
  uint32_t acc = 0u;
#pragma unroll 1
  for (int t = 0; t < 3; ++t) {
    const uint32_t aa = t == 0 ? al : ah;   // lo*hi, hi*lo, then hi*hi
    const uint32_t bb = t == 1 ? bl : bh;
#pragma unroll 1
    for (int s = 0; s < np / 8; ++s) {
      mma_tf32(tmem, umma_desc(aa + s * 2 * kTcRows * 16, kTcRows * 16, 128),
               umma_desc(bb + s * 256, 128, sbo_b), idesc, acc);
      acc = 1u;
    }
  }
}

__global__ void __launch_bounds__(kTcThreads, kTcMinCtas) basis_tc_kernel(BasisArgs a, int refine) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int bad_spd;
  __shared__ __align__(8) uint64_t gbar;   // TMA of G_b
  __shared__ __align__(8) uint64_t mbar;   // product complete
  __shared__ uint32_t tmem_slot;
  const int item = blockIdx.x;
  if (item >= a.n_items) return;
  const int s = a.item_sub[item], kk = a.item_k[item];
  const SubDev S = a.subs[s];
  const int id = (int)S.item0 + kk;
  const ItemOff off = a.off[id];
  Geo g;
  g.nx = S.nx; g.ny = S.ny; g.R = S.R; g.C = S.R + 1; g.Cp = (g.C + 7) & ~7; g.nc = S.nx * S.ny;
  g.src = S.source * S.hx * S.hy;
  const int nx = g.nx, ny = g.ny, nc = g.nc, C = g.C, Cp8 = g.Cp;
  constexpr int kP = 16;
  const int np = (nx + kPanel - 1) & ~(kPanel - 1);
  const int ntr = np >> 2;
  double* Tx = a.T + off.t;
  double* Ty = Tx + (int64_t)ny * (nx + 1);
  g.Tx = Tx; g.Ty = Ty;
  double* X = a.X + off.x;
  double* Dg = a.D + off.diag;
  float* Sg = reinterpret_cast<float*>(a.S) + off.sc;
  float* DLg = reinterpret_cast<float*>(a.DL) + off.sc;
  float* Ghi = reinterpret_cast<float*>(a.G) + off.g;       // [ny][np][np]
  float* Glo = Ghi + (int64_t)ny * np * np;                  // [ny][np][np]
  float* Zg = reinterpret_cast<float*>(a.Z) + off.z;        // [ny][np][Cp8]
  const void* gmap = reinterpret_cast<const CUtensorMap*>(a.gmaps) + id;

  // shared memory carve (see the header comment)
  const int nbf = (max(Cp8 * np, 2 * kP * np + kP * kP) + 31) & ~31;
  float* Ahi = reinterpret_cast<float*>(smem_raw);
  float* Alo = Ahi + kTcRows * kTcRows;
  float* Bhi = Alo + kTcRows * kTcRows;
  float* Blo = Bhi + nbf;
  float* sc = Blo + nbf;
  float* dlo = sc + kTcRows;
  float* txh = dlo + kTcRows;
  float* VT = Blo;                 // block-inversion scratch shares the B-lo tile
  float* W = VT + kP * np;
  float* Ablk = W + kP * np;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, chalf = warp >> 2;
  const int orow = quad * 16 + (lane & 15);           // row owned in the accumulator
  const bool owner = lane < 16 && orow < nx;
  const uint32_t tlane = (uint32_t)(quad * 32) << 16; // TMEM lane base of this warp
  const int nchunk = Cp8 >> 3;
  const uint32_t idesc = umma_idesc_tf32(kTcRows, Cp8);

  for (int e = tid; e < 2 * kTcRows * kTcRows + 2 * nbf + 3 * kTcRows; e += blockDim.x) Ahi[e] = 0.f;
  if (tid == 0) {
    bad_spd = 0;
    mbar_init(&gbar, 1);
    mbar_init(&mbar, 1);
    fence_barrier_init();
    asm volatile("prefetch.tensormap [%0];" ::"l"(gmap) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t gph = 0u, mph = 0u;
  bool g_pending = false, m_pending = false;   // a TMA / a product in flight
  int st = 0;
  bool timeout = false;
  long long t_mark = clock64(), t_fwd = 0, t_bwd = 0;
  long long* cyc = a.cycles + kCycSlots * (int64_t)id;

  // owner: the previous product's rows -> registers, chunk by chunk
  // (callers give f(c, value) for the chunks of this warp)
#define TC_FOR_OWNED(BODY)                                                   \
  for (int j = chalf; j < nchunk; j += 2) {                                  \
    float v_[8];                                                             \
    tmem_ld8(tmem + tlane + (uint32_t)(8 * j), v_);                          \
    if (owner) {                                                             \
      _Pragma("unroll") for (int jj = 0; jj < 8; ++jj) {                     \
        const int c = 8 * j + jj;                                            \
        const float val = v_[jj];                                            \
        BODY                                                                 \
      }                                                                      \
    }                                                                        \
  }

  // ---- 1. permeability, transmissibilities, diagonal and scaling ----------------
  {
    const int nt = S.n_term;
    const double* slam = a.kl + S.kl_off;
    const double* fx = slam + nt;
    const double* fy = fx + (int64_t)nt * nx;
    const double* yl = a.yloc + S.yloc_off + (int64_t)kk * nt;
    for (int c = tid; c < nc; c += blockDim.x) {
      const int ix = c % nx, iy = c / nx;
      double Y = S.mean_y;
      for (int j = 0; j < nt; ++j) Y += slam[j] * yl[j] * fx[j * nx + ix] * fy[j * ny + iy];
      const double K = exp(Y);
      if (!(K > 0.0) || !isfinite(K)) st |= ST_NONFINITE;
      X[c] = K;  // scratch: X is written only after the factorization
    }
    __syncthreads();
    const double nu = S.nu;
    for (int f = tid; f < ny * (nx + 1); f += blockDim.x) {
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
    for (int f = tid; f < (ny + 1) * nx; f += blockDim.x) {
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
    for (int c = tid; c < nc; c += blockDim.x) {
      const int b = c / nx, i = c - b * nx;
      const double d = Tx[b * (nx + 1) + i] + Tx[b * (nx + 1) + i + 1] + Ty[b * nx + i] + Ty[(b + 1) * nx + i];
      Dg[c] = d;
      Sg[c] = (float)(1.0 / sqrt(d));
    }
    __syncthreads();
    for (int c = tid; c < nc; c += blockDim.x) {
      const int b = c / nx, i = c - b * nx;
      DLg[c] = b > 0 ? (float)(Ty[b * nx + i] / sqrt(Dg[c] * Dg[c - nx])) : 0.f;
    }
    __syncthreads();
  }
  if (tid == 0) { const long long t = clock64(); cyc[0] = t - t_mark; t_mark = t; }

  // ---- 2. factorization, fused with the first forward solve -----------------------
  // Row b: wait for the product of row b-1, stage D_{b-1} z_{b-1} (owners, into
  // B-hi) and store z_{b-1}; invert S_b in registers (scratch in B-lo); write
  // G_b into the A tiles and to global memory; form u_b = s_b B_b + stage into
  // the B tiles; issue z_b = G_b u_b.
  float areg[1][4][4];
  for (int b = 0; b <= ny; ++b) {
    if (b > 0) {
      const bool ok = mbar_wait(&mbar, mph);
      mph ^= 1u;
      m_pending = !ok;
      tc_fence_after();
      if (__syncthreads_or(!ok)) { timeout = true; break; }
      float* zrow = Zg + (int64_t)(b - 1) * np * Cp8;
      const float dl = (owner && b < ny) ? DLg[b * nx + orow] : 0.f;
      TC_FOR_OWNED({
        zrow[orow * Cp8 + c] = val;
        if (b < ny && c < C) Bhi[b_off(c, orow, np)] = dl * val;
      })
      tc_fence_before();
    }
    if (b == ny) break;
    for (int i = tid; i < nx; i += blockDim.x) {
      const float si = Sg[b * nx + i];
      sc[i] = si;
      txh[i] = i > 0 ? (float)(-Tx[b * (nx + 1) + i] * (double)si * (double)Sg[b * nx + i - 1]) : 0.f;
      dlo[i] = DLg[b * nx + i];
    }
    __syncthreads();
    form_block<float, 1, kTcThreads>(areg, b, nx, ntr, txh, dlo);
    blocked_sweep<float, 1, kTcThreads, kP>(areg, np, ntr, VT, W, Ablk, &bad_spd);
    // G_b = -(register tiles): A tiles (canonical layout) and the global hi / lo rows
    {
      const int t = tid;
      if (t < ntr * ntr) {
        const int i0 = (t / ntr) * 4, j0 = (t % ntr) * 4;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float4 h, l;
          split_tf32(-areg[0][r][0], h.x, l.x);
          split_tf32(-areg[0][r][1], h.y, l.y);
          split_tf32(-areg[0][r][2], h.z, l.z);
          split_tf32(-areg[0][r][3], h.w, l.w);
          *reinterpret_cast<float4*>(Ahi + a_off(i0 + r, j0)) = h;
          *reinterpret_cast<float4*>(Alo + a_off(i0 + r, j0)) = l;
          const int64_t go = ((int64_t)b * np + i0 + r) * np + j0;
          *reinterpret_cast<float4*>(Ghi + go) = h;
          *reinterpret_cast<float4*>(Glo + go) = l;
        }
      }
    }
    // u_b = s_b B_b + D_{b-1} z_{b-1}: entries (c, i) in blocks of 8 columns x 4
    // rows per warp (conflict-free in the B layout); padding entries get zero
    for (int blk = warp; blk < (Cp8 >> 3) * (np >> 2); blk += kTcThreads / 32) {
      const int c = (blk % (Cp8 >> 3)) * 8 + (lane >> 2), i = (blk / (Cp8 >> 3)) * 4 + (lane & 3);
      const int o = b_off(c, i, np);
      float u = 0.f;
      if (i < nx && c < C) {
        u = sc[i] * f64_to_f32_bits(rhs_entry(S, g, a.proj, b, i, c));
        if (b > 0) u += Bhi[o];
      }
      float h, l;
      split_tf32(u, h, l);
      Bhi[o] = h;
      Blo[o] = l;
    }
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue_product(tmem, Ahi, Alo, Bhi, Blo, np, idesc);
      mma_commit(&mbar);
    }
    m_pending = true;
  }
  // the block inverses were written by generic stores and come back by TMA
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (tid == 0) { const long long t = clock64(); cyc[1] = t - t_mark; t_mark = t; }

  // ---- 3./4. backward sweep, then refine with FP64 residuals -----------------------
  double xref2 = 0.0, prev_corr = 0.0, est = 1.0, bnorm2 = 0.0;
  int n_done = 0;
  for (int it = 0; it <= refine && !timeout; ++it) {
    if (it > 0) {
      // forward sweep: r_b = B_b - (A x)_b in FP64 by all threads; u_b = s_b r_b + D_{b-1} z_{b-1}
      float rr = 0.f;
      for (int b = 0; b <= ny; ++b) {
        if (b > 0) {
          const bool ok = mbar_wait(&mbar, mph);
          mph ^= 1u;
          m_pending = !ok;
          tc_fence_after();
          if (__syncthreads_or(!ok)) { timeout = true; break; }
        }
        if (tid == 0 && b < ny) {
          load_g(Ahi, Alo, gmap, b, np, ny, &gbar);
          g_pending = true;
        }
        if (b > 0) {
          float* zrow = Zg + (int64_t)(b - 1) * np * Cp8;
          const float dl = (owner && b < ny) ? DLg[b * nx + orow] : 0.f;
          TC_FOR_OWNED({
            zrow[orow * Cp8 + c] = val;
            if (b < ny && c < C) Bhi[b_off(c, orow, np)] = dl * val;
          })
          tc_fence_before();
        }
        if (b == ny) break;
        for (int i = tid; i < nx; i += blockDim.x) sc[i] = Sg[b * nx + i];
        __syncthreads();
        for (int blk = warp; blk < (Cp8 >> 3) * (np >> 2); blk += kTcThreads / 32) {
          const int c = (blk % (Cp8 >> 3)) * 8 + (lane >> 2), i = (blk / (Cp8 >> 3)) * 4 + (lane & 3);
          if (i >= nx || c >= C) continue;
          const int64_t cell = (int64_t)b * nx + i;
          const double* xc = X + (int64_t)c * nc;
          double r = fma(-Dg[cell], xc[cell], rhs_entry(S, g, a.proj, b, i, c));
          if (i > 0) r = fma(Tx[b * (nx + 1) + i], xc[cell - 1], r);
          if (i < nx - 1) r = fma(Tx[b * (nx + 1) + i + 1], xc[cell + 1], r);
          if (b > 0) r = fma(Ty[b * nx + i], xc[cell - nx], r);
          if (b < ny - 1) r = fma(Ty[(b + 1) * nx + i], xc[cell + nx], r);
          const float rf = f64_to_f32_bits(r);
          rr = fmaf(rf, rf, rr);
          const int o = b_off(c, i, np);
          float u = sc[i] * rf;
          if (b > 0) u += Bhi[o];
          float h, l;
          split_tf32(u, h, l);
          Bhi[o] = h;
          Blo[o] = l;
        }
        fence_async_shared();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          const bool okg = mbar_wait(&gbar, gph);
          if (okg) {
            g_pending = false;
            tc_fence_after();
            issue_product(tmem, Ahi, Alo, Bhi, Blo, np, idesc);
            mma_commit(&mbar);
          }
        }
        gph ^= 1u;
        m_pending = true;   // (a missing commit makes the next wait run out)
      }
      if (timeout) break;
      const double rnorm2 = block_sum((double)rr, red);
      if (tid == 0) a.resid[id] = sqrt(rnorm2 / fmax(bnorm2, 1e-300));
      if (tid == 0) { const long long t = clock64(); t_fwd += t - t_mark; t_mark = t; }
    } else {
      float bb = 0.f;
      for (int e = tid; e < nc * C; e += blockDim.x) {
        const int c = e / nc, cell = e - c * nc;
        const float v = f64_to_f32_bits(rhs_entry(S, g, a.proj, cell / nx, cell % nx, c));
        bb = fmaf(v, v, bb);
      }
      bnorm2 = block_sum((double)bb, red);
    }
    // backward sweep: d_b = z_b + G_b (D_b d_{b+1}); x_b += s_b d_b. The owners
    // form d_b from their accumulator rows and write v = D_{b-1} d_b (split)
    // into the B tiles; once the product G_{b-1} v is issued, every thread
    // takes entries (c, i) of row b, recovers s_b d_b = (s_b / D_{b-1}) (hi +
    // lo) from the B tiles (relative error below 2^-21, far inside the
    // correction's own) and updates X in FP64 on full warps while the tensor
    // cores run. Row 0, with no product after it, is updated by the owners.
    float dn2f = 0.f;
    for (int b = ny - 1; b >= 0; --b) {
      if (b < ny - 1) {
        const bool ok = mbar_wait(&mbar, mph);
        mph ^= 1u;
        m_pending = !ok;
        tc_fence_after();
        if (__syncthreads_or(!ok)) { timeout = true; break; }
      }
      if (tid == 0 && b >= 1) {
        load_g(Ahi, Alo, gmap, b - 1, np, ny, &gbar);
        g_pending = true;
      }
      // s_b / D_{b-1} per row, for the update below (the previous row's
      // readers passed the barrier above)
      if (b >= 1)
        for (int i = tid; i < nx; i += blockDim.x) txh[i] = Sg[b * nx + i] / DLg[b * nx + i];
      const float* zrow = Zg + (int64_t)b * np * Cp8;
      const float sb = owner ? Sg[b * nx + orow] : 0.f;
      const float dup = (owner && b >= 1) ? DLg[b * nx + orow] : 0.f;   // D_{b-1}: rows b-1 and b
      double* xrow = X + (int64_t)b * nx + orow;
      for (int j = chalf; j < nchunk; j += 2) {
        float v[8];
        if (b < ny - 1) {
          tmem_ld8(tmem + tlane + (uint32_t)(8 * j), v);
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) v[jj] = 0.f;
        }
        if (owner) {
          const float4 z0 = *reinterpret_cast<const float4*>(zrow + orow * Cp8 + 8 * j);
          const float4 z1 = *reinterpret_cast<const float4*>(zrow + orow * Cp8 + 8 * j + 4);
          const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int c = 8 * j + jj;
            if (c >= C) break;
            const float d = zz[jj] + v[jj];
            if (b >= 1) {
              float h, l;
              split_tf32(dup * d, h, l);
              const int o = b_off(c, orow, np);
              Bhi[o] = h;
              Blo[o] = l;
            } else {
              const float dt = sb * d;
              dn2f = fmaf(dt, dt, dn2f);
              double* xp = xrow + (int64_t)c * nc;
              *xp = it == 0 ? to_f64(dt) : *xp + to_f64(dt);
            }
          }
        }
      }
      if (b == 0) break;
      fence_async_shared();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        const bool okg = mbar_wait(&gbar, gph);
        if (okg) {
          g_pending = false;
          tc_fence_after();
          issue_product(tmem, Ahi, Alo, Bhi, Blo, np, idesc);
          mma_commit(&mbar);
        }
      }
      gph ^= 1u;
      m_pending = true;
      // x_b += s_b d_b on full warps, from the B tiles the product is reading
      for (int blk = warp; blk < (Cp8 >> 3) * (np >> 2); blk += kTcThreads / 32) {
        const int c = (blk % (Cp8 >> 3)) * 8 + (lane >> 2), i = (blk / (Cp8 >> 3)) * 4 + (lane & 3);
        if (i >= nx || c >= C) continue;
        const int o = b_off(c, i, np);
        const float dt = txh[i] * (Bhi[o] + Blo[o]);
        dn2f = fmaf(dt, dt, dn2f);
        double* xp = X + (int64_t)c * nc + (int64_t)b * nx + i;
        *xp = it == 0 ? to_f64(dt) : *xp + to_f64(dt);
      }
    }
    if (timeout) break;
    const double dn2 = block_sum((double)dn2f, red);
    if (tid == 0) { const long long t = clock64(); t_bwd += t - t_mark; t_mark = t; }
    if (it == 0) {
      xref2 = dn2;
      prev_corr = 1.0;
      est = 1.0;
    } else {
      const double corr = sqrt(dn2 / fmax(xref2, 1e-300));
      const double rho = corr / fmax(prev_corr, 1e-300);
      est = rho < 1.0 ? rho / (1.0 - rho) * corr : 1.0;
      if (tid == 0 && it == 1) a.corr1[id] = corr;
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
#undef TC_FOR_OWNED
  if (timeout) {
    // give the copies and products in flight a bounded chance to land
    if (tid == 0) {
      if (g_pending) mbar_wait(&gbar, gph);
      if (m_pending) mbar_wait(&mbar, mph);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (timeout) {
    if (tid == 0) atomicOr(&a.status[id], ST_TIMEOUT);
    return;
  }
  if (tid == 0) {
    cyc[2] = t_fwd;
    cyc[3] = t_bwd;
    for (int q = 4; q < kCycSlots; ++q) cyc[q] = 0;
    a.nref[id] = n_done;
    a.errest[id] = refine > 0 ? est : 0.0;
  }
  for (int e = tid; e < nc * C; e += blockDim.x)
    if (!isfinite(X[e])) st |= ST_NONFINITE;
  __syncthreads();
  if (bad_spd) st |= ST_NOT_SPD;
  if (st) atomicOr(&a.status[id], st);
}

// Dynamic shared memory of a launch: the tiles at the class's largest grid and
// column count, and at least 58 KB, so that no more than three CTAs share an
// SM and their TMEM allocations (kTmemCols each of the SM's 512 columns) never
// wait on one another.
size_t tc_smem(int max_nx, int max_cols) {
  const int np = (max_nx + kPanel - 1) / kPanel * kPanel;
  const int cp8 = (max_cols + 7) & ~7;
  const int nbf = (std::max(cp8 * np, 2 * 16 * np + 16 * 16) + 31) & ~31;
  const size_t need = sizeof(float) * (2 * kTcRows * kTcRows + 2 * (size_t)nbf + 3 * kTcRows);
  return std::max(need, (size_t)58 * 1024);
}

}  // namespace

bool basis_tc_supported(int max_nx, int max_cols) {
  return max_nx <= kTcRows && ((max_cols + 7) & ~7) <= (int)kTmemCols;
}

cudaError_t basis_tc_ctas(int max_nx, int max_cols, int* ctas) {
  *ctas = 0;
  if (!basis_tc_supported(max_nx, max_cols)) return cudaErrorInvalidValue;
  const size_t smem = tc_smem(max_nx, max_cols);
  cudaError_t e = cudaFuncSetAttribute(basis_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, basis_tc_kernel, kTcThreads, smem);
  // every resident CTA holds kTmemCols of the SM's 512 TMEM columns (the
  // shared-memory floor of tc_smem keeps residency below that bound)
  if (e == cudaSuccess && *ctas > (int)(512 / kTmemCols)) *ctas = 512 / kTmemCols;
  return e;
}

cudaError_t launch_basis_tc(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st) {
  if (!basis_tc_supported(max_nx, max_cols) || !a.gmaps) return cudaErrorInvalidValue;
  const size_t smem = tc_smem(max_nx, max_cols);
  cudaError_t e = cudaFuncSetAttribute(basis_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  basis_tc_kernel<<<a.n_items, kTcThreads, smem, st>>>(a, refine);
  return cudaGetLastError();
}

}  // namespace sfb
