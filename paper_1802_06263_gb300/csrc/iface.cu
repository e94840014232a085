// Main loop of Method S3 (Section 5.4, Steps 3-6) for a batch of global
// collocation points, all on the device:
//  Step 4  kmap_kernel: global -> local index of every point in every KL
//          region (projection of y onto the region's dims, looked up in an
//          open-addressing table of the local realizations);
//          group_kernel: points of each subdomain grouped by local index
//          (stable), cut into tiles that share one stored basis Phi_i^k;
//  Step 5  CG on S^l = sum_i R_i^T Phi_i^{k_i(l)} R_i (Eq. 5.10), all points in
//          lockstep: matvec_kernel applies each stored basis to the tile of
//          points that use it, update_kernel assembles q = S p per point from
//          the per-subdomain products and does the CG update with
//          warp-shuffle dot products;
//  Step 6  recovery u = u*(lambda) + u_bar and the collocation-weighted
//          moments: darcy_moments_kernel / stokes_moments_kernel accumulate
//          sum w (x - shift) and sum w (x - shift)^2 per field entry in a
//          fixed order (deterministic, no atomics on floating point).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "sfb_ctx.h"

namespace sfb {

namespace {

constexpr int kTP = 8;   // points per moments sub-tile
constexpr int kTG = 32;  // points per group tile (CG products, moments tiles)

__host__ __device__ inline uint64_t mix_key(uint64_t h, int64_t v) {
  h ^= (uint64_t)v;
  h *= 1099511628211ull;
  return h;
}
__host__ __device__ inline uint64_t fin_key(uint64_t h) { return h ^ (h >> 29); }
__device__ inline int64_t qkey_dev(double v) {
  const double r = v * 1e12;
  return (int64_t)(r < 0 ? r - 0.5 : r + 0.5);
}

__global__ void kmap_kernel(const double* y, int64_t n_pts, int n_dim, const SubDev* subs, int ns,
                            const int* dim_off, const double* yloc, const int* hash, const int64_t* hash_off,
                            const int* hash_cap, int* kmap, int* pstat) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_pts * ns;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / ns;
    const int s = (int)(e - l * ns);
    const int nt = subs[s].n_term;
    const double* yl = y + l * n_dim + dim_off[s];
    uint64_t h = 1469598103934665603ull;
    for (int j = 0; j < nt; ++j) h = mix_key(h, qkey_dev(yl[j]));
    h = fin_key(h);
    const int cap = hash_cap[s];
    const int* tab = hash + hash_off[s];
    int found = -1;
    for (int probe = 0; probe < cap; ++probe) {
      const int slot = (int)((h + probe) & (uint64_t)(cap - 1));
      const int k = tab[slot];
      if (k < 0) break;
      const double* cand = yloc + subs[s].yloc_off + (int64_t)k * nt;
      bool eq = true;
      for (int j = 0; j < nt; ++j) eq = eq && (qkey_dev(cand[j]) == qkey_dev(yl[j]));
      if (eq) { found = k; break; }
    }
    kmap[l * ns + s] = found;
    if (found < 0) atomicOr(&pstat[l], 0x40000000);
  }
}

// One CTA per Darcy subdomain: histogram, scan, stable scatter, tiles.
__global__ void __launch_bounds__(256) group_kernel(const int* kmap, int64_t n_pts, int ns, const SubDev* subs,
                                                    const int64_t* loc_off, int* grp_count, int* grp_start,
                                                    int* grp_pts, int64_t pts_ld, int* tiles, int max_tiles,
                                                    int* n_tiles) {
  const int s = blockIdx.x;
  const int nl = subs[s].n_local;
  int* cnt = grp_count + loc_off[s];
  int* start = grp_start + loc_off[s];
  int* pts = grp_pts + (int64_t)s * pts_ld;
  for (int k = threadIdx.x; k < nl; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  for (int64_t l = threadIdx.x; l < n_pts; l += blockDim.x) {
    const int k = kmap[l * ns + s];
    if (k >= 0) atomicAdd(&cnt[k], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < nl; ++k) { start[k] = acc; acc += cnt[k]; cnt[k] = start[k]; }
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // stable scatter by one warp, 32 points at a time
    const int lane = threadIdx.x;
    for (int64_t base = 0; base < n_pts; base += 32) {
      const int64_t l = base + lane;
      const int k = l < n_pts ? kmap[l * ns + s] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, k);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int pos = 0;
      if (k >= 0) pos = cnt[k];
      __syncwarp();
      if (k >= 0) {
        pts[pos + rank] = (int)l;
        if (rank == 0) cnt[k] = pos + __popc(peers);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nt_ = 0;
    for (int k = 0; k < nl; ++k) {
      const int c0 = start[k], c1 = cnt[k];  // cnt now holds the end of group k
      for (int q = c0; q < c1 && nt_ < max_tiles; q += kTG) {
        tiles[3 * ((int64_t)s * max_tiles + nt_) + 0] = k;
        tiles[3 * ((int64_t)s * max_tiles + nt_) + 1] = q;
        tiles[3 * ((int64_t)s * max_tiles + nt_) + 2] = min(kTG, c1 - q);
        ++nt_;
      }
    }
    n_tiles[s] = nt_;
  }
}

// Stokes unit: one group holding every point in order.
__global__ void stokes_group_kernel(int64_t n_pts, int unit, int* grp_pts, int64_t pts_ld, int* tiles,
                                    int max_tiles, int* n_tiles) {
  int* pts = grp_pts + (int64_t)unit * pts_ld;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_pts; l += (int64_t)gridDim.x * blockDim.x)
    pts[l] = (int)l;
  const int nt_ = (int)((n_pts + kTG - 1) / kTG);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt_ && t < max_tiles; t += gridDim.x * blockDim.x) {
    tiles[3 * ((int64_t)unit * max_tiles + t) + 0] = 0;
    tiles[3 * ((int64_t)unit * max_tiles + t) + 1] = t * kTG;
    tiles[3 * ((int64_t)unit * max_tiles + t) + 2] = (int)(n_pts - (int64_t)t * kTG < kTG ? n_pts - (int64_t)t * kTG : kTG);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) n_tiles[unit] = min(nt_, max_tiles);
}

struct IfaceArgs {
  const SubDev* subs;
  int ns;               // Darcy subdomains; unit ns is the Stokes subdomain
  const ItemOff* off;
  const double* phi;    // Darcy basis store
  const double* s_phi;  // Stokes basis
  const float* phi32;   // the same, rounded to FP32 (operator of the mixed CG)
  const float* s_phi32;
  int Rs;
  const int64_t* gdof;  // Darcy local -> global
  const int64_t* sgdof; // Stokes local -> global
  const int64_t* ybase; // per unit offset into a point's Y row
  int64_t NY;
  const int* ldof;      // per global DOF: unit_a, local_a, unit_b, local_b
  const int* yoff;      // per global DOF: ybase[unit_a] + local_a, ybase[unit_b] + local_b
  int64_t n_lambda;
  const int* kmap;
  const int* grp_pts;
  int64_t pts_ld;
  const int* tiles;
  int max_tiles;
  const int* n_tiles;
  double* lam;
  double* r;
  double* p;
  double* Y;
  double* rr;
  double* gn;
  double* rlast;        // mixed CG: norm of the last FP64 residual
  int* rflag;           // mixed CG: FP64 residual due at the next check
  double* dinv;         // Jacobi preconditioner: 1 / diag(S^l) per point, or null (plain CG)
  // interface block-Jacobi preconditioner (when minv is set, it replaces dinv):
  // per point and mortar interface e the inverse of the diagonal block of S^l on
  // e's DOFs [if_off[e], if_off[e] + if_n[e]), FP32, at minv + l * minv_ld + if_moff[e]
  float* minv;
  int64_t minv_ld;
  int n_if;
  const int* if_off;
  const int* if_n;
  const int* if_moff;
  const int* dof_if;    // per global DOF: its interface
  // balancing preconditioner: when set, the tile products scale their inputs
  // and outputs by the unit's weights at its local DOFs ([n_pts][NY], the
  // layout of Y), so that they form D_u Phi_u^+ D_u R_u v
  const double* wy = nullptr;
  int* pstat;
  int64_t n_pts;
};

__device__ __forceinline__ const double* unit_phi(const IfaceArgs& a, int u, int k, int& R) {
  if (u == a.ns) { R = a.Rs; return a.s_phi; }
  const SubDev& S = a.subs[u];
  R = S.R;
  return a.phi + a.off[S.item0 + k].phi;
}

template <typename T>
__device__ __forceinline__ const T* unit_phi_t(const IfaceArgs& a, int u, int k, int& R);
template <>
__device__ __forceinline__ const double* unit_phi_t<double>(const IfaceArgs& a, int u, int k, int& R) {
  return unit_phi(a, u, k, R);
}
template <>
__device__ __forceinline__ const float* unit_phi_t<float>(const IfaceArgs& a, int u, int k, int& R) {
  if (u == a.ns) { R = a.Rs; return a.s_phi32; }
  const SubDev& S = a.subs[u];
  R = S.R;
  return a.phi32 + a.off[S.item0 + k].phi;
}

// Point states (pstat): 0 iterating; it > 0 converged after `it` iterations;
// -it stopped without convergence; kBadIdx a global point whose projection is
// not a local realization. The mixed CG pauses a point (kPending | it, plus
// kRestart after a breakdown p.Sp <= 0) until its next FP64 residual.
constexpr int kRestart = 0x10000000;
constexpr int kPending = 0x20000000;
constexpr int kBadIdx = 0x40000000;
constexpr int kItMask = 0x0fffffff;
__device__ __forceinline__ bool is_pending(int s) { return (s & (kPending | kBadIdx)) == kPending; }
// Point selection of a product: 0 iterating points; 1 points due for an FP64
// residual (paused, or iterating with the replacement flag set).
__device__ __forceinline__ bool selected(const IfaceArgs& a, int64_t l, int s, int sel) {
  return sel == 0 ? s == 0 : (is_pending(s) || (s == 0 && a.rflag[l]));
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = g = sum_i R_i^T g_i^{k_i(l)}, p = r, lambda = 0; one warp per point.
constexpr int kBlkMax = 32;   // largest interface block of the block-Jacobi preconditioner

// One warp per (point, interface): the interface's diagonal block of S^l,
// B[i][j] = sum over the two units sharing the interface of their basis
// entries (summed in FP64), inverted in FP32 by the symmetric sweep with one
// column per lane (the pivot column by shuffles) and stored in FP32. A
// preconditioner needs no more than FP32, and an FP64 sweep would make this
// kernel FP64-bound (about 2 ms on 2,049 points x 10 interfaces).
__global__ void bjacobi_setup_kernel(IfaceArgs a) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t l = wid / a.n_if;
  const int e = (int)(wid - l * a.n_if);
  if (l >= a.n_pts) return;
  if (a.pstat[l] & kBadIdx) return;
  const int n = a.if_n[e], d0 = a.if_off[e];
  float col[kBlkMax];
#pragma unroll
  for (int i = 0; i < kBlkMax; ++i) {
    double v = 0.0;
    if (lane < n && i < n) {
      const int di = d0 + i, dj = d0 + lane;
      for (int side = 0; side < 2; ++side) {
        const int u = a.ldof[4 * di + 2 * side], li = a.ldof[4 * di + 2 * side + 1];
        const int lj = a.ldof[4 * dj + 2 * side + 1];
        const int k = u < a.ns ? a.kmap[l * a.ns + u] : 0;
        int R;
        const double* ph = unit_phi(a, u, k, R);
        v += ph[li * R + lj];
      }
    } else if (i == lane) {
      v = 1.0;   // identity outside the block
    }
    col[i] = f64_to_f32_bits(v);
  }
#pragma unroll
  for (int kk = 0; kk < kBlkMax; ++kk) {
    if (kk >= n) break;
    float piv = __shfl_sync(0xffffffffu, col[kk], kk);
    if (!(piv > 0.f)) piv = 1.f;
    const float inv = 1.f / piv;
    const float rowk = col[kk];
#pragma unroll
    for (int i = 0; i < kBlkMax; ++i) {
      const float colk = __shfl_sync(0xffffffffu, col[i], kk);
      float v;
      if (i == kk) v = lane == kk ? -inv : rowk * inv;
      else v = lane == kk ? colk * inv : fmaf(-colk, rowk * inv, col[i]);
      col[i] = v;
    }
  }
  // stored column-major: entry (i, j) of the inverse at j * n + i, so that
  // the lanes of an apply, which take consecutive rows i, read consecutive
  // words for each j
  if (lane < n) {
    float* M = a.minv + l * a.minv_ld + a.if_moff[e];
#pragma unroll
    for (int i = 0; i < kBlkMax; ++i)
      if (i < n) M[lane * n + i] = -col[i];
  }
}

// z = M^{-1} r for the DOFs d = lane + 32 j of one point (warp-wide): r is
// staged in FP32 in the warp's shared buffer stage[n_lambda]; returns z_d.
__device__ __forceinline__ double bjacobi_apply(const IfaceArgs& a, int64_t l, const float* stage, int d) {
  const int e = a.dof_if[d];
  const int n = a.if_n[e], d0 = a.if_off[e], i = d - d0;
  const float* M = a.minv + l * a.minv_ld + a.if_moff[e] + i;   // column-major
  float z = 0.f;
  for (int j = 0; j < n; ++j) z = fmaf(M[j * n], stage[d0 + j], z);
  return f32_to_f64_bits(z);
}

// With the Jacobi preconditioner dinv = 1 / diag(S^l), z = dinv r, p = z and
// rr holds r.z; without it z = r and rr = r.r.
__global__ void init_kernel(IfaceArgs a) {
  extern __shared__ float stage_all[];   // [warps][n_lambda] (block preconditioner)
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= a.n_pts) return;
  float* stage = stage_all + (threadIdx.x >> 5) * a.n_lambda;
  double s2 = 0.0, rz = 0.0;
  for (int64_t d = lane; d < a.n_lambda; d += 32) {
    double g = 0.0, dg = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int u = a.ldof[4 * d + 2 * side], loc = a.ldof[4 * d + 2 * side + 1];
      int R;
      const int k = u < a.ns ? a.kmap[l * a.ns + u] : 0;
      if (k < 0) continue;
      const double* ph = unit_phi(a, u, k, R);
      g += ph[R * R + loc];
      dg += ph[loc * R + loc];
    }
    double z = g;
    if (a.dinv) {
      const double di = dg > 0.0 ? 1.0 / dg : 1.0;
      a.dinv[l * a.n_lambda + d] = di;
      z = di * g;
    }
    if (a.minv) stage[d] = f64_to_f32_bits(g);
    a.r[l * a.n_lambda + d] = g;
    a.p[l * a.n_lambda + d] = z;
    a.lam[l * a.n_lambda + d] = 0.0;
    s2 += g * g;
    rz += g * z;
  }
  if (a.minv) {   // z = M^{-1} g with the interface blocks
    __syncwarp();
    rz = 0.0;
    for (int64_t d = lane; d < a.n_lambda; d += 32) {
      const double z = bjacobi_apply(a, l, stage, (int)d);
      a.p[l * a.n_lambda + d] = z;
      rz += a.r[l * a.n_lambda + d] * z;
    }
  }
  s2 = warp_sum(s2);
  rz = warp_sum(rz);
  if (lane == 0) {
    a.rr[l] = rz;
    a.gn[l] = sqrt(s2);
    a.rlast[l] = sqrt(s2);
    a.rflag[l] = 0;
    int st = a.pstat[l] & 0x40000000;  // keep a bad-index mark
    if (!st && s2 == 0.0) st = 1;       // zero data: converged with lambda = 0
    a.pstat[l] = st;
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Y[l][ybase_u + :] = Phi_u^k (R_u v_l) for the selected points of one tile
// of up to kTG points that share the stored basis Phi_u^k. Phi arrives in
// shared memory by one bulk copy (mbarrier completion, bounded wait); the
// product runs in T (FP64, or FP32 on the rounded copy of Phi for the inner
// products of the mixed CG) with 2 x 4 register tiles (two rows of Phi, four
// points). The bulk copy rounds R*R*sizeof(T) up to 16 bytes; the extra bytes
// lie inside the same item (its g block follows Phi). The steps below serve
// matvec_kernel (one CTA per tile) and the persistent CG kernel (each CTA
// walks a strided share of all tiles) alike.
struct TileScratch {
  int sidx[kTG];        // tile slots of the selected points, in order
  int nsel;
  int64_t spt[kTG];     // the selected points' indices
  int sgd[kMaxCols];    // the unit's global DOFs
};

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One thread: `bytes` of a basis into dst, completing on bar. The proxy fence
// orders earlier generic reads of dst before the asynchronous write.
__device__ __forceinline__ void phi_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Bounded wait for the phase of bar with the given parity; false after the limit.
__device__ __forceinline__ bool phi_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok = 0;
  for (int it = 0; it < (1 << 22) && !ok; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
  return ok != 0;
}

// The tile's selected points (a block-uniform count; every thread calls it).
__device__ __forceinline__ int tile_select(const IfaceArgs& a, const int* pts, int cntp, int sel, TileScratch& ts) {
  const int act = threadIdx.x < cntp ? selected(a, pts[threadIdx.x], a.pstat[pts[threadIdx.x]], sel) : 0;
  if (threadIdx.x < 32) {     // kTG == 32: warp 0 holds one slot per lane
    const unsigned mask = __ballot_sync(0xffffffffu, act);
    if (act) ts.sidx[__popc(mask & ((1u << threadIdx.x) - 1u))] = threadIdx.x;
    if (threadIdx.x == 0) ts.nsel = __popc(mask);
  }
  if (!__syncthreads_or(act)) return 0;
  return ts.nsel;
}

// Pv[i][q] = v_{l_q}[gdof_u(i)] in T for the nsel selected points, padded to
// a multiple of 4 points with zeros; the points' indices and the unit's global
// DOFs are staged once so that each gathered entry is one dependent load.
template <typename T>
__device__ __forceinline__ void tile_gather(const IfaceArgs& a, const double* __restrict__ vin, const int* pts, int u,
                                            int R, int nsel, TileScratch& ts, T* Pv) {
  const int64_t* gd = u == a.ns ? a.sgdof : a.gdof + a.subs[u].gdof_off;
  if (threadIdx.x < nsel) ts.spt[threadIdx.x] = pts[ts.sidx[threadIdx.x]];
  for (int i = threadIdx.x; i < R; i += blockDim.x) ts.sgd[i] = (int)gd[i];
  __syncthreads();
  const int nsel4 = (nsel + 3) & ~3;
  for (int e = threadIdx.x; e < nsel4 * R; e += blockDim.x) {
    const int q = e / R, i = e - q * R;
    double v = 0.0;
    if (q < nsel) {
      v = vin[ts.spt[q] * a.n_lambda + ts.sgd[i]];
      if (a.wy) v *= a.wy[ts.spt[q] * a.NY + a.ybase[u] + i];
    }
    Pv[i * (kTG + 1) + q] = from_f64<T>(v);
  }
}

// Y rows of the selected points = Ph Pv.
template <typename T>
__device__ __forceinline__ void tile_product(const IfaceArgs& a, int u, int R, int nsel, const TileScratch& ts,
                                             const T* Ph, const T* Pv) {
  const int nsel4 = (nsel + 3) & ~3;
  const int nrp = (R + 1) >> 1;
  const int ncg = nsel4 >> 2;
  for (int tt = threadIdx.x; tt < nrp * ncg; tt += blockDim.x) {
    const int r0 = (tt / ncg) * 2, c0 = (tt % ncg) * 4;
    const bool two = r0 + 1 < R;
    T acc[2][4] = {};
    const T* p0 = Ph + r0 * R;
    const T* p1 = Ph + (two ? r0 + 1 : r0) * R;
    for (int j = 0; j < R; ++j) {
      const T f0 = p0[j], f1 = p1[j];
      const T* v = Pv + j * (kTG + 1) + c0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[0][q] = fma(f0, v[q], acc[0][q]);
        acc[1][q] = fma(f1, v[q], acc[1][q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (c0 + q >= nsel) break;
      double* y = a.Y + ts.spt[c0 + q] * a.NY + a.ybase[u];
      if (a.wy) {
        const double* wq = a.wy + ts.spt[c0 + q] * a.NY + a.ybase[u];
        y[r0] = wq[r0] * to_f64(acc[0][q]);
        if (two) y[r0 + 1] = wq[r0 + 1] * to_f64(acc[1][q]);
      } else {
        y[r0] = to_f64(acc[0][q]);
        if (two) y[r0 + 1] = to_f64(acc[1][q]);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) matvec_kernel(IfaceArgs a, const double* __restrict__ vin, int sel,
                                                     int* err, int u0) {
  extern __shared__ __align__(16) unsigned char smv_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ TileScratch ts;
  const int u = u0 + blockIdx.y;   // units u0, u0 + 1, ...
  const int t = blockIdx.x;
  if (t >= a.n_tiles[u]) return;
  const int* tl = a.tiles + 3 * ((int64_t)u * a.max_tiles + t);
  const int k = tl[0], q0 = tl[1], cntp = tl[2];
  const int* pts = a.grp_pts + (int64_t)u * a.pts_ld + q0;
  const int nsel = tile_select(a, pts, cntp, sel, ts);
  if (nsel == 0) return;   // no point of the tile is selected
  int R;
  const T* ph = unit_phi_t<T>(a, u, k, R);
  const int rr4 = (R * R + 3) & ~3;
  T* Ph = reinterpret_cast<T*>(smv_raw);   // [R][R]
  T* Pv = Ph + rr4;                        // [R][kTG + 1]
  const uint32_t bytes = (uint32_t)((R * R * (int)sizeof(T) + 15) & ~15);
  if (threadIdx.x == 0) {
    mbar_init1(&bar);
    phi_load(Ph, ph, bytes, &bar);
  }
  tile_gather<T>(a, vin, pts, u, R, nsel, ts, Pv);   // its barrier publishes the initialised mbarrier
  const bool ok = phi_wait(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(err, 1);
      phi_wait(&bar, 0);   // a bounded second chance for the copy in flight before the CTA exits
    }
    __syncthreads();
    return;
  }
  tile_product<T>(a, u, R, nsel, ts, Ph, Pv);
}

// q = S p from the per-unit products, then the CG update; one warp per point.
// Mixed CG (products from the FP32 bases): once the recursive residual falls
// below replace_ratio times the last FP64 residual the point asks for an FP64
// residual at the next check and keeps iterating; it pauses when it falls
// below pause_ratio times that residual, or below the tolerance, so that the
// recursive and the true residual never drift far apart before replacement.
constexpr int kUpd = 8;   // DOFs per lane held in registers by the update (n_lambda <= 256)

// The update of point l by its warp; stage is the warp's FP32 buffer of
// n_lambda entries (block preconditioner).
template <bool kRegs>
__device__ __forceinline__ void update_point(const IfaceArgs& a, int64_t l, int lane, float* stage, int it,
                                             double rtol, int mixed, double replace_ratio, double pause_ratio) {
  if (a.pstat[l] != 0) return;
  const double* Yl = a.Y + l * a.NY;
  double* pl = a.p + l * a.n_lambda;
  double* rl = a.r + l * a.n_lambda;
  double* ll = a.lam + l * a.n_lambda;
  const int n = (int)a.n_lambda;
  // q = S p on this lane's DOFs (kept in registers when n <= 32 kUpd)
  double qv[kRegs ? kUpd : 1], pv[kRegs ? kUpd : 1];
  double pq = 0.0;
  if (kRegs) {
#pragma unroll
    for (int j = 0; j < kUpd; ++j) {
      const int d = lane + 32 * j;
      qv[j] = 0.0;
      pv[j] = 0.0;
      if (d < n) {
        qv[j] = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]];
        pv[j] = pl[d];
        pq = fma(pv[j], qv[j], pq);
      }
    }
  } else {
    for (int d = lane; d < n; d += 32) pq += pl[d] * (Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]]);
  }
  pq = warp_sum(pq);
  const double rr = a.rr[l];
  const bool brk = !(pq > 0.0);
  // scalar FP64 divisions and roots once per point (lane 0), then broadcast:
  // on this part FP64 issues at 1/64 of the FP32 rate
  double alpha = 0.0;
  if (lane == 0 && !brk) alpha = rr / pq;
  alpha = __shfl_sync(0xffffffffu, alpha, 0);
  // rn = r.r (stopping test), rz = r.z with z = dinv r (= rn without preconditioner)
  double rn = 0.0, rz = 0.0;
  const double* dl = a.dinv ? a.dinv + l * a.n_lambda : nullptr;
  double rv_keep[kRegs ? kUpd : 1];
  if (kRegs) {
#pragma unroll
    for (int j = 0; j < kUpd; ++j) {
      const int d = lane + 32 * j;
      rv_keep[j] = 0.0;
      if (d < n) {
        ll[d] = fma(alpha, pv[j], ll[d]);
        const double rv = fma(-alpha, qv[j], rl[d]);
        rl[d] = rv;
        rn = fma(rv, rv, rn);
        if (a.minv) {
          stage[d] = f64_to_f32_bits(rv);
          rv_keep[j] = rv;
        } else {
          const double zv = dl ? dl[d] * rv : rv;
          rv_keep[j] = zv;
          rz = fma(rv, zv, rz);
        }
      }
    }
    if (a.minv) {   // z = M^{-1} r with the interface blocks (r staged in FP32)
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kUpd; ++j) {
        const int d = lane + 32 * j;
        if (d < n) {
          const double zv = bjacobi_apply(a, l, stage, d);
          rz = fma(rv_keep[j], zv, rz);
          rv_keep[j] = zv;
        }
      }
    }
  } else {
    for (int d = lane; d < n; d += 32) {
      const double q = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]];
      ll[d] += alpha * pl[d];
      const double rv = rl[d] - alpha * q;
      rl[d] = rv;
      rn += rv * rv;
      if (a.minv) stage[d] = f64_to_f32_bits(rv);
      else rz += rv * (dl ? dl[d] * rv : rv);
    }
    if (a.minv) {
      __syncwarp();
      for (int d = lane; d < n; d += 32) rz += rl[d] * bjacobi_apply(a, l, stage, d);
    }
  }
  rn = warp_sum(rn);
  rz = (dl || a.minv) ? warp_sum(rz) : rn;
  int dec = 0;   // bit 0 done, bit 1 pause, bit 2 flag
  double beta = 0.0;
  if (lane == 0) {
    const double rnorm = sqrt(rn);
    if (mixed) {
      dec |= (brk || rnorm <= fmax(rtol * a.gn[l], pause_ratio * a.rlast[l])) ? 2 : 0;
      dec |= rnorm <= replace_ratio * a.rlast[l] ? 4 : 0;
    } else {
      dec |= (rnorm <= rtol * a.gn[l] || brk) ? 1 : 0;
    }
    if (!(dec & 1) && !brk) beta = rz / rr;
  }
  dec = __shfl_sync(0xffffffffu, dec, 0);
  beta = __shfl_sync(0xffffffffu, beta, 0);
  const bool done = dec & 1, pause = dec & 2, flag = dec & 4;
  if (!done && !brk) {
    if (kRegs) {
#pragma unroll
      for (int j = 0; j < kUpd; ++j) {
        const int d = lane + 32 * j;
        if (d < n) pl[d] = fma(beta, pv[j], rv_keep[j]);
      }
    } else {
      for (int d = lane; d < n; d += 32)
        pl[d] = (a.minv ? bjacobi_apply(a, l, stage, d) : (dl ? dl[d] * rl[d] : rl[d])) + beta * pl[d];
    }
  }
  __syncwarp();
  if (lane == 0) {
    a.rr[l] = rz;
    if (done) a.pstat[l] = brk ? -(it + 1) : it + 1;
    else if (pause) a.pstat[l] = kPending | (brk ? kRestart : 0) | (it + 1);
    else if (flag) a.rflag[l] = 1;
  }
}

template <bool kRegs>
__global__ void update_kernel(IfaceArgs a, int it, double rtol, int mixed, double replace_ratio,
                              double pause_ratio) {
  extern __shared__ float stage_all[];   // [warps][n_lambda] (block preconditioner)
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (l >= a.n_pts) return;
  update_point<kRegs>(a, l, threadIdx.x & 31, stage_all + (threadIdx.x >> 5) * a.n_lambda, it, rtol, mixed,
                      replace_ratio, pause_ratio);
}

// FP64 residual replacement of the mixed CG, one warp per point due (paused
// or flagged), on the FP64 products Y = Phi (R lambda): r = g - S lambda. The
// point has converged if ||r|| <= rtol ||g||; otherwise it continues from the
// replaced residual with the same direction p (p = r after a breakdown).
__device__ __forceinline__ void reliable_point(const IfaceArgs& a, int64_t l, int lane, float* stage, double rtol,
                                               int it) {
  const int s = a.pstat[l];
  if (!selected(a, l, s, 1)) return;
  const double* Yl = a.Y + l * a.NY;
  double* rl = a.r + l * a.n_lambda;
  double rn = 0.0, rz = 0.0;
  for (int64_t d = lane; d < a.n_lambda; d += 32) {
    double g = 0.0, q = 0.0;
    for (int side = 0; side < 2; ++side) {
      const int u = a.ldof[4 * d + 2 * side], loc = a.ldof[4 * d + 2 * side + 1];
      const int k = u < a.ns ? a.kmap[l * a.ns + u] : 0;
      int R;
      const double* ph = unit_phi(a, u, k, R);
      g += ph[R * R + loc];
      q += Yl[a.ybase[u] + loc];
    }
    const double rv = g - q;
    rl[d] = rv;
    rn += rv * rv;
    if (a.minv) stage[d] = f64_to_f32_bits(rv);
    else rz += rv * (a.dinv ? a.dinv[l * a.n_lambda + d] * rv : rv);
  }
  if (a.minv) {
    __syncwarp();
    for (int64_t d = lane; d < a.n_lambda; d += 32) rz += rl[d] * bjacobi_apply(a, l, stage, (int)d);
  }
  rn = warp_sum(rn);
  rz = warp_sum(rz);
  const bool conv = sqrt(rn) <= rtol * a.gn[l];
  if (!conv && (s & kRestart)) {
    double* pl = a.p + l * a.n_lambda;
    for (int64_t d = lane; d < a.n_lambda; d += 32)
      pl[d] = a.minv ? bjacobi_apply(a, l, stage, (int)d) : (a.dinv ? a.dinv[l * a.n_lambda + d] * rl[d] : rl[d]);
  }
  __syncwarp();
  if (lane == 0) {
    a.rflag[l] = 0;
    a.rr[l] = rz;
    a.rlast[l] = sqrt(rn);
    a.pstat[l] = conv ? (s != 0 ? (s & kItMask) : it) : 0;
  }
}

__global__ void reliable_kernel(IfaceArgs a, double rtol, int it) {
  extern __shared__ float stage_all[];   // [warps][n_lambda] (block preconditioner)
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (l >= a.n_pts) return;
  reliable_point(a, l, threadIdx.x & 31, stage_all + (threadIdx.x >> 5) * a.n_lambda, rtol, it);
}

// ---- restarted GMRES ------------------------------------------------------------------
// GMRES(m) for every point's S^l lambda = g^l (Section 5.4 Step 5 names CG or
// GMRES for the interface problem), one warp per point, all points in
// lockstep like the CG. Right preconditioning with the CG's preconditioner M
// (none, Jacobi, or the interface blocks, whose FP32 inverses are applied here
// in FP64 arithmetic so that M^{-1} is one fixed linear map): the Arnoldi
// process runs on S M^{-1}, its residual is that of the unpreconditioned
// system, and lambda = M^{-1} u. Orthogonalization is classical Gram-Schmidt
// with one re-orthogonalization pass (each pass: all the cycle's dot products
// in one sweep over the DOFs, then one update sweep). Givens rotations keep
// the least-squares residual |gv[j+1]|; at the end of a cycle (that residual
// at rtol ||g||, m steps, or a breakdown) the warp solves the triangular
// system, adds M^{-1} V y to lambda and marks the point for the FP64 true
// residual g - S lambda, which either accepts it or starts the next cycle.
struct GmArgs {
  double* V;    // [kGmresMax + 1][n_pts][n_lambda]: Krylov basis
  double* st;   // [n_pts][kGmresState]: Hessenberg columns, rotations, rotated right-hand side
  int* j;       // [n_pts]: steps taken in the current cycle
  int m;        // restart length (<= kGmresMax)
  double cycle_tol;   // > 0: a cycle also ends once it has reduced its initial residual by this factor
};
// the state's last slot: the residual norm a cycle started from
constexpr int kGmBeta = kGmresState - 1;
// a point's state: column k of H (entries 0..k+1) at k * (kGmresMax + 1), then
// the cosines, the sines and the rotated right-hand side
__device__ __forceinline__ double* gm_col(const GmArgs& g, int64_t l, int k) {
  return g.st + l * kGmresState + k * (kGmresMax + 1);
}
__device__ __forceinline__ double* gm_cs(const GmArgs& g, int64_t l) {
  return g.st + l * kGmresState + kGmresMax * (kGmresMax + 1);
}
__device__ __forceinline__ double* gm_sn(const GmArgs& g, int64_t l) { return gm_cs(g, l) + kGmresMax; }
__device__ __forceinline__ double* gm_gv(const GmArgs& g, int64_t l) { return gm_cs(g, l) + 2 * kGmresMax; }
__device__ __forceinline__ double* gm_v(const GmArgs& g, const IfaceArgs& a, int i, int64_t l) {
  return g.V + ((int64_t)i * a.n_pts + l) * a.n_lambda;
}
// The Krylov basis in the Arnoldi precision VT: FP64 (GMRES) or FP32 (the
// mixed GMRES, whose cycles are the inner solver of an FP64 refinement: its
// orthogonalization then runs on the FP32 pipe, at 64 times the FP64 rate,
// and reads half the bytes). The FP32 basis occupies the front of the same
// buffer.
template <typename VT>
__device__ __forceinline__ VT* gm_vt(const GmArgs& g, const IfaceArgs& a, int i, int64_t l) {
  return reinterpret_cast<VT*>(g.V) + ((int64_t)i * a.n_pts + l) * a.n_lambda;
}
template <typename VT> __device__ __forceinline__ VT to_vt(double v);
template <> __device__ __forceinline__ double to_vt<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_vt<float>(double v) { return f64_to_f32_bits(v); }
__device__ __forceinline__ double vt_f64(double v) { return v; }
__device__ __forceinline__ double vt_f64(float v) { return f32_to_f64_bits(v); }

// (M^{-1} v)_d for point l with v in global memory, in FP64 arithmetic.
__device__ __forceinline__ double precond64(const IfaceArgs& a, int64_t l, const double* v, int d) {
  if (a.minv) {
    const int e = a.dof_if[d];
    const int n = a.if_n[e], d0 = a.if_off[e], i = d - d0;
    const float* M = a.minv + l * a.minv_ld + a.if_moff[e] + i;   // column-major
    double z = 0.0;
    for (int j = 0; j < n; ++j) z = fma(f32_to_f64_bits(M[j * n]), v[d0 + j], z);
    return z;
  }
  if (a.dinv) return a.dinv[l * a.n_lambda + d] * v[d];
  return v[d];
}

// (M^{-1} v)_d for the Krylov basis vector v in its own precision: FP64 as
// precond64, or for FP32 vectors with FP32 arithmetic (the block inverses are
// stored in FP32; the Jacobi factor rounded to FP32).
__device__ __forceinline__ double precond_t(const IfaceArgs& a, int64_t l, const double* v, int d) {
  return precond64(a, l, v, d);
}
__device__ __forceinline__ double precond_t(const IfaceArgs& a, int64_t l, const float* v, int d) {
  if (a.minv) {
    const int e = a.dof_if[d];
    const int n = a.if_n[e], d0 = a.if_off[e], i = d - d0;
    const float* M = a.minv + l * a.minv_ld + a.if_moff[e] + i;   // column-major
    float z = 0.f;
    for (int j = 0; j < n; ++j) z = fmaf(M[j * n], v[d0 + j], z);
    return f32_to_f64_bits(z);
  }
  if (a.dinv) return f32_to_f64_bits(f64_to_f32_bits(a.dinv[l * a.n_lambda + d]) * v[d]);
  return f32_to_f64_bits(v[d]);
}

// g_d of point l (the two units' flux data); with want_diag also the diagonal
// of S^l at d.
__device__ __forceinline__ double rhs_g(const IfaceArgs& a, int64_t l, int64_t d, double* diag) {
  double g = 0.0, dg = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int u = a.ldof[4 * d + 2 * side], loc = a.ldof[4 * d + 2 * side + 1];
    const int k = u < a.ns ? a.kmap[l * a.ns + u] : 0;
    if (k < 0) continue;
    int R;
    const double* ph = unit_phi(a, u, k, R);
    g += ph[R * R + loc];
    dg += ph[loc * R + loc];
  }
  if (diag) *diag = dg;
  return g;
}

// New cycle of point l from the residual r (global, n_lambda entries) of norm
// rn > 0: V_0 = r / rn, gv = (rn, 0, ...), j = 0, p = M^{-1} V_0.
template <typename VT>
__device__ __forceinline__ void gm_new_cycle(const IfaceArgs& a, const GmArgs& g, int64_t l, int lane,
                                             const double* r, double rn) {
  VT* v0 = gm_vt<VT>(g, a, 0, l);
  const double inv = 1.0 / rn;
  for (int64_t d = lane; d < a.n_lambda; d += 32) v0[d] = to_vt<VT>(r[d] * inv);
  double* gv = gm_gv(g, l);
  for (int i = lane; i <= kGmresMax; i += 32) gv[i] = i == 0 ? rn : 0.0;
  if (lane == 0) g.st[l * kGmresState + kGmBeta] = rn;
  __syncwarp();
  double* pl = a.p + l * a.n_lambda;
  for (int64_t d = lane; d < a.n_lambda; d += 32) pl[d] = precond_t(a, l, v0, (int)d);
  if (lane == 0) g.j[l] = 0;
}

// First cycle from lambda = 0: r = g, ||g||, the Jacobi diagonal when used.
template <typename VT>
__global__ void gmres_init_kernel(IfaceArgs a, GmArgs g) {
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= a.n_pts) return;
  double* rl = a.r + l * a.n_lambda;
  double s2 = 0.0;
  for (int64_t d = lane; d < a.n_lambda; d += 32) {
    double dg = 0.0;
    const double gd = rhs_g(a, l, d, &dg);
    if (a.dinv) a.dinv[l * a.n_lambda + d] = dg > 0.0 ? 1.0 / dg : 1.0;
    rl[d] = gd;
    a.lam[l * a.n_lambda + d] = 0.0;
    s2 = fma(gd, gd, s2);
  }
  s2 = warp_sum(s2);
  const double gn = sqrt(s2);
  int st = a.pstat[l] & kBadIdx;
  if (!st && s2 == 0.0) st = 1;   // zero data: converged with lambda = 0
  __syncwarp();
  if (st == 0) gm_new_cycle<VT>(a, g, l, lane, rl, gn);
  if (lane == 0) {
    a.gn[l] = gn;
    a.pstat[l] = st;
  }
}

// One Arnoldi step of every iterating point, on the products Y = S p of
// p = M^{-1} V_j: w = S M^{-1} V_j orthogonalized against V_0..V_j (two
// classical Gram-Schmidt passes), H column j, V_{j+1} = w / ||w||, the
// rotations, and at the end of the cycle the solution update.
// VT: the precision of the basis and of the Gram-Schmidt sums (FP64, or FP32
// for the mixed GMRES); the Hessenberg matrix, rotations and updates stay FP64.
template <typename VT>
__global__ void __launch_bounds__(256) gmres_arnoldi_kernel(IfaceArgs a, GmArgs g, int it, double rtol) {
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= a.n_pts) return;
  if (a.pstat[l] != 0) return;
  const int j = g.j[l];
  const int64_t n = a.n_lambda;
  const double* Yl = a.Y + l * a.NY;
  VT* w = reinterpret_cast<VT*>(a.r + l * n);   // the new direction (in r's storage)
  for (int64_t d = lane; d < n; d += 32) w[d] = to_vt<VT>(Yl[a.yoff[2 * d]]) + to_vt<VT>(Yl[a.yoff[2 * d + 1]]);
  __syncwarp();
  double* hcol = gm_col(g, l, j);
  // the warp's Gram-Schmidt coefficients (one basis vector at a time, so that
  // no thread holds the whole column: occupancy for the memory-bound sweeps)
  __shared__ double hsh[8][kGmresMax + 1];
  __shared__ VT hvsh[8][kGmresMax + 1];   // the same, in the basis precision
  double* hw = hsh[threadIdx.x >> 5];
  VT* hv = hvsh[threadIdx.x >> 5];
  // classical Gram-Schmidt, repeated only when the first pass cancelled more
  // than a factor 1/sqrt(2) of w (the criterion of Daniel, Gragg, Kaufman and
  // Stewart): one pass keeps orthogonality unless w was nearly in the span
  VT s2 = VT(0);
  for (int64_t d = lane; d < n; d += 32) s2 = fma(w[d], w[d], s2);
  const double w0 = sqrt(vt_f64(warp_sum(s2)));
  double hn = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i <= j; ++i) {
      const VT* vi = gm_vt<VT>(g, a, i, l);
      VT acc = VT(0);
      for (int64_t d = lane; d < n; d += 32) acc = fma(vi[d], w[d], acc);
      acc = warp_sum(acc);
      if (lane == 0) {
        hv[i] = acc;
        hcol[i] = pass == 0 ? vt_f64(acc) : hcol[i] + vt_f64(acc);
      }
    }
    __syncwarp();
    s2 = VT(0);
    for (int64_t d = lane; d < n; d += 32) {
      VT wd = w[d];
      for (int i = 0; i <= j; ++i) wd = fma(-hv[i], gm_vt<VT>(g, a, i, l)[d], wd);
      w[d] = wd;
      s2 = fma(wd, wd, s2);
    }
    hn = sqrt(vt_f64(warp_sum(s2)));
    __syncwarp();
    if (hn >= 0.70710678118654752 * w0) break;   // warp-uniform: every lane holds the sums
  }
  const bool brk = !(hn > 0.0);   // the Krylov space is invariant: the cycle's solution is exact
  if (!brk) {
    VT* vn = gm_vt<VT>(g, a, j + 1, l);
    const VT inv = to_vt<VT>(1.0 / hn);
    for (int64_t d = lane; d < n; d += 32) vn[d] = w[d] * inv;
  }
  // rotations (lane 0): the earlier ones on column j, then the one that
  // annihilates H[j+1][j]; the rotated right-hand side's last entry is the
  // least-squares residual of the cycle
  int end = 0;
  if (lane == 0) {
    double* cs = gm_cs(g, l);
    double* sn = gm_sn(g, l);
    double* gv = gm_gv(g, l);
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
      hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
      hcol[i] = t;
    }
    const double hjj = hcol[j];
    const double rho = hypot(hjj, hn);
    const double c = rho > 0.0 ? hjj / rho : 1.0, s = rho > 0.0 ? hn / rho : 0.0;
    cs[j] = c;
    sn[j] = s;
    hcol[j] = rho;
    hcol[j + 1] = 0.0;
    gv[j + 1] = -s * gv[j];
    gv[j] = c * gv[j];
    const double target = fmax(rtol * a.gn[l], g.cycle_tol * g.st[l * kGmresState + kGmBeta]);
    end = (fabs(gv[j + 1]) <= target || j + 1 >= g.m || brk) ? 1 : 0;
  }
  end = __shfl_sync(0xffffffffu, end, 0);
  __syncwarp();
  if (!end) {
    const VT* vn = gm_vt<VT>(g, a, j + 1, l);
    double* pl = a.p + l * n;
    for (int64_t d = lane; d < n; d += 32) pl[d] = precond_t(a, l, vn, (int)d);
    if (lane == 0) g.j[l] = j + 1;
    return;
  }
  // end of the cycle: H(0:jn, 0:jn) y = gv(0:jn) by back substitution (lane k
  // holds y_k), then lambda += M^{-1} (V y)
  const int jn = j + 1;
  const double* gv = gm_gv(g, l);
  double yk = 0.0;
  for (int i = jn - 1; i >= 0; --i) {
    double part = (lane > i && lane < jn) ? gm_col(g, l, lane)[i] * yk : 0.0;
    part = warp_sum(part);
    if (lane == i) yk = (gv[i] - part) / gm_col(g, l, i)[i];
  }
  if (lane < jn) hw[lane] = yk;
  __syncwarp();
  double* u = a.p + l * n;   // V y in FP64, in p's storage (no next direction)
  for (int64_t d = lane; d < n; d += 32) {
    double ud = 0.0;
    for (int i = 0; i < jn; ++i) ud = fma(hw[i], vt_f64(gm_vt<VT>(g, a, i, l)[d]), ud);
    u[d] = ud;
  }
  __syncwarp();
  double* ll = a.lam + l * n;
  for (int64_t d = lane; d < n; d += 32) ll[d] += precond64(a, l, u, (int)d);
  if (lane == 0) {
    g.j[l] = 0;
    a.pstat[l] = kPending | (it + 1);
  }
}

// The FP64 true residual r = g - S lambda of every point whose cycle ended,
// on the products Y = S lambda: accepted when ||r|| <= rtol ||g||, otherwise
// the next cycle starts from r.
template <typename VT>
__global__ void gmres_restart_kernel(IfaceArgs a, GmArgs g, double rtol) {
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= a.n_pts) return;
  const int s = a.pstat[l];
  if (!is_pending(s)) return;
  const double* Yl = a.Y + l * a.NY;
  double* rl = a.r + l * a.n_lambda;
  double s2 = 0.0;
  for (int64_t d = lane; d < a.n_lambda; d += 32) {
    const double rv = rhs_g(a, l, d, nullptr) - (Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]]);
    rl[d] = rv;
    s2 = fma(rv, rv, s2);
  }
  const double rn = sqrt(warp_sum(s2));
  __syncwarp();
  if (rn <= rtol * a.gn[l]) {
    if (lane == 0) a.pstat[l] = s & kItMask;
    return;
  }
  gm_new_cycle<VT>(a, g, l, lane, rl, rn);
  if (lane == 0) a.pstat[l] = 0;
}

__global__ void count_active(const int* pstat, int64_t n, int* out) {
  int c = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
    c += pstat[l] == 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void finish_status(int* pstat, int64_t n, int max_it, int* iters_out) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x) {
    int s = pstat[l];
    if (s == 0) s = -max_it;
    else if (s & (kBadIdx | kPending)) s = -max_it;
    pstat[l] = s;
    if (iters_out) iters_out[l] = s;
  }
}

// ---- persistent CG ----------------------------------------------------------------
// The whole CG of a batch in one cooperative launch. Every CTA takes a strided
// share of the product tiles, then a strided share of the points (one warp per
// point), with a grid barrier between the two; the checks of the launch-per-step
// loop (FP64 residuals of the mixed CG, the count of iterating points) come
// every `chunk` iterations as there. The per-point and per-tile arithmetic is
// the same code in the same order, so the results are identical; what goes are
// two launches per iteration and the host round trip per check. The grid holds
// no more CTAs than fit on the device at once (a cooperative launch checks
// it), so a CTA waiting at a barrier waits only for CTAs that are running.
struct PcgCtl {
  unsigned* bar;   // [0] arrivals, [1] generation; both zero at launch
  int* abort;      // set when a barrier or copy wait runs out; zero at launch
  int* act;        // [4] iterating-point counts, a ring over the checks; zero at launch
  int* iters;      // iterations run
  int* err;        // bit 0: a bulk copy of a basis did not complete within the wait limit
  unsigned long long* cyc;   // [6] SM cycles summed over the CTAs: tile products, barrier after them,
                             // updates, barrier after them, FP64 check products, the rest of the checks
  int test_skip;   // test hook: CTA 0 skips its first barrier, so that the other CTAs' waits run out
};
constexpr int kPcgUnits = 64;                                // units (subdomains + Stokes) it handles
constexpr unsigned long long kBarrierNs = 1000000000ull;     // 1 s, far above any CG step

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier, called by every thread of every CTA: one arrival counter (an
// acquire-release add by each CTA's thread 0 after the CTA's barrier), the
// release by a generation number (counted by every thread in gen) that the last
// arrival stores with release semantics and the others load with acquire
// semantics. A wait ends after kBarrierNs, or when another CTA has set abort.
// False, for the whole CTA, once abort is set.
__device__ bool grid_sync(const PcgCtl& c, unsigned& gen) {
  __shared__ int ok_s;
  __syncthreads();
  const unsigned target = gen + 1;   // every thread counts the barriers: the branches below are block-uniform
  gen = target;
  if (c.test_skip && blockIdx.x == 0 && target == 1) return true;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (atom_add_acq_rel(&c.bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&c.bar[0], 0u);
      st_release(&c.bar[1], target);
    } else {
      // a tight spin on the release flag first; the abort flag and the clock
      // are read every 32 polls, and the spin backs off to short sleeps only
      // after a few hundred polls
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (ld_acquire(&c.bar[1]) != target) {
        if ((++polls & 31u) == 0) {
          if (*((volatile int*)c.abort)) { ok = 0; break; }
          if (global_ns() - t0 > kBarrierNs) {
            atomicExch(c.abort, 1);
            ok = 0;
            break;
          }
        }
        if (polls > 512) __nanosleep(32);
      }
    }
    if (*((volatile int*)c.abort)) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Tile f of the flat list: unit u with tpre[u] <= f < tpre[u + 1], tile t.
__device__ __forceinline__ void tile_locate(const int* tpre, int f, int& u, int& t) {
  u = 0;
  while (tpre[u + 1] <= f) ++u;
  t = f - tpre[u];
}

// One product step over all tiles: CTA b takes the flat tiles b, b + G, ...
// With two buffers (dbl) the basis of its next tile is in flight while one
// tile is applied; with one (Ph[0] == Ph[1]) the next copy starts once the
// tile is done. False (block-uniform) when a copy did not complete; the
// copies still in flight get a bounded wait first.
template <typename T>
__device__ bool tiles_phase(const IfaceArgs& a, const double* __restrict__ vin, int sel, const int* tpre, int nu,
                            T* const (&Ph)[2], bool dbl, T* Pv, TileScratch& ts, uint64_t* tbar, uint32_t (&par)[2],
                            const PcgCtl& c) {
  const int ntot = tpre[nu];
  int f = blockIdx.x;
  if (f >= ntot) return true;
  auto issue = [&](int ff, int buf) {
    int u, t;
    tile_locate(tpre, ff, u, t);
    int R;
    const T* ph = unit_phi_t<T>(a, u, a.tiles[3 * ((int64_t)u * a.max_tiles + t)], R);
    phi_load(Ph[buf], ph, (uint32_t)((R * R * (int)sizeof(T) + 15) & ~15), &tbar[buf]);
  };
  if (threadIdx.x == 0) issue(f, 0);
  int cur = 0;
  for (; f < ntot; f += gridDim.x, cur ^= 1) {
    const int fn = f + gridDim.x;
    // with two buffers the other one was released at the end of the last tile
    if (dbl && threadIdx.x == 0 && fn < ntot) issue(fn, cur ^ 1);
    int u, t;
    tile_locate(tpre, f, u, t);
    const int* tl = a.tiles + 3 * ((int64_t)u * a.max_tiles + t);
    const int q0 = tl[1], cntp = tl[2];
    const int* pts = a.grp_pts + (int64_t)u * a.pts_ld + q0;
    const int R = u == a.ns ? a.Rs : a.subs[u].R;
    const int nsel = tile_select(a, pts, cntp, sel, ts);
    if (nsel > 0) tile_gather<T>(a, vin, pts, u, R, nsel, ts, Pv);
    const bool ok = phi_wait(&tbar[cur], par[cur]);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(c.err, 1);
        atomicExch(c.abort, 1);
        phi_wait(&tbar[cur], par[cur]);
        if (dbl && fn < ntot) phi_wait(&tbar[cur ^ 1], par[cur ^ 1]);
      }
      __syncthreads();
      return false;
    }
    par[cur] ^= 1u;
    if (nsel > 0) tile_product<T>(a, u, R, nsel, ts, Ph[cur], Pv);
    __syncthreads();   // Ph[cur], Pv and ts are free again
    if (!dbl && threadIdx.x == 0 && fn < ntot) issue(fn, cur ^ 1);
  }
  return true;
}

// Resident tiles of the mixed CG's FP32 products: a CTA's tiles stay in its
// shared memory for the whole solve (the transposed bases, the point lists
// and the units' global DOFs), so that an iteration is one selection pass,
// one gather pass and one product pass over all of them. The products are
// 4 x 4 register tiles fed by float4 loads; every entry accumulates
// Phi[r][j] v_j over j in ascending order from zero, as tile_product does,
// so the results are the same.
constexpr int kResMax = 8;     // resident tiles per CTA (capacity of ResTiles)
constexpr int kResMax3 = 3;    // the resident tiles a CTA is given (shared memory for two CTAs per SM)
constexpr int kPvS = 36;       // row stride of a resident gathered block (floats)

// Shared-memory layout of the persistent CG (byte offsets into the dynamic
// allocation), set by the host.
struct PcgLayout {
  int phi_bytes;   // per streaming basis buffer (an FP64 basis of R_max^2)
  int nbuf;        // streaming buffers: 2 (prefetch) or 1
  int pv_off;      // streaming gathered vectors, R_max x (kTG + 1) doubles
  int stage_off;   // FP32 stage of n_lambda entries per warp (block preconditioner); may alias pv_off
  int resident;    // 1: the iteration products use resident tiles
  int r4;          // R_max rounded up to a multiple of 4
  int rphi_off;    // kResMax-capped m_max x r4 x r4 floats: transposed bases
  int rpv_off;     // m_max x r4 x kPvS floats: gathered vectors
  int rpts_off;    // m_max x kTG ints: the tile's points
  int rspt_off;    // m_max x kTG int64: the selected points
  int rgd_off;     // m_max x r4 ints: the unit's global DOFs
  const int* part; // resident: CTA b holds the flat tiles [part[b], part[b + 1])
};

struct ResTiles {
  int m;                   // tiles of this CTA
  int u[kResMax], R[kResMax], cnt[kResMax], nsel[kResMax];
  float* phiT;             // [m][r4][r4]
  float* pv;               // [m][r4][kPvS]
  int* pts;                // [m][kTG]
  int64_t* spt;            // [m][kTG]
  int* gd;                 // [m][r4]
  int r4;
};

// Once per launch: this CTA's tiles [part[b], part[b + 1]) into shared
// memory (a contiguous range of the flat tile list, balanced by cost on the
// host; at most kResMax tiles).
__device__ void resident_setup(const IfaceArgs& a, const int* tpre, int nu, const int* part, ResTiles& rt) {
  const int ntot = tpre[nu];
  const int f0 = min(part[blockIdx.x], ntot), f1 = min(part[blockIdx.x + 1], ntot);
  const int m = max(0, min(f1 - f0, kResMax));
  if (threadIdx.x == 0) rt.m = m;
  for (int j = 0; j < m; ++j) {
    const int f = f0 + j;
    int u, t;
    tile_locate(tpre, f, u, t);
    const int* tl = a.tiles + 3 * ((int64_t)u * a.max_tiles + t);
    const int k = tl[0], q0 = tl[1], cnt = tl[2];
    int R;
    const float* ph = unit_phi_t<float>(a, u, k, R);
    const int64_t* gd = u == a.ns ? a.sgdof : a.gdof + a.subs[u].gdof_off;
    const int* pts = a.grp_pts + (int64_t)u * a.pts_ld + q0;
    if (threadIdx.x == 0) { rt.u[j] = u; rt.R[j] = R; rt.cnt[j] = cnt; }
    const int r4 = rt.r4;
    float* phT = rt.phiT + (int64_t)j * r4 * r4;
    for (int e = threadIdx.x; e < r4 * r4; e += blockDim.x) {
      const int jj = e / r4, r = e - jj * r4;   // phT[jj][r] = Phi[r][jj]
      phT[e] = (jj < R && r < R) ? ph[r * R + jj] : 0.f;
    }
    for (int q = threadIdx.x; q < kTG; q += blockDim.x) rt.pts[j * kTG + q] = q < cnt ? pts[q] : 0;
    for (int i = threadIdx.x; i < r4; i += blockDim.x) rt.gd[j * r4 + i] = i < R ? (int)gd[i] : 0;
  }
  __syncthreads();
}

// One FP32 product step over the resident tiles (selection: iterating points).
__device__ void resident_products(const IfaceArgs& a, ResTiles& rt) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int m = rt.m, r4 = rt.r4;
  for (int j = warp; j < m; j += wpb) {   // one warp per tile (kTG == 32)
    const int cnt = rt.cnt[j];
    const int pt = rt.pts[j * kTG + lane];
    const bool act = lane < cnt && a.pstat[pt] == 0;
    const unsigned mask = __ballot_sync(0xffffffffu, act);
    if (act) rt.spt[j * kTG + __popc(mask & ((1u << lane) - 1u))] = pt;
    if (lane == 0) rt.nsel[j] = __popc(mask);
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const int nsel = rt.nsel[j], R = rt.R[j], nsel4 = (nsel + 3) & ~3;
    const int64_t* spt = rt.spt + j * kTG;
    const int* gd = rt.gd + j * r4;
    float* pv = rt.pv + (int64_t)j * r4 * kPvS;
    for (int e = threadIdx.x; e < nsel4 * R; e += blockDim.x) {
      const int q = e / R, i = e - q * R;
      float v = 0.f;
      if (q < nsel) v = from_f64<float>(a.p[spt[q] * a.n_lambda + gd[i]]);
      pv[i * kPvS + q] = v;
    }
  }
  __syncthreads();
  int total = 0;
  for (int j = 0; j < m; ++j) total += (((rt.R[j] + 3) >> 2) * ((rt.nsel[j] + 3) >> 2));
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    int j = 0, w0 = w;
    for (;;) {
      const int nj = ((rt.R[j] + 3) >> 2) * ((rt.nsel[j] + 3) >> 2);
      if (w0 < nj) break;
      w0 -= nj;
      ++j;
    }
    const int R = rt.R[j], nsel = rt.nsel[j], ncg = (nsel + 3) >> 2;
    const int r0 = (w0 / ncg) * 4, c0 = (w0 % ncg) * 4;
    const float* phT = rt.phiT + (int64_t)j * r4 * r4 + r0;
    const float* pv = rt.pv + (int64_t)j * r4 * kPvS + c0;
    float acc[4][4] = {};
    for (int jj = 0; jj < R; ++jj) {
      const float4 f = *reinterpret_cast<const float4*>(phT + jj * r4);
      const float4 v = *reinterpret_cast<const float4*>(pv + jj * kPvS);
      const float fr[4] = {f.x, f.y, f.z, f.w}, vq[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int ra = 0; ra < 4; ++ra)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[ra][q] = fmaf(fr[ra], vq[q], acc[ra][q]);
    }
    const int64_t* spt = rt.spt + j * kTG;
    const int64_t yb = a.ybase[rt.u[j]];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (c0 + q >= nsel) break;
      double* y = a.Y + spt[c0 + q] * a.NY + yb;
#pragma unroll
      for (int ra = 0; ra < 4; ++ra)
        if (r0 + ra < R) y[r0 + ra] = to_f64(acc[ra][q]);
    }
  }
}

// Grid of at most the co-resident CTAs of 256 threads; dynamic shared memory
// as PcgLayout sets it. T is the product type of the iterations (float: the
// mixed CG, whose checks take FP64 products; double: the FP64 CG).
template <typename T, bool kRegs>
__global__ void __launch_bounds__(256) cg_persistent_kernel(IfaceArgs a, PcgCtl c, double rtol, int max_it,
                                                            int chunk, double replace_ratio, double pause_ratio,
                                                            PcgLayout L) {
  extern __shared__ __align__(16) unsigned char pcg_raw[];
  __shared__ __align__(8) uint64_t tbar[2];
  __shared__ TileScratch ts;
  __shared__ int tpre[kPcgUnits + 1];
  __shared__ ResTiles rt;
  constexpr bool kMixed = sizeof(T) == 4;
  const bool resident = kMixed && L.resident;
  const int nu = a.ns + 1;
  unsigned char* buf0 = pcg_raw;
  unsigned char* buf1 = pcg_raw + (L.nbuf == 2 ? L.phi_bytes : 0);
  unsigned char* pvb = pcg_raw + L.pv_off;
  float* stage_all = reinterpret_cast<float*>(pcg_raw + L.stage_off);
  T* const PhT[2] = {reinterpret_cast<T*>(buf0), reinterpret_cast<T*>(buf1)};
  double* const PhD[2] = {reinterpret_cast<double*>(buf0), reinterpret_cast<double*>(buf1)};
  const bool dbl = L.nbuf == 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  float* stage = stage_all + warp * a.n_lambda;
  if (threadIdx.x == 0) {
    mbar_init1(&tbar[0]);
    mbar_init1(&tbar[1]);
    tpre[0] = 0;
    for (int u = 0; u < nu; ++u) tpre[u + 1] = tpre[u] + min(a.n_tiles[u], a.max_tiles);
    rt.r4 = L.r4;
    rt.phiT = reinterpret_cast<float*>(pcg_raw + L.rphi_off);
    rt.pv = reinterpret_cast<float*>(pcg_raw + L.rpv_off);
    rt.pts = reinterpret_cast<int*>(pcg_raw + L.rpts_off);
    rt.spt = reinterpret_cast<int64_t*>(pcg_raw + L.rspt_off);
    rt.gd = reinterpret_cast<int*>(pcg_raw + L.rgd_off);
  }
  __syncthreads();
  if (resident) resident_setup(a, tpre, nu, L.part, rt);
  uint32_t par[2] = {0u, 0u};
  unsigned gen = 0;
  int it = 0, chk = 0;
  bool ok = true;
  // thread 0's clock between the steps
  long long cyc[6] = {0, 0, 0, 0, 0, 0}, t_last = clock64();
  auto mark = [&](int k) {
    if (threadIdx.x == 0) {
      const long long t = clock64();
      cyc[k] += t - t_last;
      t_last = t;
    }
  };
  while (it < max_it) {
    for (int q = 0; q < chunk && it < max_it; ++q, ++it) {
      if (resident) {
        resident_products(a, rt);
        ok = true;
      } else {
        ok = tiles_phase<T>(a, a.p, 0, tpre, nu, PhT, dbl, reinterpret_cast<T*>(pvb), ts, tbar, par, c);
      }
      mark(0);
      ok = grid_sync(c, gen) && ok;
      mark(1);
      if (!ok) break;
      // point l to CTA l mod G: every CTA (and SM) gets its share of the FP64 updates
      for (int64_t l = (int64_t)warp * gridDim.x + blockIdx.x; l < a.n_pts; l += (int64_t)gridDim.x * wpb)
        update_point<kRegs>(a, l, lane, stage, it, rtol, kMixed ? 1 : 0, replace_ratio, pause_ratio);
      mark(2);
      ok = grid_sync(c, gen);
      mark(3);
      if (!ok) break;
    }
    if (!ok) break;
    if (kMixed) {   // FP64 residuals of the points that asked for one
      ok = tiles_phase<double>(a, a.lam, 1, tpre, nu, PhD, dbl, reinterpret_cast<double*>(pvb), ts, tbar, par, c);
      mark(4);
      ok = grid_sync(c, gen) && ok;
      if (!ok) break;
      for (int64_t l = (int64_t)warp * gridDim.x + blockIdx.x; l < a.n_pts; l += (int64_t)gridDim.x * wpb)
        reliable_point(a, l, lane, stage, rtol, it);
      ok = grid_sync(c, gen);
      if (!ok) break;
    }
    // iterating points; the slot two checks ahead is cleared for reuse (every
    // CTA has read it: it has passed barriers since)
    int* slot = c.act + (chk & 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) c.act[(chk + 2) & 3] = 0;
    int cnt = 0;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < a.n_pts; l += (int64_t)gridDim.x * blockDim.x)
      cnt += a.pstat[l] == 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(slot, cnt);
    ok = grid_sync(c, gen);
    mark(5);
    if (!ok) break;
    ++chk;
    if (*((volatile int*)slot) == 0) break;
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) atomicAdd(&c.cyc[k], (unsigned long long)cyc[k]);
  if (blockIdx.x == 0 && threadIdx.x == 0) *c.iters = it;
}

// ---- moments ---------------------------------------------------------------------
// Darcy fields: per-point recovery p = X^k [R lambda; 1] on a tile of grid rows
// (plus one halo row for the y-face fluxes), face velocities from p, and the
// shifted sums sum w (x - shift), sum w (x - shift)^2 accumulated in registers
// by the thread that owns each field entry; one partial per point chunk,
// summed in a fixed order afterwards (deterministic, no floating atomics).
struct MomArgs {
  IfaceArgs ia;
  const double* X;
  const double* T;
  const double* proj;
  const double* w;
  double* shift;            // [len_d] shifts (the field at point 0 of the first batch)
  double* part;             // [n_chunks][2][len_d] partial sums of this batch
  int64_t len_d;            // Darcy entries: all cell pressures, then all face velocities
  int64_t off_f;            // first face-velocity entry
  const int64_t* cell_off;  // per subdomain first cell
  const int64_t* face_off;  // per subdomain first face
  int mode;                 // 0: write the shifts from point 0; 1: accumulate
  int rt;                   // grid rows per CTA
  int n_chunks;
  // groups larger than big_factor * (R+1) points go through their coefficient moments
  double big_factor;
  const int* grp_start;     // per (subdomain, local realization): first sorted point
  const int* grp_end;       // ... and one past the last
  const int64_t* loc_off;   // per subdomain offset into the group arrays
  double* gmom;             // per group: W | cbar[C] | m[C] | M[C][C]
  int64_t gmom_stride;
  int df;                   // 1: the contractions in double-float (mixed form), 0: FP64
};

// Double-float arithmetic: a value as an FP32 pair hi + lo (about 48
// significant bits), with the error-free product by FMA and Knuth's
// error-free sum, so that the mixed form's moment contractions run on the
// FP32 pipe (FP64 issues at 1/64 of its rate here). The explicit _rn
// intrinsics keep the compiler from contracting the error terms.
__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  h = f64_to_f32_bits(x);
  l = f64_to_f32_bits(x - f32_to_f64_bits(h));
}
// (sh, sl) += (ah + al)(bh + bl), the al bl term dropped
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float x = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float sum = __fadd_rn(sh, p);
  const float v = __fsub_rn(sum, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(sum, v)), __fsub_rn(p, v));
  sh = sum;
  sl = __fadd_rn(sl, __fadd_rn(e, __fadd_rn(pe, x)));
}
// hi the rounded value of hi + lo
__device__ __forceinline__ void df_renorm(float& h, float& l) {
  const float t = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(t, h));
  h = t;
}
// (ah, al) += (bh, bl), renormalized
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  const float sum = __fadd_rn(ah, bh);
  const float v = __fsub_rn(sum, ah);
  const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, v)), __fsub_rn(bh, v));
  ah = sum;
  al = __fadd_rn(e, __fadd_rn(al, bl));
  df_renorm(ah, al);
}
__device__ __forceinline__ double df_value(float h, float l) { return f32_to_f64_bits(h) + f32_to_f64_bits(l); }

__device__ __forceinline__ bool big_group(const MomArgs& m, const SubDev& S, int s, int k) {
  const int64_t g = m.loc_off[s] + k;
  return m.big_factor > 0.0 && (double)(m.grp_end[g] - m.grp_start[g]) > m.big_factor * (S.R + 1);
}

constexpr int kMomT = 256;   // threads of the Darcy moments kernel
constexpr int kMaxE = 8;     // field entries owned per thread

__device__ __forceinline__ double darcy_value(const SubDev& S, const MomArgs& m, int64_t e_loc, int r0, int r1,
                                              int h0, const double* Tx, const double* Ty, const double* Z,
                                              const double* Cf, int q, int C, double ihx, double ihy) {
  const int nx = S.nx, ny = S.ny, R = S.R;
  const int np = (r1 - r0) * nx, nxf = (r1 - r0) * (nx + 1);
  if (e_loc < np) {
    const int c = (r0 - h0) * nx + (int)e_loc;
    return Z[c * kTP + q];
  }
  if (e_loc < np + nxf) {
    const int f = (int)(e_loc - np);
    const int rr_ = r0 + f / (nx + 1), ix = f % (nx + 1);
    const int zrow = (rr_ - h0) * nx;
    const double t = Tx[(int64_t)rr_ * (nx + 1) + ix];
    if (ix > 0 && ix < nx) return t * ihy * (Z[(zrow + ix - 1) * kTP + q] - Z[(zrow + ix) * kTP + q]);
    const int side = ix == 0 ? 3 : 1;
    if (S.side_type[side] == SIDE_NOFLOW) return 0.0;
    double gb = S.side_val[side];
    if (S.side_type[side] == SIDE_IFACE) {
      const double* P = m.proj + S.proj_off[side] + (int64_t)rr_ * R;
      gb = 0.0;
      for (int i = 0; i < R; ++i) gb += P[i] * Cf[q * C + i];
    }
    const double F = t * ihy * (Z[(zrow + (ix == 0 ? 0 : nx - 1)) * kTP + q] - gb);
    return ix == 0 ? -F : F;
  }
  const int f = (int)(e_loc - np - nxf);
  const int j = r0 + f / nx, ix = f % nx;
  const double t = Ty[(int64_t)j * nx + ix];
  if (j > 0 && j < ny) return t * ihx * (Z[((j - 1 - h0) * nx + ix) * kTP + q] - Z[((j - h0) * nx + ix) * kTP + q]);
  const int side = j == 0 ? 0 : 2;
  if (S.side_type[side] == SIDE_NOFLOW) return 0.0;
  double gb = S.side_val[side];
  if (S.side_type[side] == SIDE_IFACE) {
    const double* P = m.proj + S.proj_off[side] + (int64_t)ix * R;
    gb = 0.0;
    for (int i = 0; i < R; ++i) gb += P[i] * Cf[q * C + i];
  }
  const double F = t * ihx * (Z[((j == 0 ? 0 : ny - 1) - h0) * nx * kTP + ix * kTP + q] - gb);
  return j == 0 ? -F : F;
}

// Global entry index of a tile-local entry.
__device__ __forceinline__ int64_t darcy_entry(const SubDev& S, const MomArgs& m, int s, int64_t e_loc, int r0,
                                               int r1) {
  const int nx = S.nx, ny = S.ny;
  const int np = (r1 - r0) * nx, nxf = (r1 - r0) * (nx + 1);
  if (e_loc < np) return m.cell_off[s] + (int64_t)r0 * nx + e_loc;
  if (e_loc < np + nxf) return m.off_f + m.face_off[s] + (int64_t)r0 * (nx + 1) + (e_loc - np);
  return m.off_f + m.face_off[s] + (int64_t)ny * (nx + 1) + (int64_t)r0 * nx + (e_loc - np - nxf);
}

// Z[c][q] = sum_i X[c][i] Cf[q][i] for the cells c < ncell of a row tile
// (X column-major with column stride nc) and the first NQ points of the
// sub-tile; FP64, one cell per thread.
template <int NQ>
__device__ __forceinline__ void field_rows(const double* __restrict__ X, int nc, int C, int ncell,
                                           const double* Cf, double* Z) {
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const double* xr = X + c;
    // at least four independent FMA chains: NQ accumulators, each split over
    // 4 / NQ interleaved column ranges when NQ < 4
    constexpr int NS = NQ >= 4 ? 1 : 4 / NQ;
    double z[NS][NQ];
#pragma unroll
    for (int u = 0; u < NS; ++u)
#pragma unroll
      for (int q = 0; q < NQ; ++q) z[u][q] = 0.0;
    int i = 0;
    for (; i + NS <= C; i += NS) {
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        const double xv = xr[(int64_t)(i + u) * nc];
#pragma unroll
        for (int q = 0; q < NQ; ++q) z[u][q] = fma(xv, Cf[q * C + i + u], z[u][q]);
      }
    }
    for (; i < C; ++i) {
      const double xv = xr[(int64_t)i * nc];
#pragma unroll
      for (int q = 0; q < NQ; ++q) z[0][q] = fma(xv, Cf[q * C + i], z[0][q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double v = z[0][q];
#pragma unroll
      for (int u = 1; u < NS; ++u) v += z[u][q];
      Z[c * kTP + q] = v;
    }
  }
}

// field_rows in double-float: Z = X rows times the points' coefficients,
// each X entry split once (one FP64 subtraction) for NQ points.
template <int NQ>
__device__ __forceinline__ void field_rows_df(const double* __restrict__ X, int nc, int C, int ncell,
                                              const float* Cfh, const float* Cfl, double* Z) {
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const double* xr = X + c;
    float sh[NQ], sl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { sh[q] = 0.f; sl[q] = 0.f; }
#pragma unroll 4
    for (int i = 0; i < C; ++i) {
      float xh, xl;
      df_split(xr[(int64_t)i * nc], xh, xl);
#pragma unroll
      for (int q = 0; q < NQ; ++q) df_mac(xh, xl, Cfh[q * C + i], Cfl[q * C + i], sh[q], sl[q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) Z[c * kTP + q] = df_value(sh[q], sl[q]);
  }
}

// Row tile blockIdx.x of subdomain s, point chunk ch: mode 0 writes the shifts
// (the fields at point 0), mode 1 the partial sums of chunk ch.
__device__ __forceinline__ void darcy_moments_tile(const MomArgs& m, double* sm, int s, int ch, int& gsub) {
  const IfaceArgs& a = m.ia;
  const SubDev S = a.subs[s];
  const int nx = S.nx, ny = S.ny, R = S.R, C = R + 1, nc = nx * ny;
  const int r0 = blockIdx.x * m.rt;
  if (r0 >= ny) return;
  if (m.mode == 0 && ch != 0) return;
  const int r1 = min(ny, r0 + m.rt);
  const int h0 = max(0, r0 - 1);
  const int ncell = (r1 - h0) * nx;
  const int n_ent = (r1 - r0) * nx + (r1 - r0) * (nx + 1) + ((r1 == ny ? ny + 1 : r1) - r0) * nx;
  double* Cf = sm;                  // [kTP][C]
  double* Z = Cf + kTP * C;         // [ncell][kTP]
  double* Wt = Z + ncell * kTP;     // [kTP]
  const int64_t* gd = a.gdof + S.gdof_off;
  double sh[kMaxE], acc1[kMaxE], acc2[kMaxE];
#pragma unroll
  for (int q = 0; q < kMaxE; ++q) {
    const int64_t el = threadIdx.x + (int64_t)q * kMomT;
    sh[q] = (m.mode == 1 && el < n_ent) ? m.shift[darcy_entry(S, m, s, el, r0, r1)] : 0.0;
    acc1[q] = 0.0;
    acc2[q] = 0.0;
  }
  const double ihx = 1.0 / S.hx, ihy = 1.0 / S.hy;
  // mode 0 scans every tile for point 0; mode 1 takes every n_chunks-th
  // sub-tile of kTP points in a running count over all subdomains (gsub), so
  // large tiles spread over several CTAs
  for (int t = 0; t < a.n_tiles[s]; ++t) {
    const int* tl = a.tiles + 3 * ((int64_t)s * a.max_tiles + t);
    const int k = tl[0];
    if (m.mode == 1 && big_group(m, S, s, k)) continue;  // handled by its coefficient moments
    const ItemOff off = a.off[S.item0 + k];
    const double* X = m.X + off.x;
    const double* Tx = m.T + off.t;
    const double* Ty = Tx + (int64_t)ny * (nx + 1);
    const int cnt_tile = tl[2];
    const int* tpts = a.grp_pts + (int64_t)s * a.pts_ld + tl[1];
    int q_begin = 0, q_end = cnt_tile;
    if (m.mode == 0) {
      int has0 = -1;
      for (int q = 0; q < cnt_tile; ++q)
        if (tpts[q] == 0) has0 = q;
      if (has0 < 0) continue;
      q_begin = has0;
      q_end = has0 + 1;
    }
    for (int qs = q_begin; qs < q_end; qs += kTP) {
      if (m.mode == 1 && (gsub++ % m.n_chunks) != ch) continue;
      const int* pts = tpts + qs;
      const int cntp = min(kTP, q_end - qs);
      __syncthreads();
      for (int e = threadIdx.x; e < cntp * C; e += blockDim.x) {
        const int q = e / C, i = e - q * C;
        Cf[e] = i < R ? a.lam[(int64_t)pts[q] * a.n_lambda + gd[i]] : 1.0;
      }
      for (int q = threadIdx.x; q < kTP; q += blockDim.x) Wt[q] = q < cntp ? m.w[pts[q]] : 0.0;
      __syncthreads();
      // only the sub-tile's points: 1, 2, 4 or kTP columns
      if (cntp == 1) field_rows<1>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
      else if (cntp == 2) field_rows<2>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
      else if (cntp <= 4) field_rows<4>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
      else field_rows<kTP>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kMaxE; ++j) {
        const int64_t el = threadIdx.x + (int64_t)j * kMomT;
        if (el >= n_ent) break;
        for (int q = 0; q < cntp; ++q) {
          const double v = darcy_value(S, m, el, r0, r1, h0, Tx, Ty, Z, Cf, q, C, ihx, ihy);
          if (m.mode == 0) {
            sh[j] = v;
          } else {
            const double d = v - sh[j];
            acc1[j] = fma(Wt[q], d, acc1[j]);
            acc2[j] = fma(Wt[q] * d, d, acc2[j]);
          }
        }
      }
    }
    if (m.mode == 0) break;
  }
#pragma unroll
  for (int j = 0; j < kMaxE; ++j) {
    const int64_t el = threadIdx.x + (int64_t)j * kMomT;
    if (el >= n_ent) break;
    const int64_t ge = darcy_entry(S, m, s, el, r0, r1);
    if (m.mode == 0) {
      m.shift[ge] = sh[j];
    } else {
      m.part[((int64_t)ch * 2) * m.len_d + ge] = acc1[j];
      m.part[((int64_t)ch * 2 + 1) * m.len_d + ge] = acc2[j];
    }
  }
}

// Mode 0: grid (row tiles, subdomains). Mode 1: grid (row tiles, 1, chunks);
// every CTA walks all subdomains, taking every n_chunks-th tile of each, so
// the point-by-point work spreads over all CTAs whichever subdomains hold it.
__global__ void __launch_bounds__(kMomT) darcy_moments_kernel(MomArgs m) {
  extern __shared__ __align__(16) double sm[];
  int gsub = 0;
  darcy_moments_tile(m, sm, blockIdx.y, 0, gsub);
}

// The point-by-point sub-tiles of kTP points of every subdomain, in
// subdomain order: work[i] = (subdomain, tile, first point in the tile).
// One CTA: per subdomain a block scan of the sub-tile counts of its tiles.
__global__ void __launch_bounds__(256) moments_worklist_kernel(MomArgs m, int4* work, int* nwork, int cap,
                                                                int* err) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const IfaceArgs& a = m.ia;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  for (int s = 0; s < a.ns; ++s) {
    const SubDev& S = a.subs[s];
    const int nt = a.n_tiles[s];
    for (int t0 = 0; t0 < nt; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      int cnt = 0;
      if (t < nt) {
        const int* tl = a.tiles + 3 * ((int64_t)s * a.max_tiles + t);
        if (!big_group(m, S, s, tl[0])) cnt = (tl[2] + kTP - 1) / kTP;
      }
      int v = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
      }
      if (lane == 31) wsum[warp] = v;
      __syncthreads();
      if (warp == 0) {
        int w = lane < nwarps ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
          const int n = __shfl_up_sync(0xffffffffu, w, o);
          if (lane >= o) w += n;
        }
        if (lane < nwarps) wsum[lane] = w;
      }
      __syncthreads();
      const int excl = v - cnt + (warp > 0 ? wsum[warp - 1] : 0);
      const int total = wsum[nwarps - 1];
      const int base = base_s;
      for (int q = 0; q < cnt; ++q) {
        if (base + excl + q < cap) work[base + excl + q] = make_int4(s, t, q * kTP, 0);
        else atomicOr(err, 4);   // list longer than its buffer: the entry is dropped
      }
      __syncthreads();
      if (threadIdx.x == 0) base_s = base + total;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) *nwork = min(base_s, cap);
}

// Mode-1 accumulation over the work list: CTA (row tile, chunk) takes every
// n_chunks-th sub-tile of the list and keeps register accumulators for the
// entries of its row tile of the current subdomain, writing them to partial
// slot `chunk` when the list moves to the next subdomain. Slots of
// (subdomain, chunk) pairs without work stay at the zeros written before.
__global__ void __launch_bounds__(kMomT) darcy_moments_list_kernel(MomArgs m, const int4* work, const int* nwork,
                                                                  int* err) {
  extern __shared__ __align__(16) double sm[];
  const IfaceArgs& a = m.ia;
  const int ch = blockIdx.z;
  const int nw = *nwork;
  int cur = -1;
  bool valid = false;
  SubDev S;
  int nx = 0, ny = 0, R = 0, C = 0, nc = 0, r0 = 0, r1 = 0, h0 = 0, ncell = 0, n_ent = 0;
  double ihx = 0.0, ihy = 0.0;
  double sh[kMaxE], acc1[kMaxE], acc2[kMaxE];
  // the accumulators of the current subdomain's row tile into slot ch
  auto flush = [&]() {
    if (cur < 0 || !valid) return;
#pragma unroll
    for (int j = 0; j < kMaxE; ++j) {
      const int64_t el = threadIdx.x + (int64_t)j * kMomT;
      if (el >= n_ent) break;
      const int64_t ge = darcy_entry(S, m, cur, el, r0, r1);
      m.part[((int64_t)ch * 2) * m.len_d + ge] = acc1[j];
      m.part[((int64_t)ch * 2 + 1) * m.len_d + ge] = acc2[j];
    }
  };
  for (int e = ch; e < nw; e += m.n_chunks) {
    const int4 w = work[e];
    if (w.x != cur) {
      flush();
      if (w.x < 0 || w.x >= a.ns) {   // a malformed list entry ends this CTA's walk and is reported
        if (threadIdx.x == 0) atomicOr(err, 8);
        cur = -1;
        break;
      }
      cur = w.x;
      S = a.subs[cur];
      nx = S.nx; ny = S.ny; R = S.R; C = R + 1; nc = nx * ny;
      r0 = blockIdx.x * m.rt;
      valid = r0 < ny;
      r1 = min(ny, r0 + m.rt);
      h0 = max(0, r0 - 1);
      ncell = (r1 - h0) * nx;
      n_ent = valid ? (r1 - r0) * nx + (r1 - r0) * (nx + 1) + ((r1 == ny ? ny + 1 : r1) - r0) * nx : 0;
      ihx = 1.0 / S.hx; ihy = 1.0 / S.hy;
#pragma unroll
      for (int q = 0; q < kMaxE; ++q) {
        const int64_t el = threadIdx.x + (int64_t)q * kMomT;
        sh[q] = el < n_ent ? m.shift[darcy_entry(S, m, cur, el, r0, r1)] : 0.0;
        acc1[q] = 0.0;
        acc2[q] = 0.0;
      }
    }
    if (!valid) continue;
    if (w.y < 0 || w.y >= a.n_tiles[cur]) {   // a malformed list entry is skipped and reported
      if (threadIdx.x == 0) atomicOr(err, 8);
      continue;
    }
    const int* tl = a.tiles + 3 * ((int64_t)cur * a.max_tiles + w.y);
    const int k = tl[0];
    if (k < 0 || k >= S.n_local || w.z < 0 || w.z >= tl[2] || tl[1] < 0 || tl[1] + tl[2] > a.n_pts) {
      if (threadIdx.x == 0) atomicOr(err, 16);
      continue;
    }
    const ItemOff off = a.off[S.item0 + k];
    const double* X = m.X + off.x;
    const double* Tx = m.T + off.t;
    const double* Ty = Tx + (int64_t)ny * (nx + 1);
    const int* pts = a.grp_pts + (int64_t)cur * a.pts_ld + tl[1] + w.z;
    const int cntp = min(kTP, tl[2] - w.z);
    const int64_t* gd = a.gdof + S.gdof_off;
    double* Cf = sm;                  // [kTP][C]
    double* Z = Cf + kTP * C;         // [ncell][kTP]
    double* Wt = Z + ncell * kTP;     // [kTP]
    float* Cfh = reinterpret_cast<float*>(Wt + kTP);   // [kTP][C] double-float split of Cf
    float* Cfl = Cfh + kTP * C;
    const bool dfp = m.df && cntp > 2;   // double-float once an X entry serves 4 or more points
    __syncthreads();
    for (int e2 = threadIdx.x; e2 < kTP * C; e2 += blockDim.x) {
      const int q = e2 / C, i = e2 - q * C;
      const double v = q < cntp ? (i < R ? a.lam[(int64_t)pts[q] * a.n_lambda + gd[i]] : 1.0) : 0.0;
      if (q < cntp) Cf[e2] = v;
      if (dfp) df_split(v, Cfh[e2], Cfl[e2]);
    }
    for (int q = threadIdx.x; q < kTP; q += blockDim.x) Wt[q] = q < cntp ? m.w[pts[q]] : 0.0;
    __syncthreads();
    if (cntp == 1) field_rows<1>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
    else if (cntp == 2) field_rows<2>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
    else if (dfp && cntp <= 4) field_rows_df<4>(X + (int64_t)h0 * nx, nc, C, ncell, Cfh, Cfl, Z);
    else if (dfp) field_rows_df<kTP>(X + (int64_t)h0 * nx, nc, C, ncell, Cfh, Cfl, Z);
    else if (cntp <= 4) field_rows<4>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
    else field_rows<kTP>(X + (int64_t)h0 * nx, nc, C, ncell, Cf, Z);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kMaxE; ++j) {
      const int64_t el = threadIdx.x + (int64_t)j * kMomT;
      if (el >= n_ent) break;
      for (int q = 0; q < cntp; ++q) {
        const double v = darcy_value(S, m, el, r0, r1, h0, Tx, Ty, Z, Cf, q, C, ihx, ihy);
        const double d = v - sh[j];
        acc1[j] = fma(Wt[q], d, acc1[j]);
        acc2[j] = fma(Wt[q] * d, d, acc2[j]);
      }
    }
  }
  flush();
}

constexpr int kGChunks = 16;   // point chunks per large group (partials reduced in order)

// Partial coefficient moments of one large group k of subdomain s over point
// chunk blockIdx.z, about the coefficients cbar of the group's first point:
// W = sum w, m = sum w d, M = sum w d d^T with d = [R lambda_l; 1] - cbar.
// M is computed in 4 x 4 register tiles; points are staged 16 at a time.
__global__ void __launch_bounds__(256) group_moments_kernel(MomArgs m, double* part) {
  __shared__ double Dl[16][kMaxCols + 3];
  __shared__ double Wl[16];
  __shared__ double cbar[kMaxCols];
  const IfaceArgs& a = m.ia;
  const int k = blockIdx.x, s = blockIdx.y, ch = blockIdx.z;
  const SubDev& S = a.subs[s];
  if (k >= S.n_local || !big_group(m, S, s, k)) return;
  const int R = S.R, C = R + 1;
  const int64_t g = m.loc_off[s] + k;
  const int g0 = m.grp_start[g], g1 = m.grp_end[g];
  const int per = (g1 - g0 + kGChunks - 1) / kGChunks;
  const int p0 = g0 + ch * per, p1 = min(g1, p0 + per);
  const int* pts = a.grp_pts + (int64_t)s * a.pts_ld;
  const int64_t* gd = a.gdof + S.gdof_off;
  for (int i = threadIdx.x; i < C; i += blockDim.x)
    cbar[i] = i < R ? a.lam[(int64_t)pts[g0] * a.n_lambda + gd[i]] : 1.0;
  const int nt4 = (C + 3) >> 2;
  const int ntile = nt4 * nt4;
  double* out = part + ((int64_t)g * kGChunks + ch) * m.gmom_stride;
  for (int tb = 0; tb < ntile; tb += blockDim.x) {
    const int t = tb + threadIdx.x;
    const int a0 = (t / nt4) * 4, b0 = (t % nt4) * 4;
    double acc[4][4] = {};
    double accm = 0.0, accW = 0.0;
    for (int q0 = p0; q0 < p1; q0 += 16) {
      const int nq = min(16, p1 - q0);
      __syncthreads();
      for (int e = threadIdx.x; e < nq * (C + 3); e += blockDim.x) {
        const int q = e / (C + 3), i = e - q * (C + 3);
        double v = 0.0;
        if (i < C) {
          const int64_t l = pts[q0 + q];
          v = (i < R ? a.lam[l * a.n_lambda + gd[i]] : 1.0) - cbar[i];
        }
        Dl[q][i] = v;
      }
      for (int q = threadIdx.x; q < nq; q += blockDim.x) Wl[q] = m.w[pts[q0 + q]];
      __syncthreads();
      if (t < ntile) {
        for (int q = 0; q < nq; ++q) {
          const double wq = Wl[q];
          double da[4], db[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) { da[i] = wq * Dl[q][a0 + i]; db[i] = Dl[q][b0 + i]; }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(da[i], db[j], acc[i][j]);
          if (tb == 0 && threadIdx.x < C) accm = fma(wq, Dl[q][threadIdx.x], accm);
          if (tb == 0 && threadIdx.x == 0) accW += wq;
        }
      }
    }
    if (t < ntile)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (a0 + i < C && b0 + j < C) out[1 + 2 * C + (a0 + i) * C + b0 + j] = acc[i][j];
    if (tb == 0) {
      if (threadIdx.x < C) { out[1 + threadIdx.x] = cbar[threadIdx.x]; out[1 + C + threadIdx.x] = accm; }
      if (threadIdx.x == 0) out[0] = accW;
    }
  }
}

// gmom[g] = sum over the point chunks of the partial moments (fixed order).
__global__ void group_moments_reduce(MomArgs m, const double* part) {
  const IfaceArgs& a = m.ia;
  const int k = blockIdx.x, s = blockIdx.y;
  const SubDev& S = a.subs[s];
  if (k >= S.n_local || !big_group(m, S, s, k)) return;
  const int C = S.R + 1;
  const int64_t g = m.loc_off[s] + k;
  const int n = 1 + 2 * C + C * C;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    double v = 0.0;
    if (e >= 1 + C && e < 1 + 2 * C || e == 0 || e >= 1 + 2 * C) {
      for (int c = 0; c < kGChunks; ++c) v += part[((int64_t)g * kGChunks + c) * m.gmom_stride + e];
    } else {
      v = part[((int64_t)g * kGChunks) * m.gmom_stride + e];  // cbar: the same in every chunk
    }
    m.gmom[g * m.gmom_stride + e] = v;
  }
}

constexpr int kBigT = 128;   // threads of the large-group moments kernel
constexpr int kBigE = 2;     // field entries per thread

// Affine map of one Darcy entry onto the columns a of X (item with
// transmissibilities Tx, Ty): v_a = t (X[a][c1] - X[a][c2]) for interior faces,
// t (X[a][c1] - g_a) for faces on a Dirichlet or interface side (g_a the
// mortar projection P[a] for a < R, or the side value in column R), X[a][c1]
// for cells (t = 1, no second term); t carries the face sign and is zero on
// no-flow sides.
struct EntryMap {
  int c1, c2;          // cells; c2 < 0: boundary or cell entry
  double t;
  const double* P;     // interface side: projection row of the face (length R)
  double dval;         // Dirichlet side: value carried by column R
};

__device__ __forceinline__ EntryMap entry_map(const SubDev& S, const MomArgs& m, int64_t e_loc, const double* Tx,
                                              const double* Ty, double ihx, double ihy) {
  const int nx = S.nx, ny = S.ny, R = S.R;
  const int np = ny * nx, nxf = ny * (nx + 1);
  EntryMap em;
  em.c2 = -1; em.P = nullptr; em.dval = 0.0;
  if (e_loc < np) { em.c1 = (int)e_loc; em.t = 1.0; return em; }
  int side, cell;
  double t;
  if (e_loc < np + nxf) {
    const int f = (int)(e_loc - np);
    const int row = f / (nx + 1), ix = f % (nx + 1);
    t = Tx[(int64_t)row * (nx + 1) + ix] * ihy;
    if (ix > 0 && ix < nx) { em.c1 = row * nx + ix - 1; em.c2 = row * nx + ix; em.t = t; return em; }
    side = ix == 0 ? 3 : 1;
    cell = row * nx + (ix == 0 ? 0 : nx - 1);
    if (S.side_type[side] == SIDE_IFACE) em.P = m.proj + S.proj_off[side] + (int64_t)row * R;
  } else {
    const int f = (int)(e_loc - np - nxf);
    const int j = f / nx, ix = f % nx;
    t = Ty[(int64_t)j * nx + ix] * ihx;
    if (j > 0 && j < ny) { em.c1 = (j - 1) * nx + ix; em.c2 = j * nx + ix; em.t = t; return em; }
    side = j == 0 ? 0 : 2;
    cell = (j == 0 ? 0 : ny - 1) * nx + ix;
    if (S.side_type[side] == SIDE_IFACE) em.P = m.proj + S.proj_off[side] + (int64_t)ix * R;
  }
  em.c1 = cell;
  if (S.side_type[side] == SIDE_NOFLOW) t = 0.0;
  if (S.side_type[side] == SIDE_DIRICHLET) em.dval = S.side_val[side];
  em.t = (side == 0 || side == 3) ? -t : t;
  return em;
}

__device__ __forceinline__ double entry_map_coef(const EntryMap& em, const double* X, int64_t nc, int R, int a) {
  const double x1 = X[(int64_t)a * nc + em.c1];
  double x2;
  if (em.c2 >= 0) x2 = X[(int64_t)a * nc + em.c2];
  else if (em.P) x2 = a < R ? em.P[a] : 0.0;
  else x2 = a == R ? em.dval : 0.0;
  return em.t * (x1 - x2);
}

// Large groups: with F the entry's coefficient row and v = F c,
// sum_l w (v_l - s) = F m + W (F cbar - s) and
// sum_l w (v_l - s)^2 = F M F^T + 2 (F cbar - s) F m + W (F cbar - s)^2,
// F M F^T summed over the upper triangle of the symmetric M. A CTA owns
// kBigT * kBigE consecutive entries of one subdomain (cells, x-faces, y-faces)
// and writes partial slot `slot` for each of them (zeros when the subdomain
// has no large group).
__global__ void __launch_bounds__(kBigT) bigroup_moments_kernel(MomArgs m, int slot) {
  extern __shared__ __align__(16) double smb[];
  const IfaceArgs& a = m.ia;
  const int s = blockIdx.y;
  const SubDev S = a.subs[s];
  const int nx = S.nx, ny = S.ny, R = S.R, C = R + 1;
  const int n_ent = ny * nx + ny * (nx + 1) + (ny + 1) * nx;
  const int nt = blockDim.x;   // kBigT, or fewer when C*C + C*kBigT doubles exceed shared memory
  const int64_t e0 = (int64_t)blockIdx.x * nt * kBigE;
  if (e0 >= n_ent) return;
  double* Ms = smb;                 // [C][C]
  double* cb = Ms + C * C;          // [C]
  double* mv = cb + C;              // [C]
  double* Fs = mv + C;              // [C][nt]
  const double ihx = 1.0 / S.hx, ihy = 1.0 / S.hy;
  double sh[kBigE], acc1[kBigE], acc2[kBigE];
#pragma unroll
  for (int j = 0; j < kBigE; ++j) {
    const int64_t el = e0 + threadIdx.x + (int64_t)j * nt;
    sh[j] = el < n_ent ? m.shift[darcy_entry(S, m, s, el, 0, ny)] : 0.0;
    acc1[j] = 0.0;
    acc2[j] = 0.0;
  }
  double* Fc = Fs + threadIdx.x;    // this thread's column of F, stride nt
  for (int k = 0; k < S.n_local; ++k) {
    if (!big_group(m, S, s, k)) continue;
    const double* gm = m.gmom + (m.loc_off[s] + k) * m.gmom_stride;
    const ItemOff off = a.off[S.item0 + k];
    const double* X = m.X + off.x;
    const double* Tx = m.T + off.t;
    const double* Ty = Tx + (int64_t)ny * (nx + 1);
    __syncthreads();
    // M in FP64, or split into FP32 hi and lo halves (the same bytes) for double-float
    float* MsH = reinterpret_cast<float*>(Ms);
    float* MsL = MsH + C * C;
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
      if (m.df) df_split(gm[1 + 2 * C + e], MsH[e], MsL[e]);
      else Ms[e] = gm[1 + 2 * C + e];
    }
    for (int e = threadIdx.x; e < C; e += blockDim.x) { cb[e] = gm[1 + e]; mv[e] = gm[1 + C + e]; }
    const double W = gm[0];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBigE; ++j) {
      const int64_t el = e0 + threadIdx.x + (int64_t)j * nt;
      if (el >= n_ent) break;
      const EntryMap em = entry_map(S, m, el, Tx, Ty, ihx, ihy);
      double fc = 0.0, fm = 0.0;
      float2* Fc2 = reinterpret_cast<float2*>(Fc);
#pragma unroll 4
      for (int ia = 0; ia < C; ++ia) {
        const double f = entry_map_coef(em, X, (int64_t)nx * ny, R, ia);
        if (m.df) {
          float fh, fl;
          df_split(f, fh, fl);
          Fc2[ia * nt] = make_float2(fh, fl);
        } else {
          Fc[ia * nt] = f;
        }
        fc = fma(f, cb[ia], fc);
        fm = fma(f, mv[ia], fm);
      }
      double q = 0.0;
      if (m.df) {
        // F M F^T in double-float: per row the upper-triangle sum in two
        // chains, then row = M_aa F_a + 2 r and q += F_a row
        float qh = 0.f, ql = 0.f;
        for (int ia = 0; ia < C; ++ia) {
          const float* Mh = MsH + ia * C;
          const float* Ml = MsL + ia * C;
          float r0h = 0.f, r0l = 0.f, r1h = 0.f, r1l = 0.f;
          int ib = ia + 1;
          for (; ib + 1 < C; ib += 2) {
            const float2 f0 = Fc2[ib * nt], f1 = Fc2[(ib + 1) * nt];
            df_mac(Mh[ib], Ml[ib], f0.x, f0.y, r0h, r0l);
            df_mac(Mh[ib + 1], Ml[ib + 1], f1.x, f1.y, r1h, r1l);
          }
          if (ib < C) {
            const float2 f0 = Fc2[ib * nt];
            df_mac(Mh[ib], Ml[ib], f0.x, f0.y, r0h, r0l);
          }
          df_add(r0h, r0l, r1h, r1l);
          const float2 fa = Fc2[ia * nt];
          float rowh = 2.f * r0h, rowl = 2.f * r0l;   // exact
          df_mac(Mh[ia], Ml[ia], fa.x, fa.y, rowh, rowl);
          df_renorm(rowh, rowl);
          df_mac(fa.x, fa.y, rowh, rowl, qh, ql);
        }
        q = df_value(qh, ql);
      } else {
      // F M F^T over the upper triangle; four partial sums per row keep four
      // independent FP64 FMA chains in flight
      for (int ia = 0; ia < C; ++ia) {
        const double* Mr = Ms + ia * C;
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        int ib = ia + 1;
        for (; ib + 3 < C; ib += 4) {
          r0 = fma(Mr[ib], Fc[ib * nt], r0);
          r1 = fma(Mr[ib + 1], Fc[(ib + 1) * nt], r1);
          r2 = fma(Mr[ib + 2], Fc[(ib + 2) * nt], r2);
          r3 = fma(Mr[ib + 3], Fc[(ib + 3) * nt], r3);
        }
        for (; ib < C; ++ib) r0 = fma(Mr[ib], Fc[ib * nt], r0);
        const double fa = Fc[ia * nt];
        q = fma(fa, fma(2.0, (r0 + r1) + (r2 + r3), Mr[ia] * fa), q);
      }
      }
      const double dv = fc - sh[j];
      acc1[j] += fm + W * dv;
      acc2[j] += q + 2.0 * dv * fm + W * dv * dv;
    }
  }
#pragma unroll
  for (int j = 0; j < kBigE; ++j) {
    const int64_t el = e0 + threadIdx.x + (int64_t)j * nt;
    if (el >= n_ent) break;
    const int64_t ge = darcy_entry(S, m, s, el, 0, ny);
    m.part[((int64_t)slot * 2) * m.len_d + ge] = acc1[j];
    m.part[((int64_t)slot * 2 + 1) * m.len_d + ge] = acc2[j];
  }
}

// S1 += sum over chunks of the partials, S2 likewise (fixed order).
__global__ void reduce_partials(const double* part, int n_chunks, int64_t len, double* S1, double* S2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double a1 = 0.0, a2 = 0.0;
    for (int c = 0; c < n_chunks; ++c) {
      a1 += part[(int64_t)(2 * c) * len + e];
      a2 += part[(int64_t)(2 * c + 1) * len + e];
    }
    S1[e] += a1;
    S2[e] += a2;
  }
}

// Stokes fields: x_l = U [R_s lambda_l; 1] for every entry, so with
// d_l = c_l - c_0 (c_0: the coefficients of point 0 of the first batch) the
// shifted sums are U m and diag(U M U^T) with m = sum w d, M = sum w d d^T.
// One CTA per point chunk: partial m and M (4 x 4 register tiles of M, points
// staged 16 at a time), summed over the chunks in order by stokes_cov_reduce.
__global__ void __launch_bounds__(256) stokes_cov_kernel(const IfaceArgs a, const double* w, int first, double* c0,
                                                         double* part) {
  const int Rs = a.Rs, Cs = Rs + 1;
  const int ch = blockIdx.x;
  __shared__ double c0s[kMaxCols];
  __shared__ double Dl[16][kMaxCols + 3];
  __shared__ double Wl[16];
  for (int i = threadIdx.x; i < Cs; i += blockDim.x) {
    const double v = i < Rs ? a.lam[a.sgdof[i]] : 1.0;   // point 0
    c0s[i] = first ? v : c0[i];
  }
  __syncthreads();
  if (first && ch == 0)
    for (int i = threadIdx.x; i < Cs; i += blockDim.x) c0[i] = c0s[i];
  const int64_t per = (a.n_pts + kStokesChunks - 1) / kStokesChunks;
  const int64_t p0 = ch * per, p1 = min(a.n_pts, p0 + per);
  double* out = part + (int64_t)ch * (Cs + (int64_t)Cs * Cs);
  const int nt4 = (Cs + 3) >> 2;
  const int ntile = nt4 * nt4;
  for (int tb = 0; tb < ntile; tb += blockDim.x) {
    const int t = tb + threadIdx.x;
    const int a0 = (t / nt4) * 4, b0 = (t % nt4) * 4;
    double acc[4][4] = {};
    double accm = 0.0;
    for (int64_t q0 = p0; q0 < p1; q0 += 16) {
      const int nq = (int)min((int64_t)16, p1 - q0);
      __syncthreads();
      for (int e = threadIdx.x; e < nq * (Cs + 3); e += blockDim.x) {
        const int q = e / (Cs + 3), i = e - q * (Cs + 3);
        double v = 0.0;
        if (i < Cs) v = (i < Rs ? a.lam[(q0 + q) * a.n_lambda + a.sgdof[i]] : 1.0) - c0s[i];
        Dl[q][i] = v;
      }
      for (int q = threadIdx.x; q < nq; q += blockDim.x) Wl[q] = w[q0 + q];
      __syncthreads();
      if (t < ntile) {
        for (int q = 0; q < nq; ++q) {
          const double wq = Wl[q];
          double da[4], db[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) { da[i] = wq * Dl[q][a0 + i]; db[i] = Dl[q][b0 + i]; }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(da[i], db[j], acc[i][j]);
          if (tb == 0 && threadIdx.x < Cs) accm = fma(wq, Dl[q][threadIdx.x], accm);
        }
      }
    }
    if (t < ntile)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (a0 + i < Cs && b0 + j < Cs) out[Cs + (a0 + i) * Cs + b0 + j] = acc[i][j];
    if (tb == 0 && threadIdx.x < Cs) out[threadIdx.x] = accm;
  }
}

// m += sum of the chunk partials of m, M likewise, in chunk order.
__global__ void stokes_cov_reduce(const double* part, int Cs, double* mvec, double* Mmat) {
  const int64_t len = Cs + (int64_t)Cs * Cs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < kStokesChunks; ++c) v += part[c * len + e];
    if (e < Cs) mvec[e] += v;
    else Mmat[e - Cs] += v;
  }
}

// out += sum of the weights (one CTA; strided partial sums, then a fixed tree).
__global__ void weight_sum(const double* w, int64_t n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) s += w[l];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] += red[0];
}

// mean = shift W + S1, var = S2 - 2 (mean - shift) S1 + (mean - shift)^2 W
__global__ void finalize_darcy(const double* shift, const double* S1, const double* S2, int64_t off, int64_t n,
                               const double* W, double* mean, double* var) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double sh = shift[off + e], s1 = S1[off + e], s2 = S2[off + e], w = W[0];
    const double mu = sh * w + s1;
    const double dm = mu - sh;
    mean[e] = mu;
    var[e] = s2 - 2.0 * dm * s1 + dm * dm * w;
  }
}

// Stokes: shift = U_e c0, S1 = U_e m, S2 = U_e M U_e^T; one warp per entry.
__global__ void finalize_stokes(const double* U, int64_t n, int Cs, const double* c0, const double* mvec,
                                const double* Mmat, const double* W, double* mean, double* var) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= n) return;
  const double* u = U + e * Cs;
  double sh = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = lane; i < Cs; i += 32) {
    sh = fma(u[i], c0[i], sh);
    s1 = fma(u[i], mvec[i], s1);
    double row = 0.0;
    for (int j = 0; j < Cs; ++j) row = fma(Mmat[(int64_t)i * Cs + j], u[j], row);
    s2 = fma(u[i], row, s2);
  }
  sh = warp_sum(sh);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double w = W[0];
    const double mu = sh * w + s1;
    const double dm = mu - sh;
    mean[e] = mu;
    var[e] = s2 - 2.0 * dm * s1 + dm * dm * w;
  }
}

// ---- balancing Neumann-Neumann preconditioner ---------------------------------------------
// Section 7 suggests a balancing preconditioner (Mandel's balancing domain
// decomposition) to cut the interface CG's iterations. For S = sum_u R_u^T
// Phi_u R_u over the units (Darcy subdomains, then Stokes):
//  - weights D_u: at a mortar DOF shared by units u and v, u's share of the
//    two local stiffnesses, (Phi_u)_dd / ((Phi_u)_dd + (Phi_v)_dd), per point
//    (they depend on the point's items); sum_u R_u^T D_u R_u = I;
//  - Neumann step N r = sum_u R_u^T D_u Phi_u^+ D_u R_u r (the tile products
//    on the pseudo-inverses, weighted through IfaceArgs::wy);
//  - coarse space Z = [R_u^T D_u 1] over the floating Darcy subdomains (no
//    outer Dirichlet side), S_0 = Z^T S Z per point, Q = Z S_0^{-1} Z^T;
//  - CG from the balanced start lambda_0 = Q g, so that every residual stays
//    balanced (Z^T r = 0) and the preconditioned residual is
//    z = (I - Q S) N r = w - Z S_0^{-1} (S Z)^T w with w = N r.
// S Z is formed once per point by the tile products (n_c of them); each
// iteration then costs the product S p, the Neumann step and n_c dot products.
constexpr int kBddMaxCoarse = 16;

struct BddArgs {
  double* wy;          // [n_pts][NY] weights of each unit at its local DOFs
  double* sz;          // [n_pts][n_c][n_lambda] S Z
  double* L;           // [n_pts][n_c * n_c] Cholesky factor of S_0
  const int* cidx;     // [units] the coarse vector of each unit, or -1
  int n_c;
};

// Pseudo-inverse of one Darcy item's flux basis: Phi^{-1}, or for a floating
// subdomain (null space the constants) (Phi + (a/R) 1 1^T)^{-1} - 1 1^T/(a R)
// with a = trace(Phi)/R. Gauss-Jordan sweep of the SPD matrix in shared
// memory (after all R pivots it holds -A^{-1}); a non-positive pivot sets bad.
__global__ void __launch_bounds__(256) bdd_pinv_kernel(const SubDev* subs, const ItemOff* off, const int* item_sub,
                                                        const int* item_k, int n_items, const double* phi,
                                                        double* pinv, int* bad) {
  extern __shared__ __align__(16) double bsm[];
  const int item = blockIdx.x;
  if (item >= n_items) return;
  const SubDev& S = subs[item_sub[item]];
  const int64_t po = off[S.item0 + item_k[item]].phi;
  const int R = S.R;
  bool floating = true;
  for (int q = 0; q < 4; ++q) floating = floating && S.side_type[q] != SIDE_DIRICHLET;
  double* A = bsm;            // [R][R]
  double* col = A + R * R;    // pivot column
  __shared__ double shift;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) A[e] = phi[po + e];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < R; ++i) tr += A[i * R + i];
    shift = floating ? tr / ((double)R * R) : 0.0;
  }
  __syncthreads();
  if (floating)
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) A[e] += shift;
  __syncthreads();
  for (int k = 0; k < R; ++k) {
    for (int i = threadIdx.x; i < R; i += blockDim.x) col[i] = A[i * R + k];
    __syncthreads();
    double d = col[k];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicOr(bad, 1);
      d = 1.0;
    }
    const double id = 1.0 / d;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const int i = e / R, j = e - i * R;
      double v;
      if (i == k && j == k) v = -id;
      else if (i == k) v = col[j] * id;
      else if (j == k) v = col[i] * id;
      else v = A[e] - col[i] * col[j] * id;
      A[e] = v;
    }
    __syncthreads();
  }
  // A = -(Phi + shift 1 1^T)^{-1}; with shift = a/R, the constant term of the
  // pseudo-inverse is 1/(a R) = 1/(shift R^2)
  const double c = floating ? 1.0 / (shift * (double)R * R) : 0.0;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) pinv[po + e] = -A[e] - c;
}

// wy: each unit's share of the local stiffness at each of its DOFs.
__global__ void bdd_weights_kernel(IfaceArgs a, BddArgs b) {
  const int64_t tot = a.n_pts * a.n_lambda;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / a.n_lambda;
    const int d = (int)(e - l * a.n_lambda);
    if (a.pstat[l] & 0x40000000) continue;
    double dg[2];
    for (int side = 0; side < 2; ++side) {
      const int u = a.ldof[4 * d + 2 * side], loc = a.ldof[4 * d + 2 * side + 1];
      const int k = u < a.ns ? a.kmap[l * a.ns + u] : 0;
      int R;
      const double* ph = unit_phi(a, u, k, R);
      dg[side] = ph[(int64_t)loc * R + loc];
    }
    const double tot2 = dg[0] + dg[1];
    for (int side = 0; side < 2; ++side)
      b.wy[l * a.NY + a.yoff[2 * d + side]] = tot2 > 0.0 ? dg[side] / tot2 : 0.5;
  }
}

// Entry d of coarse vector j at point l: the weight at d of the unit whose
// coarse vector is j, or 0.
__device__ __forceinline__ double coarse_entry(const IfaceArgs& a, const BddArgs& b, int64_t l, int d, int j) {
  double v = 0.0;
  for (int side = 0; side < 2; ++side)
    if (b.cidx[a.ldof[4 * d + 2 * side]] == j) v = b.wy[l * a.NY + a.yoff[2 * d + side]];
  return v;
}

// (Z t)_d: the coarse combination at DOF d (at most its two units contribute).
__device__ __forceinline__ double coarse_comb(const IfaceArgs& a, const BddArgs& b, int64_t l, int d,
                                              const double* t) {
  double v = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int j = b.cidx[a.ldof[4 * d + 2 * side]];
    if (j >= 0) v = fma(t[j], b.wy[l * a.NY + a.yoff[2 * d + side]], v);
  }
  return v;
}

// vout = coarse vector j of every point
__global__ void bdd_coarse_vec_kernel(IfaceArgs a, BddArgs b, int j, double* vout) {
  const int64_t tot = a.n_pts * a.n_lambda;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / a.n_lambda;
    const int d = (int)(e - l * a.n_lambda);
    vout[e] = (a.pstat[l] & 0x40000000) ? 0.0 : coarse_entry(a, b, l, d, j);
  }
}

// column j of S Z: the gathered tile products
__global__ void bdd_gather_kernel(IfaceArgs a, BddArgs b, int j) {
  const int64_t tot = a.n_pts * a.n_lambda;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / a.n_lambda;
    const int d = (int)(e - l * a.n_lambda);
    const double* Yl = a.Y + l * a.NY;
    b.sz[(l * b.n_c + j) * a.n_lambda + d] = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]];
  }
}

// y = S_0^{-1} t in place with the Cholesky factor L (row-major, lower), one lane.
__device__ __forceinline__ void chol_solve(const double* L, int n, double* y) {
  for (int i = 0; i < n; ++i) {
    double v = y[i];
    for (int k = 0; k < i; ++k) v -= L[i * n + k] * y[k];
    y[i] = v / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * y[k];
    y[i] = v / L[i * n + i];
  }
}

// One warp per point: S_0 = Z^T (S Z), its Cholesky factor, then the balanced
// start lambda_0 = Z S_0^{-1} Z^T g and r_0 = g - (S Z) S_0^{-1} Z^T g (r holds
// g on entry). A non-positive pivot of S_0 fails the point.
__global__ void bdd_setup_kernel(IfaceArgs a, BddArgs b) {
  __shared__ double s0[8][kBddMaxCoarse * kBddMaxCoarse];
  __shared__ double tv[8][kBddMaxCoarse];
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  if (l >= a.n_pts) return;
  if (a.pstat[l] != 0) return;
  const int nc = b.n_c, n = (int)a.n_lambda;
  const double* sz = b.sz + l * nc * a.n_lambda;
  double* rl = a.r + l * a.n_lambda;
  double* ll = a.lam + l * a.n_lambda;
  for (int ab = 0; ab < nc * nc + nc; ++ab) {
    const int ia = ab < nc * nc ? ab / nc : ab - nc * nc, ib = ab < nc * nc ? ab % nc : -1;
    double acc = 0.0;
    for (int d = lane; d < n; d += 32) {
      const double ca = coarse_entry(a, b, l, d, ia);
      if (ca != 0.0) acc = fma(ca, ib >= 0 ? sz[ib * a.n_lambda + d] : rl[d], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      if (ib >= 0) s0[wl][ab] = acc;
      else tv[wl][ia] = acc;
    }
  }
  __syncwarp();
  int ok = 1;
  if (lane == 0) {
    double* S0 = s0[wl];
    for (int i = 0; i < nc; ++i)   // symmetrize (rounding) and factor in place
      for (int j = 0; j < i; ++j) S0[i * nc + j] = S0[j * nc + i] = 0.5 * (S0[i * nc + j] + S0[j * nc + i]);
    for (int j = 0; j < nc && ok; ++j) {
      double dj = S0[j * nc + j];
      for (int k = 0; k < j; ++k) dj -= S0[j * nc + k] * S0[j * nc + k];
      if (!(dj > 0.0)) { ok = 0; break; }
      const double ljj = sqrt(dj);
      S0[j * nc + j] = ljj;
      for (int i = j + 1; i < nc; ++i) {
        double v = S0[i * nc + j];
        for (int k = 0; k < j; ++k) v -= S0[i * nc + k] * S0[j * nc + k];
        S0[i * nc + j] = v / ljj;
      }
    }
    if (ok) {
      for (int e = 0; e < nc * nc; ++e) b.L[l * nc * nc + e] = S0[e];
      chol_solve(S0, nc, tv[wl]);
    } else {
      a.pstat[l] = -1;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  if (!ok) return;
  for (int d = lane; d < n; d += 32) {
    double sv = 0.0;
    for (int j = 0; j < nc; ++j) sv = fma(tv[wl][j], sz[j * a.n_lambda + d], sv);
    ll[d] = coarse_comb(a, b, l, d, tv[wl]);
    rl[d] -= sv;
  }
}

// One warp per iterating point: q = S p from the tile products, alpha =
// (r.z)/(p.q), lambda += alpha p, r -= alpha q, and the stopping test
// ||r|| <= rtol ||g|| (the point's status becomes its iteration count, negative
// after a breakdown p.q <= 0).
__global__ void bdd_update1_kernel(IfaceArgs a, int it, double rtol) {
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= a.n_pts || a.pstat[l] != 0) return;
  const double* Yl = a.Y + l * a.NY;
  const double* pl = a.p + l * a.n_lambda;
  double* rl = a.r + l * a.n_lambda;
  double* ll = a.lam + l * a.n_lambda;
  const int n = (int)a.n_lambda;
  double pq = 0.0;
  for (int d = lane; d < n; d += 32) pq = fma(pl[d], Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]], pq);
  pq = warp_sum(pq);
  const bool brk = !(pq > 0.0);
  const double alpha = brk ? 0.0 : a.rr[l] / pq;
  double rn = 0.0;
  for (int d = lane; d < n; d += 32) {
    const double q = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]];
    ll[d] = fma(alpha, pl[d], ll[d]);
    const double rv = fma(-alpha, q, rl[d]);
    rl[d] = rv;
    rn = fma(rv, rv, rn);
  }
  rn = warp_sum(rn);
  if (lane == 0 && (brk || sqrt(rn) <= rtol * a.gn[l])) a.pstat[l] = brk ? -(it + 1) : it + 1;
}

// One warp per iterating point: w = N r from the weighted tile products on the
// pseudo-inverses, z = w - Z S_0^{-1} (S Z)^T w, then p = z (first) or
// p = z + (r.z / rr) p, rr = r.z (z is formed twice: for r.z, then for p).
__global__ void bdd_update2_kernel(IfaceArgs a, BddArgs b, int first) {
  __shared__ double tv[8][kBddMaxCoarse];
  const int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  if (l >= a.n_pts || a.pstat[l] != 0) return;
  const double* Yl = a.Y + l * a.NY;
  const int nc = b.n_c, n = (int)a.n_lambda;
  const double* sz = b.sz + l * nc * a.n_lambda;
  double* pl = a.p + l * a.n_lambda;
  const double* rl = a.r + l * a.n_lambda;
  for (int j = 0; j < nc; ++j) {
    double acc = 0.0;
    for (int d = lane; d < n; d += 32)
      acc = fma(sz[j * a.n_lambda + d], Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]], acc);
    acc = warp_sum(acc);
    if (lane == 0) tv[wl][j] = acc;
  }
  __syncwarp();
  if (lane == 0 && nc > 0) chol_solve(b.L + l * nc * nc, nc, tv[wl]);
  __syncwarp();
  double rz = 0.0;
  for (int d = lane; d < n; d += 32) {
    const double z = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]] - coarse_comb(a, b, l, d, tv[wl]);
    rz = fma(rl[d], z, rz);
  }
  rz = warp_sum(rz);
  double beta = 0.0;
  if (!first && lane == 0) beta = a.rr[l] > 0.0 ? rz / a.rr[l] : 0.0;
  beta = __shfl_sync(0xffffffffu, beta, 0);
  for (int d = lane; d < n; d += 32) {
    const double z = Yl[a.yoff[2 * d]] + Yl[a.yoff[2 * d + 1]] - coarse_comb(a, b, l, d, tv[wl]);
    pl[d] = first ? z : fma(beta, pl[d], z);
  }
  if (lane == 0) a.rr[l] = rz;
}

}  // namespace

// ---- host orchestration -----------------------------------------------------------------
void build_hash_tables(sfb_ctx* c, std::vector<int>& table, std::vector<int64_t>& off, std::vector<int>& cap) {
  const int ns = (int)c->subs.size();
  table.clear(); off.assign(ns, 0); cap.assign(ns, 0);
  for (int s = 0; s < ns; ++s) {
    int cp = 1;
    while (cp < 2 * c->n_local[s] + 1) cp <<= 1;
    off[s] = (int64_t)table.size();
    cap[s] = cp;
    table.resize(table.size() + cp, -1);
    const int nt = c->subs[s].n_term;
    for (int k = 0; k < c->n_local[s]; ++k) {
      uint64_t h = 1469598103934665603ull;
      for (int j = 0; j < nt; ++j) h = mix_key(h, qkey(c->loc_y[s][(size_t)k * nt + j]));
      h = fin_key(h);
      for (int probe = 0; probe < cp; ++probe) {
        const int slot = (int)((h + probe) & (uint64_t)(cp - 1));
        if (table[off[s] + slot] < 0) { table[off[s] + slot] = k; break; }
      }
    }
  }
}

static IfaceArgs make_args(sfb_ctx* c, int64_t n_pts) {
  Dev& d = c->dev;
  IfaceArgs a;
  a.subs = d.subs; a.ns = (int)c->subs.size(); a.off = d.off; a.phi = d.phi; a.s_phi = d.s_phi;
  a.phi32 = d.phi32; a.s_phi32 = d.s_phi32;
  a.Rs = (int)c->stokes.dofs.size(); a.gdof = d.gdof; a.sgdof = d.s_gdof; a.ybase = d.ybase; a.NY = c->NY;
  a.ldof = d.ldof; a.yoff = d.yoff; a.n_lambda = c->n_lambda; a.kmap = d.kmap; a.grp_pts = d.grp_pts; a.pts_ld = c->ws_pts;
  a.tiles = d.tiles; a.max_tiles = c->max_tiles; a.n_tiles = d.n_tiles; a.lam = d.lam; a.r = d.r; a.p = d.p;
  a.Y = d.Y; a.rr = d.rr; a.gn = d.gn; a.rlast = d.rlast; a.rflag = d.rflag; a.pstat = d.pstat; a.n_pts = n_pts;
  // interface blocks wider than kBlkMax DOFs fall back to the Jacobi preconditioner
  const bool blocks = c->opt_cg_precond == 2 && c->max_if_dof <= kBlkMax;
  a.dinv = (c->opt_cg_precond == 1 || (c->opt_cg_precond == 2 && !blocks)) ? d.dinv : nullptr;
  a.minv = blocks ? d.minv : nullptr;
  a.minv_ld = c->minv_ld;
  a.n_if = (int)c->ifaces.size();
  a.if_off = d.if_off; a.if_n = d.if_n; a.if_moff = d.if_moff; a.dof_if = d.dof_if;
  return a;
}

// Moore-Penrose pseudo-inverse of a symmetric n x n matrix (row-major) on the
// host: cyclic Jacobi rotations to diagonal form (Golub and Van Loan, Section
// 8.5), then V diag(1/e) V^T over the eigenvalues e above rcut max|e|.
static void sym_pinv_host(const std::vector<double>& A0, int n, double rcut, std::vector<double>& out) {
  std::vector<double> A(A0), V((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double v : A) fro += v * v;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off <= 1e-30 * fro) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {   // V <- V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = cs * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  double emax = 0.0;
  for (int i = 0; i < n; ++i) emax = std::max(emax, std::fabs(A[(size_t)i * n + i]));
  out.assign((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    const double e = A[(size_t)k * n + k];
    if (!(std::fabs(e) > rcut * emax)) continue;
    for (int i = 0; i < n; ++i) {
      const double vi = V[(size_t)i * n + k] / e;
      for (int j = 0; j < n; ++j) out[(size_t)i * n + j] += vi * V[(size_t)j * n + k];
    }
  }
}

__global__ void count_failed(const int* pstat, int64_t n, int* out) {
  int c = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n; l += (int64_t)gridDim.x * blockDim.x)
    c += pstat[l] < 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

sfb_status iface_solve_device(sfb_ctx* c, int64_t n_pts, double rtol, int max_it, int krylov, int* n_failed) {
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  const int ns = (int)c->subs.size();
  const int nu = ns + 1;
  cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) { c->err = std::string("interface solve: ") + cudaGetErrorString(e); return SFB_ERR_CUDA; } } while (0)
  for (int q = 0; q < 6; ++q)
    if (!c->ev[q]) CK(cudaEventCreate(&c->ev[q]));
  CK(cudaEventRecord(c->ev[0], st));
  CK(cudaMemsetAsync(d.pstat, 0, sizeof(int) * n_pts, st));
  CK(cudaMemsetAsync(d.active, 0, sizeof(int) * 4, st));
  const int64_t tot = n_pts * ns;
  kmap_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, st>>>(
      d.y, n_pts, c->grid.n_dim, d.subs, ns, d.dim_off, d.yloc, d.hash, d.hash_off, d.hash_cap, d.kmap, d.pstat);
  ++c->launches;
  CK(cudaGetLastError());
  group_kernel<<<ns, 256, 0, st>>>(d.kmap, n_pts, ns, d.subs, d.loc_off, d.grp_count, d.grp_start, d.grp_pts,
                                   c->ws_pts, d.tiles, c->max_tiles, d.n_tiles);
  ++c->launches;
  stokes_group_kernel<<<64, 256, 0, st>>>(n_pts, ns, d.grp_pts, c->ws_pts, d.tiles, c->max_tiles, d.n_tiles);
  ++c->launches;
  CK(cudaGetLastError());
  IfaceArgs a = make_args(c, n_pts);
  // Method S1: unpreconditioned FP64 CG, the Darcy units' products by subdomain solves
  const bool dtn = krylov == SFB_CG_DTN;
  if (dtn) { a.dinv = nullptr; a.minv = nullptr; }
  c->last_dtn = dtn;
  // balancing preconditioner (FP64 CG): the pseudo-inverses of the bases,
  // once per build (Darcy items) and per Stokes basis
  const bool bdd = krylov == SFB_CG && c->opt_cg_precond == 3;
  if (bdd) {
    if (!c->bdd_items_ready && c->n_items > 0) {
      int maxR = 1;
      for (const HostSub& S : c->subs) maxR = std::max(maxR, (int)S.dofs.size());
      const size_t smp = sizeof(double) * ((size_t)maxR * maxR + maxR);
      CK(cudaFuncSetAttribute(bdd_pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp));
      CK(cudaMemsetAsync(d.active + 9, 0, sizeof(int), st));
      bdd_pinv_kernel<<<(unsigned)c->n_items, 256, smp, st>>>(d.subs, d.off, d.item_sub, d.item_k, (int)c->n_items,
                                                             d.phi, d.bdd_pinv, d.active + 9);
      ++c->launches;
      CK(cudaGetLastError());
      c->bdd_items_ready = true;
    }
    if (!c->bdd_stokes_ready) {
      const int Rs = (int)c->stokes.dofs.size();
      std::vector<double> ph((size_t)Rs * Rs), pi;
      CK(cudaMemcpyAsync(ph.data(), d.s_phi, sizeof(double) * ph.size(), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      sym_pinv_host(ph, Rs, 1e-10, pi);
      CK(cudaMemcpyAsync(d.bdd_spinv, pi.data(), sizeof(double) * pi.size(), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
      c->bdd_stokes_ready = true;
    }
  }
  CK(cudaEventRecord(c->ev[1], st));
  const int warps_per_block = 8;
  const int ublocks = (int)((n_pts + warps_per_block - 1) / warps_per_block);
  const size_t stg = a.minv ? sizeof(float) * warps_per_block * (size_t)c->n_lambda : 0;
  if (stg > 48 * 1024) {
    CK(cudaFuncSetAttribute(init_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stg));
    CK(cudaFuncSetAttribute(update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stg));
    CK(cudaFuncSetAttribute(update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stg));
    CK(cudaFuncSetAttribute(reliable_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stg));
  }
  if (a.minv) {
    const int64_t warps = n_pts * a.n_if;
    bjacobi_setup_kernel<<<(int)((warps + 7) / 8), 256, 0, st>>>(a);
    ++c->launches;
    CK(cudaGetLastError());
  }
  const bool gmres = krylov == SFB_GMRES || krylov == SFB_GMRES_MIXED;
  const bool gmres_mixed = krylov == SFB_GMRES_MIXED;
  GmArgs gma;
  gma.V = d.gmV; gma.st = d.gmS; gma.j = d.gmJ; gma.m = c->opt_gmres_m;
  // mixed GMRES: the FP32 products limit what one cycle can resolve; a cycle
  // ends once it has gained this factor, and the FP64 true residual restarts it
  gma.cycle_tol = gmres_mixed ? 1e-5 : 0.0;
  if (gmres) {
    CK(cudaMemsetAsync(d.rflag, 0, sizeof(int) * n_pts, st));
    if (gmres_mixed) gmres_init_kernel<float><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma);
    else gmres_init_kernel<double><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma);
  } else {
    init_kernel<<<ublocks, 32 * warps_per_block, stg, st>>>(a);
  }
  ++c->launches;
  CK(cudaGetLastError());
  int maxR = (int)c->stokes.dofs.size();
  for (const HostSub& S : c->subs) maxR = std::max(maxR, (int)S.dofs.size());
  const size_t smv = sizeof(double) * ((size_t)((maxR * maxR + 3) & ~3) + (size_t)(kTG + 1) * maxR);
  const size_t smv32 = sizeof(float) * ((size_t)((maxR * maxR + 3) & ~3) + (size_t)(kTG + 1) * maxR);
  CK(cudaFuncSetAttribute(matvec_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv));
  CK(cudaFuncSetAttribute(matvec_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv32));
  dim3 mgrid(c->max_tiles, nu);
  // balancing preconditioner: weights, S Z (one round of tile products per
  // coarse vector), S_0 and the balanced start, then z_0 = (I - Q S) N r_0
  BddArgs bdda;
  bdda.wy = d.bdd_wy; bdda.sz = d.bdd_sz; bdda.L = d.bdd_L; bdda.cidx = d.bdd_cidx; bdda.n_c = c->bdd_nc;
  IfaceArgs ai = a;   // the Neumann step: tile products on the pseudo-inverses, weighted
  ai.phi = d.bdd_pinv; ai.s_phi = d.bdd_spinv; ai.wy = d.bdd_wy;
  if (bdd) {
    const int eb = (int)std::min<int64_t>((n_pts * c->n_lambda + 255) / 256, 8192);
    bdd_weights_kernel<<<eb, 256, 0, st>>>(a, bdda);
    ++c->launches;
    for (int j = 0; j < bdda.n_c; ++j) {
      bdd_coarse_vec_kernel<<<eb, 256, 0, st>>>(a, bdda, j, d.p);
      matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.p, 0, d.active + 2, 0);
      bdd_gather_kernel<<<eb, 256, 0, st>>>(a, bdda, j);
      c->launches += 3;
    }
    bdd_setup_kernel<<<ublocks, 32 * warps_per_block, 0, st>>>(a, bdda);
    matvec_kernel<double><<<mgrid, 256, smv, st>>>(ai, d.r, 0, d.active + 2, 0);
    bdd_update2_kernel<<<ublocks, 32 * warps_per_block, 0, st>>>(a, bdda, 1);
    c->launches += 3;
    CK(cudaGetLastError());
  }
  const int chunk = c->opt_cg_chunk;
  const bool mixed = krylov == SFB_CG_MIXED;
  const double replace_ratio = c->opt_cg_replace, pause_ratio = 0.1 * c->opt_cg_replace;
  const bool regs = c->n_lambda <= 32 * kUpd;
  // the persistent CG: one cooperative launch when the device supports it and
  // its shared memory fits (for the mixed CG: when its FP32 tiles can stay
  // resident); otherwise one launch per step below
  bool persistent = false;
  if (c->opt_cg_persistent && nu <= kPcgUnits && !gmres && !dtn && !bdd) {
    int dev = 0, coop = 0, n_sm = 0, smem_max = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const void* fn = mixed ? (regs ? (const void*)cg_persistent_kernel<float, true> : (const void*)cg_persistent_kernel<float, false>)
                           : (regs ? (const void*)cg_persistent_kernel<double, true> : (const void*)cg_persistent_kernel<double, false>);
    // the flat tile list and each tile's cost (4 x 4 product items times R,
    // plus its gather), for the resident partition of the mixed CG
    int ntot = 0;
    std::vector<double> cost;
    if (mixed && coop) {
      std::vector<int> h_nt((size_t)nu), h_tl((size_t)nu * c->max_tiles * 3);
      CK(cudaMemcpyAsync(h_nt.data(), d.n_tiles, sizeof(int) * nu, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(h_tl.data(), d.tiles, sizeof(int) * h_tl.size(), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int u = 0; u < nu; ++u) {
        const int R = u == ns ? (int)c->stokes.dofs.size() : (int)c->subs[(size_t)u].dofs.size();
        const int R4 = (R + 3) & ~3;
        for (int t = 0; t < std::min(h_nt[(size_t)u], c->max_tiles); ++t) {
          const int cnt = h_tl[3 * ((size_t)u * c->max_tiles + t) + 2];
          const int c4 = (cnt + 3) & ~3;
          cost.push_back((double)R4 * c4 * R / 16.0 + (double)R * cnt / 8.0 + 64.0);
        }
      }
      ntot = (int)cost.size();
    }
    // contiguous ranges of at most cap tiles for grid CTAs, the largest range
    // cost as small as the greedy cut allows (bisection on the bound)
    auto partition = [&](int grid, int cap, std::vector<int>& starts) -> bool {
      auto cut = [&](double bound) -> bool {
        starts.assign(1, 0);
        double acc = 0.0;
        int n = 0;
        for (int j = 0; j < ntot; ++j) {
          if (n > 0 && (acc + cost[(size_t)j] > bound || n == cap)) {
            starts.push_back(j);
            if ((int)starts.size() > grid) return false;
            acc = 0.0;
            n = 0;
          }
          acc += cost[(size_t)j];
          ++n;
        }
        while ((int)starts.size() <= grid) starts.push_back(ntot);
        return true;
      };
      double lo = 0.0, hi = 0.0;
      for (double v : cost) { lo = std::max(lo, v); hi += v; }
      if (!cut(hi)) return false;
      for (int k = 0; k < 40; ++k) {
        const double mid = 0.5 * (lo + hi);
        if (cut(mid)) hi = mid; else lo = mid;
      }
      return cut(hi);
    };
    auto layout = [&](int grid, bool res, int nbuf, PcgLayout& L) -> size_t {
      size_t off = 0;
      auto put = [&](size_t bytes) {
        off = (off + 15) & ~(size_t)15;
        const size_t o = off;
        off += bytes;
        return (int)o;
      };
      L.phi_bytes = (int)((sizeof(double) * (size_t)maxR * maxR + 15) & ~(size_t)15);
      L.nbuf = nbuf;
      put((size_t)nbuf * L.phi_bytes);
      L.r4 = (maxR + 3) & ~3;
      L.resident = res ? 1 : 0;
      L.part = d.pcg_part;
      const int m = res ? kResMax3 : 0;
      const size_t pv64 = sizeof(double) * (size_t)maxR * (kTG + 1);
      const size_t rpv = sizeof(float) * (size_t)m * L.r4 * kPvS;
      L.rphi_off = put(sizeof(float) * (size_t)m * L.r4 * L.r4);
      L.rpv_off = put(std::max(rpv, pv64));
      L.pv_off = L.rpv_off;   // the streaming vectors reuse the resident ones (never live at once)
      L.rpts_off = put(sizeof(int) * (size_t)m * kTG);
      L.rspt_off = put(sizeof(int64_t) * (size_t)m * kTG);
      L.rgd_off = put(sizeof(int) * (size_t)m * L.r4);
      // the FP32 stage of the block preconditioner (update and residual steps)
      // reuses the gathered-vector block (product steps): a grid barrier
      // always separates the two
      L.stage_off = stg <= std::max(rpv, pv64) ? L.rpv_off : put(stg);
      return off;
    };
    // candidates, best first: CTAs per SM, resident tiles, streaming buffers
    const int cand[7][3] = {{2, 1, 2}, {2, 1, 1}, {1, 1, 2}, {1, 1, 1}, {2, 0, 2}, {1, 0, 2}, {1, 0, 1}};
    for (int ci = 0; ci < 7 && coop && !persistent; ++ci) {
      const int per = cand[ci][0], nbuf = cand[ci][2];
      const bool res = cand[ci][1] == 1;
      if (res && !(mixed && ntot > 0)) continue;
      // the mixed CG's streaming form measured slower than a launch per step
      if (mixed && !res) continue;
      const int grid = n_sm * per;
      std::vector<int>& starts = c->pcg_starts;
      if (res && (grid > kPcgMaxGrid || !partition(grid, kResMax3, starts))) continue;
      PcgLayout L;
      const size_t smp = layout(grid, res, nbuf, L);
      if (smp + 4096 > (size_t)smem_max) continue;
      CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp));
      int per_sm = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smp));
      if (per_sm < per) continue;
      PcgCtl ctl;
      ctl.bar = reinterpret_cast<unsigned*>(d.active + 4);
      ctl.abort = d.active + 6;
      ctl.iters = d.active + 7;
      ctl.act = d.active + 8;
      ctl.err = d.active + 2;
      ctl.cyc = reinterpret_cast<unsigned long long*>(d.active + 16);
      ctl.test_skip = c->test_barrier_skip;
      c->test_barrier_skip = 0;   // one solve only
      CK(cudaMemsetAsync(d.active + 4, 0, sizeof(int) * 28, st));
      if (res)
        CK(cudaMemcpyAsync(d.pcg_part, starts.data(), sizeof(int) * (grid + 1), cudaMemcpyHostToDevice, st));
      c->pcg_grid = grid;
      c->pcg_mode = (res ? 1 : 0) + 2 * (nbuf - 1);
      double rt_ = rtol, rr_ = replace_ratio, pr_ = pause_ratio;
      int mi = max_it, ch = chunk;
      void* args[] = {&a, &ctl, &rt_, &mi, &ch, &rr_, &pr_, &L};
      CK(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, smp, st));
      ++c->launches;
      persistent = true;
    }
  }
  int it = 0;
  // GMRES: chunks of Arnoldi steps, then the true residuals of the points
  // whose cycle ended (accepted, or the next cycle)
  for (; gmres && it < max_it;) {
    for (int q = 0; q < chunk && it < max_it; ++q, ++it) {
      if (gmres_mixed) matvec_kernel<float><<<mgrid, 256, smv32, st>>>(a, d.p, 0, d.active + 2, 0);
      else matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.p, 0, d.active + 2, 0);
      if (gmres_mixed) gmres_arnoldi_kernel<float><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma, it, rtol);
      else gmres_arnoldi_kernel<double><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma, it, rtol);
      c->launches += 2;
    }
    matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.lam, 1, d.active + 2, 0);
    if (gmres_mixed) gmres_restart_kernel<float><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma, rtol);
    else gmres_restart_kernel<double><<<ublocks, 32 * warps_per_block, 0, st>>>(a, gma, rtol);
    c->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(d.active, 0, sizeof(int), st));
    count_active<<<std::min(1024, (int)((n_pts + 255) / 256)), 256, 0, st>>>(d.pstat, n_pts, d.active);
    ++c->launches;
    int h_active = 0;
    CK(cudaMemcpyAsync(&h_active, d.active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_active == 0) break;
  }
  // balanced CG: product, update, Neumann step, preconditioned direction
  for (; bdd && it < max_it;) {
    for (int q = 0; q < chunk && it < max_it; ++q, ++it) {
      matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.p, 0, d.active + 2, 0);
      bdd_update1_kernel<<<ublocks, 32 * warps_per_block, 0, st>>>(a, it, rtol);
      matvec_kernel<double><<<mgrid, 256, smv, st>>>(ai, d.r, 0, d.active + 2, 0);
      bdd_update2_kernel<<<ublocks, 32 * warps_per_block, 0, st>>>(a, bdda, 0);
      c->launches += 4;
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(d.active, 0, sizeof(int), st));
    count_active<<<std::min(1024, (int)((n_pts + 255) / 256)), 256, 0, st>>>(d.pstat, n_pts, d.active);
    ++c->launches;
    int h_active = 0;
    CK(cudaMemcpyAsync(&h_active, d.active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_active == 0) break;
  }
  for (; it < max_it && !persistent && !gmres && !bdd;) {
    for (int q = 0; q < chunk && it < max_it; ++q, ++it) {
      if (dtn) {
        // Darcy units by one subdomain solve per (point, subdomain); the Stokes unit by its basis
        CK(launch_dtn(c, d.p, 0, n_pts, 0, nullptr, st));
        matvec_kernel<double><<<dim3(c->max_tiles, 1), 256, smv, st>>>(a, d.p, 0, d.active + 2, ns);
      } else if (mixed) {
        matvec_kernel<float><<<mgrid, 256, smv32, st>>>(a, d.p, 0, d.active + 2, 0);
      } else {
        matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.p, 0, d.active + 2, 0);
      }
      ++c->launches;
      if (regs)
        update_kernel<true><<<ublocks, 32 * warps_per_block, stg, st>>>(a, it, rtol, mixed ? 1 : 0, replace_ratio,
                                                                      pause_ratio);
      else
        update_kernel<false><<<ublocks, 32 * warps_per_block, stg, st>>>(a, it, rtol, mixed ? 1 : 0, replace_ratio,
                                                                       pause_ratio);
      ++c->launches;
    }
    if (mixed) {
      // FP64 residuals of the points that asked for one
      matvec_kernel<double><<<mgrid, 256, smv, st>>>(a, d.lam, 1, d.active + 2, 0);
      ++c->launches;
      reliable_kernel<<<ublocks, 32 * warps_per_block, stg, st>>>(a, rtol, it);
      ++c->launches;
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(d.active, 0, sizeof(int), st));
    count_active<<<std::min(1024, (int)((n_pts + 255) / 256)), 256, 0, st>>>(d.pstat, n_pts, d.active);
    ++c->launches;
    int h_active = 0;
    CK(cudaMemcpyAsync(&h_active, d.active, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_active == 0) break;
  }
  CK(cudaEventRecord(c->ev[2], st));
  finish_status<<<std::min(1024, (int)((n_pts + 255) / 256)), 256, 0, st>>>(d.pstat, n_pts, max_it, nullptr);
  ++c->launches;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(d.active + 1, 0, sizeof(int), st));
  count_failed<<<std::min(1024, (int)((n_pts + 255) / 256)), 256, 0, st>>>(d.pstat, n_pts, d.active + 1);
  ++c->launches;
  int h_flags[32] = {};
  CK(cudaMemcpyAsync(h_flags, d.active, sizeof(int) * 32, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int k = 0; k < 6; ++k) {
    unsigned long long v;
    std::memcpy(&v, h_flags + 16 + 2 * k, sizeof(v));
    c->pcg_cycles[k] = persistent ? (double)v / c->pcg_grid : 0.0;
  }
  *n_failed = h_flags[1];
  c->cg_iters_run = persistent ? h_flags[7] : it;
  c->cg_persistent_run = persistent;
  if (h_flags[2]) {
    c->err = "interface solve: a bulk copy of a basis did not complete within the wait limit";
    return SFB_ERR_TIMEOUT;
  }
  if (bdd && h_flags[9]) {
    c->err = "interface solve: a non-positive pivot inverting a flux basis for the balancing preconditioner";
    return SFB_ERR_NOT_SPD;
  }
  if (persistent && h_flags[6]) {
    c->err = "interface solve: a grid barrier of the persistent CG did not complete within the wait limit";
    return SFB_ERR_TIMEOUT;
  }
  return SFB_OK;
#undef CK
}

sfb_status moments_accumulate_device(sfb_ctx* c, int64_t n_pts) {
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  const int ns = (int)c->subs.size();
  cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) { c->err = std::string("moments: ") + cudaGetErrorString(e); return SFB_ERR_CUDA; } } while (0)
  // SFB_SYNC_CHECK=1: synchronise after every launch and name the kernel that failed
  static const bool sync_check = getenv("SFB_SYNC_CHECK") && getenv("SFB_SYNC_CHECK")[0] == '1';
#define LAUNCHED(name)                                                                         \
  do {                                                                                         \
    ++c->launches;                                                                             \
    if (sync_check) {                                                                          \
      e = cudaStreamSynchronize(st);                                                           \
      if (e == cudaSuccess) e = cudaGetLastError();                                            \
      if (e != cudaSuccess) {                                                                  \
        c->err = std::string("moments kernel ") + name + ": " + cudaGetErrorString(e);         \
        return SFB_ERR_CUDA;                                                                   \
      }                                                                                        \
    }                                                                                          \
  } while (0)
  MomArgs m;
  m.ia = make_args(c, n_pts);
  m.X = d.X; m.T = d.T; m.proj = d.proj; m.w = d.w;
  m.len_d = c->mom_len[0] + c->mom_len[1];
  m.off_f = c->mom_len[0];
  m.shift = d.mom; m.part = d.mom_part;
  m.cell_off = d.cell_off; m.face_off = d.face_off;
  int max_ny = 0, max_nx = 0, maxC = 0;
  for (const HostSub& S : c->subs) {
    max_ny = std::max(max_ny, S.ny); max_nx = std::max(max_nx, S.nx);
    maxC = std::max(maxC, (int)S.dofs.size() + 1);
  }
  // rows per CTA: about 512 cells, so the owned entries fit kMaxE per thread
  m.rt = std::max(1, std::min(max_ny, 512 / max_nx));
  m.n_chunks = c->mom_chunks;
  m.big_factor = c->opt_big_factor;
  m.grp_start = d.grp_start; m.grp_end = d.grp_count; m.loc_off = d.loc_off;
  m.gmom = d.gmom; m.gmom_stride = c->gmom_stride;
  m.df = (c->basis_prec == SFB_MIXED && c->opt_mom_df) ? 1 : 0;
  // Cf | Z | Wt | the double-float split of Cf (two float blocks of kTP x C)
  const size_t smd = sizeof(double) * ((size_t)kTP * maxC + (size_t)(m.rt + 1) * max_nx * kTP + kTP) +
                     2 * sizeof(float) * (size_t)kTP * maxC;
  CK(cudaFuncSetAttribute(darcy_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
  const int row_tiles = (max_ny + m.rt - 1) / m.rt;
  const int first = c->mom_shift_set ? 0 : 1;
  CK(cudaEventRecord(c->ev[3], st));
  if (c->last_dtn) {
    // Method S1: the Darcy entries of every point from one more subdomain
    // solve each (the recovery), point chunk by point chunk as rows of the
    // partial-sum buffer, then their shifted moments
    const int64_t rows = 2 * ((int64_t)c->mom_chunks + 1);
    for (int64_t p0 = 0; p0 < n_pts; p0 += rows) {
      const int64_t cnt = std::min(rows, n_pts - p0);
      CK(cudaMemsetAsync(d.mom_part, 0, sizeof(double) * cnt * m.len_d, st));
      CK(launch_dtn(c, d.lam, p0, cnt, 1, d.mom_part, st));
      CK(launch_s1_moments(c, d.mom_part, p0, cnt, first && p0 == 0 ? 1 : 0, st));
    }
  } else {
    if (first) {
      m.mode = 0;
      darcy_moments_kernel<<<dim3(row_tiles, ns, 1), kMomT, smd, st>>>(m);
      LAUNCHED("darcy_moments_kernel");
      CK(cudaGetLastError());
    }
    m.mode = 1;
    CK(cudaFuncSetAttribute(darcy_moments_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
    CK(cudaMemsetAsync(d.mom_part, 0, sizeof(double) * 2 * (size_t)m.n_chunks * m.len_d, st));
    moments_worklist_kernel<<<1, 256, 0, st>>>(m, d.mom_work, d.active + 3, c->mom_work_cap, d.active + 2);
    LAUNCHED("moments_worklist_kernel");
    darcy_moments_list_kernel<<<dim3(row_tiles, 1, m.n_chunks), kMomT, smd, st>>>(m, d.mom_work, d.active + 3,
                                                                                 d.active + 2);
    LAUNCHED("darcy_moments_list_kernel");
    CK(cudaGetLastError());
    int max_local = 1;
    for (int nl : c->n_local) max_local = std::max(max_local, nl);
    group_moments_kernel<<<dim3(max_local, ns, kGChunks), 256, 0, st>>>(m, d.gmom_part);
    LAUNCHED("group_moments_kernel");
    group_moments_reduce<<<dim3(max_local, ns), 256, 0, st>>>(m, d.gmom_part);
    LAUNCHED("group_moments_reduce");
    int big_t = kBigT;
    auto smb_of = [&](int t) { return sizeof(double) * ((size_t)maxC * maxC + 2 * (size_t)maxC + (size_t)maxC * t); };
    while (big_t > 32 && smb_of(big_t) > 227 * 1024) big_t >>= 1;
    const size_t smb = smb_of(big_t);
    CK(cudaFuncSetAttribute(bigroup_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
    int max_ent = 0;
    for (const HostSub& S : c->subs) max_ent = std::max(max_ent, S.ny * S.nx + S.ny * (S.nx + 1) + (S.ny + 1) * S.nx);
    bigroup_moments_kernel<<<dim3((max_ent + big_t * kBigE - 1) / (big_t * kBigE), ns), big_t, smb, st>>>(m, m.n_chunks);
    LAUNCHED("bigroup_moments_kernel");
    CK(cudaGetLastError());
    reduce_partials<<<256, 256, 0, st>>>(d.mom_part, m.n_chunks + 1, m.len_d, d.mom + m.len_d, d.mom + 2 * m.len_d);
    LAUNCHED("reduce_partials");
  }
  CK(cudaEventRecord(c->ev[4], st));
  const int Cs = (int)c->stokes.dofs.size() + 1;
  stokes_cov_kernel<<<kStokesChunks, 256, 0, st>>>(m.ia, d.w, first, d.st_c0, d.st_part);
  LAUNCHED("stokes_cov_kernel");
  stokes_cov_reduce<<<32, 256, 0, st>>>(d.st_part, Cs, d.st_m, d.st_M);
  LAUNCHED("stokes_cov_reduce");
  CK(cudaGetLastError());
  c->mom_shift_set = true;
  weight_sum<<<1, 256, 0, st>>>(d.w, n_pts, d.mom_w);
  LAUNCHED("weight_sum");
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->ev[5], st));
  return SFB_OK;
#undef LAUNCHED
#undef CK
}

sfb_status moments_finalize_device(sfb_ctx* c, int field, double* mean_d, double* var_d) {
  Dev& d = c->dev;
  const int64_t len_d = c->mom_len[0] + c->mom_len[1];
  if (field <= 1) {
    const int64_t off = field == 0 ? 0 : c->mom_len[0];
    finalize_darcy<<<256, 256, 0, c->stream>>>(d.mom, d.mom + len_d, d.mom + 2 * len_d, off, c->mom_len[field],
                                               d.mom_w, mean_d, var_d);
    ++c->launches;
  } else {
    const int Cs = (int)c->stokes.dofs.size() + 1;
    const double* U = field == 2 ? d.s_U : d.s_P;
    const int64_t n = c->mom_len[field];
    finalize_stokes<<<(int)((n * 32 + 255) / 256), 256, 0, c->stream>>>(U, n, Cs, d.st_c0, d.st_m, d.st_M,
                                                                          d.mom_w, mean_d, var_d);
    ++c->launches;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return SFB_ERR_CUDA; }
  return SFB_OK;
}

}  // namespace sfb
