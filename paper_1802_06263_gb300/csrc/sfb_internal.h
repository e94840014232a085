// Internal data layout shared by the host orchestration (sfb_host.cpp) and
// the CUDA kernels. Everything here is plain data: device arrays are carved
// out of the caller's workspace and addressed by 64-bit element offsets.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfb {

constexpr int kMaxNx = 128;      // cells per block row of a Darcy subdomain
constexpr int kMaxCols = 129;    // mortar DOFs per subdomain + 1 particular column
constexpr int kSides = 4;        // bottom, right, top, left
enum SideType { SIDE_NOFLOW = 0, SIDE_IFACE = 1, SIDE_DIRICHLET = 2 };

// Error bits written by kernels into a per-item / per-point status word.
enum : int {
  ST_NONFINITE = 1,
  ST_NOT_SPD = 2,
  ST_NOT_CONVERGED = 4,
  ST_BAD_INDEX = 8,
  ST_TIMEOUT = 16,
};

// One Darcy subdomain. Side order: 0 bottom, 1 right, 2 top, 3 left; the
// faces of a side are ordered by increasing coordinate.
struct SubDev {
  int nx, ny, R, n_term, n_local;
  double x0, y0, hx, hy, nu, source, mean_y;
  int side_type[kSides];
  double side_val[kSides];
  int64_t proj_off[kSides];  // into proj: dense [faces][R] face averages of the mortar basis
  int64_t dofinfo_off;       // into dofinfo: per local DOF (side, first face, end face)
  int64_t kl_off;            // into kl: sqrt(lambda)[nt] | fx[nt][nx] | fy[nt][ny]
  int64_t yloc_off;          // into yloc: local realizations [n_local][nt]
  int64_t gdof_off;          // into gdof: local -> global mortar DOF
  int64_t item0;             // first basis item of this subdomain (items k = 0..n_local-1)
};

#ifdef __CUDACC__
// Conversions between binary64 and binary32 on the integer pipe, from the
// IEEE 754 formats (exponent biases 1023 and 127, 52 and 23 fraction bits).
// The conversion instructions issue on the FP64 pipe, which on this part runs
// at 1/64 of the FP32 rate, and the mixed form converts every residual entry
// and every correction once per refinement pass.
// binary64 -> binary32: fraction truncated (round toward zero, relative error
// below 2^-23), magnitudes below the binary32 normal range give zero, above it
// (and non-finite values) NaN.
__device__ __forceinline__ float f64_to_f32_bits(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const unsigned e = (hi >> 20) & 0x7ffu;
  unsigned bits = hi & 0x80000000u;
  if (e > 1150u) bits = 0x7fc00000u;
  else if (e >= 897u) bits |= ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(bits);
}
// binary32 -> binary64, exact for normal values; subnormals give zero,
// non-finite values NaN.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  unsigned hi = b & 0x80000000u, lo = 0u;
  if (e == 255u) hi = 0x7ff80000u;
  else if (e != 0u) { hi |= ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3); lo = b << 29; }
  return __hiloint2double((int)hi, (int)lo);
}
template <typename T>
__device__ __forceinline__ T from_f64(double v);
template <>
__device__ __forceinline__ float from_f64<float>(double v) { return f64_to_f32_bits(v); }
template <>
__device__ __forceinline__ double from_f64<double>(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f32_to_f64_bits(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return f64_to_f32_bits(v); }

#endif  // __CUDACC__

// SM-cycle record per basis item: setup, factor, forward sweeps, backward
// sweeps, then 12 sub-phases of the row steps (see sfb_basis_stats).
constexpr int kCycSlots = 16;

// Pivots per panel of the blocked block inversion; the diagonal blocks are
// identity-padded to a multiple of it.
constexpr int kPanel = 16;

// Largest grid of the persistent interface CG with resident tiles (the
// per-CTA tile ranges live in the workspace).
constexpr int kPcgMaxGrid = 2048;

// Point chunks of the Stokes coefficient moments (partials summed in order).
constexpr int kStokesChunks = 32;

// Restarted GMRES of the interface problem: the largest restart length, and
// the per-point state (Hessenberg columns, Givens rotations, rotated
// right-hand side) in doubles.
constexpr int kGmresMax = 30;
constexpr int kGmresState = 1024;

// Per-item storage offsets (elements) into the basis store arrays.
struct ItemOff {
  int64_t x;    // X: [R+1][n_cells] FP64 pressure responses (column-major)
  int64_t t;    // T: x-faces [ny][nx+1] then y-faces [ny+1][nx] FP64 transmissibilities
  int64_t g;    // G: [ny][nx][nx] inverse Schur blocks (FP64 or FP32)
  int64_t z;    // Z: [R+1][n_cells] solve scratch (factor precision)
  int64_t phi;  // Phi: [R][R] then g: [R], padded to a multiple of 4 elements
  int64_t diag; // D: [n_cells] FP64 diagonal of A
  int64_t sc;   // S: [n_cells] diag(A)^{-1/2} in the factor precision
};

struct BasisArgs {
  const SubDev* subs;
  const double* proj;
  const int* dofinfo;
  const double* kl;
  const double* yloc;
  const int* item_sub;     // item -> subdomain (items sorted by decreasing cost)
  const int* item_k;       // item -> local realization
  const ItemOff* off;      // indexed by item id = subs[s].item0 + k
  int n_items;
  double* X;
  double* T;
  void* G;
  void* Z;                 // [R+1][n_cells] solve scratch in the factor precision
  void* S;                 // [n_cells] diagonal scaling in the factor precision
  void* DL;                // [n_cells] scaled row couplings s_{b-1,i} Ty[b][i] s_{b,i} (row 0: 0), same offsets as S
  double* phi;
  float* phi32;            // Phi and g rounded to FP32 (same offsets)
  double* D;
  int* status;             // per item
  double* resid;           // per item: last relative residual ||B - A X|| / ||B||
  double* corr1;           // per item: relative size of the first correction
  double* errest;          // per item: estimated relative error of the final X
  int* nref;               // per item: refinement steps taken
  long long* cycles;       // per item: SM cycles in [setup, factor, forward, backward]
  int max_refine;
  double refine_tol;
  const void* gmaps = nullptr;  // per item id: CUtensorMap of its block inverses (tensor-core form)
  int particular_only = 0;      // Method S1's set-up: factor and particular solution only (FP64 kernel)
  // split launch shapes: the solve kernel's work units, column chunks of the
  // class's items (class-local item index, first column, column count); their
  // refinement statistics go to slots n_items_all + chunk of the per-item arrays
  const int* chunk_item = nullptr;
  const int* chunk_c0 = nullptr;
  const int* chunk_cnt = nullptr;
  int n_chunks = 0;
  int chunk_slot0 = 0;          // the class's first chunk among all chunks
  int n_items_all = 0;
};

// Launchers (basis.cu).
cudaError_t launch_basis_fp64(const BasisArgs& a, int max_nx, int max_cols, cudaStream_t st);
// loads the allocation-free entry point's module (and its static array) on the current device
void noalloc_preload();
cudaError_t launch_basis_mixed(const BasisArgs& a, int max_nx, int max_cols, int refine,
                               cudaStream_t st);
cudaError_t launch_flux_epilogue(const BasisArgs& a, int max_R, cudaStream_t st);

// Launch shapes of the basis kernel per precision (fp64 0/1) and size class
// (wide: grids more than 64 cells wide); the autotuner's candidates.
struct BasisShape {
  int threads;    // threads per CTA
  int min_ctas;   // CTAs per SM the register budget is compiled for
  int g_buffers;  // shared-memory buffers of G_b (2: the next block row is prefetched)
  int tcgen05;    // 1: block-row products on the tensor cores (basis_tc.cu)
  int split = 0;  // 1: a factor launch per item, then a solve launch per chunk of kChunkCols columns
};
// Columns of a split shape's solve work unit (at most; chunks are multiples of 4 but the last)
constexpr int kChunkCols = 24;
// The chunks of an item with C right-hand sides: n = ceil(C / kChunkCols) of
// base = round4(ceil(C / n)) columns each but the last (C - base (n - 1)).
inline int chunk_count(int C) { return (C + kChunkCols - 1) / kChunkCols; }
inline int chunk_base(int C) {
  const int n = chunk_count(C);
  return (((C + n - 1) / n) + 3) & ~3;
}
int basis_shape_count(int fp64);
bool basis_shape_desc(int fp64, int wide, int shape, BasisShape* out);
bool basis_shape_split(int fp64, int wide, int shape);
// The persistent FP32 launch over every item of both size classes (a: all
// items in build order, all chunks; counter and flags: workspace words it
// clears first). ctas: when non-null, only reports the resident CTAs per SM.
cudaError_t launch_basis_persistent(const BasisArgs& a, int* counter, int* flags, int n_wide, int chunk_n0,
                                    int max_nx, int max_cols, int refine, cudaStream_t st, int* ctas);
// One part of a split FP32 shape: 1 the factor launch (a.n_items items), 2
// the solve launch (a.n_chunks chunks).
cudaError_t launch_basis_part(const BasisArgs& a, int wide, int shape, int part, int max_nx, int max_cols, int refine,
                              cudaStream_t st);
// Resident CTAs per SM of a shape at the class's largest grid and column count.
cudaError_t basis_shape_ctas(int fp64, int wide, int shape, int max_nx, int max_cols, int* ctas);
cudaError_t launch_basis_shape(const BasisArgs& a, int fp64, int wide, int shape, int max_nx, int max_cols,
                               int refine, cudaStream_t st);
// Tensor-core form of the mixed basis kernel (basis_tc.cu): grids up to 64
// cells wide, up to 128 right-hand sides; needs BasisArgs::gmaps.
bool basis_tc_supported(int max_nx, int max_cols);
cudaError_t basis_tc_ctas(int max_nx, int max_cols, int* ctas);
cudaError_t launch_basis_tc(const BasisArgs& a, int max_nx, int max_cols, int refine, cudaStream_t st);

}  // namespace sfb
