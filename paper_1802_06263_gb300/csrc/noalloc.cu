// An entry point that builds one stochastic-basis item without allocating any
// device memory. Some hosts of this library cannot call cudaMalloc: an
// application that reserved all device memory for its own pool up front (so
// an extra allocation fails or fragments it), or a caller that must not
// allocate on its hot path (allocation can synchronise the device and take
// unbounded time). For them the working memory of this variant lives in a
// file-scope device array that the module carries; the caller passes only the
// input context and the output buffers.
//
// The array is kNoAllocBytes (8 MiB) and, once the module is loaded on a GPU,
// stays allocated there until the process exits. The module (and with it the
// array) is loaded on the device that is current when sfb_create runs, so a
// caller that reserves its own memory pool should create its contexts first.
// Every call shares the array and it keeps the previous call's contents, so
// the call clears the words that must start at zero itself. Calls that
// overlap on the GPU (other streams or host threads using the same device)
// race on the array; serialise them.
#include <string>

#include "sfb_ctx.h"

namespace sfb {

namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The host-side name of the array is not a device address: look the address up
// with the device current. It is looked up again on every call (cheap once the
// module is loaded), so a context torn down and created again on the device
// never leaves a stale address behind.
cudaError_t scratch_address(void** out) {
  *out = nullptr;
  return cudaGetSymbolAddress(out, g_noalloc_scratch);
}

}  // namespace

// Loads this file's module on the current device, which reserves the static
// array there, and checks that its address resolves. Called by sfb_create;
// on a machine without a usable device it does nothing (the entry point below
// then reports the CUDA error itself).
void noalloc_preload() {
  int dev = 0;
  void* p = nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess || scratch_address(&p) != cudaSuccess) cudaGetLastError();
}

}  // namespace sfb

using namespace sfb;

extern "C" sfb_status sfb_build_basis_item_noalloc(sfb_ctx* c, int32_t sub, int32_t k, int32_t prec,
                                                   double* phi_out, double* g_out, double* x_out) {
  if (!c) return SFB_ERR_ARG;
  if (!c->kl_done || !c->coll_done) {
    c->err = "sfb_kl_setup and sfb_collocation_setup must come first";
    return SFB_ERR_STATE;
  }
  if (sub < 0 || sub >= (int)c->subs.size() || k < 0 || k >= c->n_local[sub] || prec < 0 || prec > 2 ||
      !phi_out || !x_out) {
    c->err = "bad arguments to sfb_build_basis_item_noalloc";
    return SFB_ERR_ARG;
  }
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, x_out) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    c->err = "x_out must be device memory";
    return SFB_ERR_ARG;
  }
  const HostSub& H = c->subs[sub];
  const int nx = H.nx, ny = H.ny, nc = nx * ny, R = (int)H.dofs.size(), C = R + 1, nt = H.n_term;
  const int64_t np = (nx + kPanel - 1) / kPanel * kPanel, cp = (C + 3) & ~3;
  const size_t gsz = prec == SFB_FP64 ? sizeof(double) : sizeof(float);
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    c->err = std::string("no-alloc scratch: ") + cudaGetErrorString(e);
    return SFB_ERR_CUDA;
  }
  // layout of this item's tables and working arrays inside the static array
  Carver cv;
  cv.base = reinterpret_cast<char*>(base);
  int64_t nproj = 0;
  for (int q = 0; q < 4; ++q) nproj += (int64_t)H.proj[q].size();
  SubDev* d_sub = cv.take<SubDev>(1);
  double* d_proj = cv.take<double>(nproj);
  int* d_info = cv.take<int>(3 * R);
  double* d_kl = cv.take<double>((size_t)nt * (1 + nx + ny));
  double* d_yloc = cv.take<double>((size_t)c->n_local[sub] * nt);
  int* d_item = cv.take<int>(2);
  ItemOff* d_off = cv.take<ItemOff>(1);
  double* d_T = cv.take<double>((size_t)ny * (nx + 1) + (size_t)(ny + 1) * nx);
  double* d_D = cv.take<double>(nc);
  char* d_S = cv.take<char>((size_t)nc * gsz);
  char* d_DL = cv.take<char>((size_t)nc * gsz);
  char* d_G = cv.take<char>((size_t)ny * np * np * gsz);
  char* d_Z = cv.take<char>((size_t)ny * np * cp * gsz);
  double* d_phi = cv.take<double>((size_t)R * R + R);
  int* d_status = cv.take<int>(2);
  double* d_diag = cv.take<double>(3);
  long long* d_cyc = cv.take<long long>(kCycSlots);
  if (cv.used > kNoAllocBytes) {
    c->err = "item needs " + std::to_string(cv.used) + " bytes of scratch; the no-alloc entry point has " +
             std::to_string(kNoAllocBytes);
    return SFB_ERR_UNSUPPORTED;
  }
  // host images of the tables
  SubDev S;
  S.nx = nx; S.ny = ny; S.R = R; S.n_term = nt; S.n_local = c->n_local[sub];
  S.x0 = H.x0; S.y0 = H.y0; S.hx = H.hx; S.hy = H.hy; S.nu = c->prob.nu_d; S.source = H.source;
  S.mean_y = H.mean_y;
  std::vector<double> proj;
  for (int q = 0; q < 4; ++q) {
    S.side_type[q] = H.side_type[q];
    S.side_val[q] = H.side_val[q];
    S.proj_off[q] = (int64_t)proj.size();
    proj.insert(proj.end(), H.proj[q].begin(), H.proj[q].end());
  }
  S.dofinfo_off = 0; S.kl_off = 0; S.yloc_off = 0; S.gdof_off = 0;
  S.item0 = -(int64_t)k;  // the single item then has storage index 0
  std::vector<double> kl(H.slam.begin(), H.slam.end());
  kl.insert(kl.end(), H.fx.begin(), H.fx.end());
  kl.insert(kl.end(), H.fy.begin(), H.fy.end());
  const int item[2] = {0, k};  // item_sub[0] = 0 (the one SubDev), item_k[0] = k
  ItemOff off;
  off.x = 0; off.t = 0; off.g = 0; off.z = 0; off.phi = 0; off.diag = 0; off.sc = 0;
  cudaStream_t st = c->stream;
#define NA_CK(x)                                                              \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      c->err = std::string("no-alloc basis item: ") + cudaGetErrorString(e_); \
      return SFB_ERR_CUDA;                                                    \
    }                                                                         \
  } while (0)
  NA_CK(cudaMemcpyAsync(d_sub, &S, sizeof(S), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_proj, proj.data(), sizeof(double) * proj.size(), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_info, H.dofinfo.data(), sizeof(int) * H.dofinfo.size(), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_kl, kl.data(), sizeof(double) * kl.size(), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_yloc, c->loc_y[sub].data(), sizeof(double) * c->loc_y[sub].size(),
                        cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_item, item, sizeof(item), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_off, &off, sizeof(off), cudaMemcpyHostToDevice, st));
  // the words the kernels accumulate into start at zero on every call
  NA_CK(cudaMemsetAsync(d_status, 0, sizeof(int) * 2, st));
  NA_CK(cudaMemsetAsync(d_diag, 0, sizeof(double) * 3, st));
  BasisArgs a;
  a.subs = d_sub; a.proj = d_proj; a.dofinfo = d_info; a.kl = d_kl; a.yloc = d_yloc;
  a.item_sub = d_item; a.item_k = d_item + 1; a.off = d_off; a.n_items = 1;
  a.X = x_out; a.T = d_T; a.G = d_G; a.Z = d_Z; a.S = d_S; a.DL = d_DL; a.phi = d_phi; a.phi32 = nullptr; a.D = d_D;
  a.status = d_status; a.resid = d_diag; a.corr1 = d_diag + 1; a.errest = d_diag + 2; a.nref = d_status + 1;
  a.cycles = d_cyc;
  a.max_refine = c->opt_refine_max;
  a.refine_tol = c->opt_refine_tol;
  if (prec == SFB_FP64) NA_CK(launch_basis_fp64(a, nx, C, st));
  else NA_CK(launch_basis_mixed(a, nx, C, prec == SFB_MIXED ? a.max_refine : 0, st));
  NA_CK(launch_flux_epilogue(a, R, st));
  c->launches += 2;
  NA_CK(cudaMemcpyAsync(phi_out, d_phi, sizeof(double) * R * R, cudaMemcpyDefault, st));
  if (g_out) NA_CK(cudaMemcpyAsync(g_out, d_phi + (size_t)R * R, sizeof(double) * R, cudaMemcpyDefault, st));
  int status = 0;
  NA_CK(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  if (status & ST_NONFINITE) { c->err = "non-finite permeability or solution"; return SFB_ERR_NONFINITE; }
  if (status & ST_NOT_SPD) { c->err = "non-positive pivot"; return SFB_ERR_NOT_SPD; }
  if (status & ST_TIMEOUT) { c->err = "a bulk copy did not complete"; return SFB_ERR_TIMEOUT; }
  if (status & ST_NOT_CONVERGED) { c->err = "refinement stopped above tolerance"; return SFB_ERR_NOT_CONVERGED; }
  return SFB_OK;
}
