// C ABI of the library (include/sfb.h): context, set-up, workspace carving
// and the orchestration of the CUDA kernels on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "sfb_ctx.h"

namespace sfb {
void stokes_assemble_host(sfb_ctx* c);
size_t basis_smem_bytes(int prec_fp64, int max_nx, int max_cols);
cudaError_t stokes_solve_device(sfb_ctx* c);
sfb_status iface_solve_device(sfb_ctx* c, int64_t n_pts, double rtol, int max_it, int krylov, int* n_failed);
sfb_status moments_finalize_device(sfb_ctx* c, int field, double* mean_d, double* var_d);
void build_hash_tables(sfb_ctx* c, std::vector<int>& table, std::vector<int64_t>& off, std::vector<int>& cap);
sfb_status moments_accumulate_device(sfb_ctx* c, int64_t n_pts);
}  // namespace sfb

using namespace sfb;

namespace {

sfb_status fail(sfb_ctx* c, sfb_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

sfb_status cuda_fail(sfb_ctx* c, cudaError_t e, const char* where) {
  return fail(c, SFB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SFB_CUDA(call, where)                     \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int n_units(const sfb_ctx* c) { return (int)c->subs.size() + 1; }

// Geometry: interfaces, mortar DOF numbering, face projections (Section 3.1,
// 3.3; the subdomain-side L2 projections of Section 5.2 step 1).
sfb_status build_geometry(sfb_ctx* c) {
  const sfb_problem& P = c->prob;
  const int px = P.px, py = P.py;
  const double x0 = P.darcy_box[0], x1 = P.darcy_box[1], y0 = P.darcy_box[2], y1 = P.darcy_box[3];
  const double W = (x1 - x0) / px, H = (y1 - y0) / py;
  const int deg = P.mortar_degree;
  c->subs.assign(px * py, HostSub());
  for (int iy = 0; iy < py; ++iy)
    for (int ix = 0; ix < px; ++ix) {
      const int s = iy * px + ix;
      HostSub& S = c->subs[s];
      S.nx = c->nx[s]; S.ny = c->ny[s];
      S.x0 = x0 + ix * W; S.x1 = S.x0 + W; S.y0 = y0 + iy * H; S.y1 = S.y0 + H;
      S.hx = W / S.nx; S.hy = H / S.ny;
      for (int q = 0; q < 4; ++q) { S.side_type[q] = SIDE_NOFLOW; S.side_val[q] = 0.0; S.side_iface[q] = -1; }
      S.source = c->source.empty() ? 0.0 : c->source[s];
    }
  c->ifaces.clear();
  int64_t off = 0;
  auto add_iface = [&](int kind, double s0, double s1, int n_el, int sa, int qa, int sb, int qb) {
    HostIface f;
    f.kind = kind; f.s0 = s0; f.s1 = s1; f.n_el = n_el; f.deg = deg;
    f.sub_a = sa; f.side_a = qa; f.sub_b = sb; f.side_b = qb;
    f.off = off; f.n_dof = n_el * (deg + 1);
    off += f.n_dof;
    const int id = (int)c->ifaces.size();
    c->ifaces.push_back(f);
    if (sa >= 0) { c->subs[sa].side_type[qa] = SIDE_IFACE; c->subs[sa].side_iface[qa] = id; }
    if (sb >= 0) { c->subs[sb].side_type[qb] = SIDE_IFACE; c->subs[sb].side_iface[qb] = id; }
  };
  for (int ix = 0; ix < px; ++ix)
    add_iface(0, x0 + ix * W, x0 + (ix + 1) * W, c->msd[ix], (py - 1) * px + ix, 2, -1, 0);
  for (int iy = 0; iy < py; ++iy)
    for (int ix = 0; ix + 1 < px; ++ix)
      add_iface(1, y0 + iy * H, y0 + (iy + 1) * H, c->mdv[iy * (px - 1) + ix], iy * px + ix, 1,
                iy * px + ix + 1, 3);
  for (int iy = 0; iy + 1 < py; ++iy)
    for (int ix = 0; ix < px; ++ix)
      add_iface(2, x0 + ix * W, x0 + (ix + 1) * W, c->mdh[iy * px + ix], iy * px + ix, 2,
                (iy + 1) * px + ix, 0);
  for (int ix = 0; ix < px; ++ix) {
    c->subs[ix].side_type[0] = SIDE_DIRICHLET;
    c->subs[ix].side_val[0] = P.bottom_pressure;
  }
  c->n_lambda = off;
  // local DOFs, projections, per-DOF face ranges
  for (HostSub& S : c->subs) {
    std::vector<int> its;
    for (int q = 0; q < 4; ++q) if (S.side_iface[q] >= 0) its.push_back(S.side_iface[q]);
    std::sort(its.begin(), its.end());
    S.dofs.clear();
    for (int id : its)
      for (int a = 0; a < c->ifaces[id].n_dof; ++a) S.dofs.push_back(c->ifaces[id].off + a);
    const int R = (int)S.dofs.size();
    if (R + 1 > kMaxCols) return fail(c, SFB_ERR_UNSUPPORTED, "too many mortar DOFs on a subdomain");
    S.dofinfo.assign(3 * R, 0);
    for (int q = 0; q < 4; ++q) {
      const int nf = (q == 0 || q == 2) ? S.nx : S.ny;
      S.proj[q].assign((size_t)nf * R, 0.0);
      if (S.side_iface[q] < 0) continue;
      const HostIface& itf = c->ifaces[S.side_iface[q]];
      const double start = (q == 0 || q == 2) ? S.x0 : S.y0;
      const double h = (q == 0 || q == 2) ? S.hx : S.hy;
      std::vector<int> cols(itf.n_dof);
      for (int a = 0; a < itf.n_dof; ++a)
        cols[a] = (int)(std::lower_bound(S.dofs.begin(), S.dofs.end(), itf.off + a) - S.dofs.begin());
      face_projection(itf, start, h, nf, cols, R, S.proj[q].data());
      const double He = (itf.s1 - itf.s0) / itf.n_el;
      for (int a = 0; a < itf.n_dof; ++a) {
        const int e = a / (itf.deg + 1);
        const double e0 = itf.s0 + e * He, e1 = e0 + He;
        int fb = (int)std::floor((e0 - start) / h - 1e-9);
        int fe = (int)std::ceil((e1 - start) / h + 1e-9);
        fb = std::max(0, fb); fe = std::min(nf, fe);
        S.dofinfo[3 * cols[a]] = q; S.dofinfo[3 * cols[a] + 1] = fb; S.dofinfo[3 * cols[a] + 2] = fe;
      }
    }
    if (S.nx > kMaxNx || S.nx < 2 || S.ny < 2)
      return fail(c, SFB_ERR_UNSUPPORTED, "Darcy grid sizes must satisfy 2 <= nx <= 128, ny >= 2");
  }
  c->stokes.dofs.clear();
  for (const HostIface& f : c->ifaces)
    if (f.kind == 0)
      for (int a = 0; a < f.n_dof; ++a) c->stokes.dofs.push_back(f.off + a);
  return SFB_OK;
}

// Workspace layout; `c->dev` gets the slices when carver.base is set.
size_t layout(sfb_ctx* c, Carver& cv, int prec, int64_t max_pts) {
  Dev& d = c->dev;
  const int ns = (int)c->subs.size();
  const size_t gsz = prec == SFB_FP64 ? sizeof(double) : sizeof(float);
  int64_t n_items = 0, nX = 0, nZ = 0, nT = 0, nG = 0, nPhi = 0, nD = 0, nproj = 0, ninfo = 0, nkl = 0, nyl = 0,
          ngd = 0;
  int64_t n_loc_tot = 0, n_chunks = 0;
  c->offs.clear();
  for (int s = 0; s < ns; ++s) {
    const HostSub& S = c->subs[s];
    const int R = (int)S.dofs.size(), C = R + 1, nc = S.nx * S.ny;
    const int nl = c->n_local.empty() ? 0 : c->n_local[s];
    for (int k = 0; k < nl; ++k) {
      ItemOff o;
      // row blocks of Z: [ny][npad][C rounded up to 8] (the tensor-core form's
      // accumulator columns; the CUDA-core form uses C rounded up to 4)
      const int64_t npad_ = (S.nx + kPanel - 1) / kPanel * kPanel, cpad_ = (C + 7) & ~7;
      o.x = nX; nX += (int64_t)nc * C;
      o.z = nZ; nZ += (int64_t)S.ny * npad_ * cpad_;   // row blocks in the shared-memory layout
      o.t = nT; nT += (int64_t)S.ny * (S.nx + 1) + (int64_t)(S.ny + 1) * S.nx;
      const int64_t npad = (S.nx + kPanel - 1) / kPanel * kPanel;  // identity-padded block size of the factor
      // G: [ny][npad][npad]; twice that, for the tensor-core form's TF32 hi and lo parts
      o.g = nG; nG += 2 * (int64_t)S.ny * npad * npad;
      o.phi = nPhi; nPhi += ((int64_t)R * R + R + 3) & ~int64_t(3);   // 16-byte aligned in FP32 and FP64
      o.diag = nD; o.sc = nD; nD += nc;
      c->offs.push_back(o);
    }
    n_items += nl;
    n_loc_tot += nl;
    n_chunks += (int64_t)nl * chunk_count(C);
    for (int q = 0; q < 4; ++q) nproj += (int64_t)S.proj[q].size();
    ninfo += 3 * R;
    nkl += S.n_term * (1 + S.nx + S.ny);
    nyl += (int64_t)nl * S.n_term;
    ngd += R;
  }
  c->n_items = n_items;
  c->n_chunks = n_chunks;
  d.subs = cv.take<SubDev>(ns);
  d.proj = cv.take<double>(nproj);
  d.dofinfo = cv.take<int>(ninfo);
  d.kl = cv.take<double>(nkl);
  d.yloc = cv.take<double>(nyl);
  d.gdof = cv.take<int64_t>(ngd);
  d.item_sub = cv.take<int>(n_items);
  d.item_k = cv.take<int>(n_items);
  d.off = cv.take<ItemOff>(n_items);
  d.X = cv.take<double>(nX);
  d.T = cv.take<double>(nT);
  d.G = cv.take<char>(nG * gsz);
  d.Z = cv.take<char>(nZ * gsz);
  d.gmaps = cv.take<char>((size_t)n_items * 128);
  d.phi = cv.take<double>(nPhi);
  d.phi32 = cv.take<float>(nPhi);
  d.D = cv.take<double>(nD);
  d.S = cv.take<char>(nD * gsz);
  d.DL = cv.take<char>(nD * gsz);
  // per item, then per column chunk of a split launch shape
  d.status = cv.take<int>(n_items);
  d.resid = cv.take<double>(n_items + n_chunks);
  d.corr1 = cv.take<double>(n_items + n_chunks);
  d.errest = cv.take<double>(n_items + n_chunks);
  d.cycles = cv.take<long long>(kCycSlots * (n_items + n_chunks));
  d.nref = cv.take<int>(n_items + n_chunks);
  d.chunk_item = cv.take<int>(std::max<int64_t>(n_chunks, 1));
  d.chunk_c0 = cv.take<int>(std::max<int64_t>(n_chunks, 1));
  d.chunk_cnt = cv.take<int>(std::max<int64_t>(n_chunks, 1));
  d.persist_counter = cv.take<int>(4);
  d.persist_flags = cv.take<int>(std::max<int64_t>(n_items, 1));
  // Stokes
  const StokesHost& St = c->stokes;
  const int Rs = (int)St.dofs.size(), Cs = Rs + 1;
  // the band of the Stokes system's LU factors: row i holds columns
  // i - kl .. i + kl + ku (partial pivoting widens U to kl + ku)
  d.s_mat = cv.take<double>((size_t)St.n_free * (2 * St.kl + St.ku + 1) + 8);
  d.s_pl = cv.take<double>((size_t)(32 + St.kl) * 32);
  d.s_piv = cv.take<int>(St.n_free);
  d.s_rhs = cv.take<double>((size_t)St.n_free * Cs);
  d.s_b = cv.take<double>((size_t)St.n_free * Cs);
  d.s_res = cv.take<double>((size_t)St.n_free * Cs);
  d.s_row_ptr = cv.take<int>((size_t)St.n_free + 1);
  d.s_U = cv.take<double>((size_t)St.n_u * Cs);
  d.s_P = cv.take<double>((size_t)St.n_p * Cs);
  d.s_phi = cv.take<double>((size_t)Rs * Rs + Rs);
  d.s_phi32 = cv.take<float>(((size_t)Rs * Rs + Rs + 3) & ~size_t(3));
  d.s_dir = cv.take<double>(St.n_u);
  d.s_nb = cv.take<double>(St.nb.size());
  d.s_nb_node = cv.take<int>(St.nb_node.size());
  d.s_free_to_full = cv.take<int>(St.n_free);
  d.s_tr_row = cv.take<int>(St.tr_row.size());
  d.s_tr_col = cv.take<int>(St.tr_col.size());
  d.s_tr_val = cv.take<double>(St.tr_val.size());
  d.s_status = cv.take<int>(4);
  // interface solve
  const int nu = n_units(c);
  c->ybase.assign(nu + 1, 0);
  for (int s = 0; s < ns; ++s) c->ybase[s + 1] = c->ybase[s] + (int64_t)c->subs[s].dofs.size();
  c->ybase[nu] = c->ybase[ns] + Rs;
  c->NY = c->ybase[nu];
  int max_local = 1;
  for (int nl : c->n_local) max_local = std::max(max_local, nl);
  c->max_tiles = (int)std::min<int64_t>(max_pts, (int64_t)max_local + (max_pts + 31) / 32);
  c->max_tiles = std::max(c->max_tiles, 1);
  const int ndim = c->grid.n_dim;
  int64_t hash_tot = 0;
  for (int s = 0; s < ns; ++s) {
    int cap = 1;
    const int nl = c->n_local.empty() ? 1 : c->n_local[s];
    while (cap < 2 * nl + 1) cap <<= 1;
    hash_tot += cap;
  }
  const int64_t P = std::max<int64_t>(max_pts, 1);
  d.y = cv.take<double>((size_t)P * std::max(ndim, 1));
  d.w = cv.take<double>(P);
  d.kmap = cv.take<int>((size_t)P * ns);
  d.hash = cv.take<int>(hash_tot);
  d.hash_off = cv.take<int64_t>(ns);
  d.hash_cap = cv.take<int>(ns);
  d.grp_count = cv.take<int>(std::max<int64_t>(n_loc_tot, 1));
  d.grp_start = cv.take<int>(std::max<int64_t>(n_loc_tot, 1));
  d.grp_pts = cv.take<int>((size_t)P * nu);
  d.tiles = cv.take<int>((size_t)nu * c->max_tiles * 3);
  d.n_tiles = cv.take<int>(nu);
  d.ldof = cv.take<int>((size_t)c->n_lambda * 4);
  d.yoff = cv.take<int>((size_t)c->n_lambda * 2);
  d.lam = cv.take<double>((size_t)P * c->n_lambda);
  d.r = cv.take<double>((size_t)P * c->n_lambda);
  d.p = cv.take<double>((size_t)P * c->n_lambda);
  d.Y = cv.take<double>((size_t)P * c->NY);
  d.rr = cv.take<double>(P);
  d.gn = cv.take<double>(P);
  d.rlast = cv.take<double>(P);
  d.dinv = cv.take<double>((size_t)P * c->n_lambda);
  d.gmV = cv.take<double>((size_t)(kGmresMax + 1) * P * c->n_lambda);
  d.gmS = cv.take<double>((size_t)P * kGmresState);
  d.gmJ = cv.take<int>(P);
  // balancing preconditioner: pseudo-inverses of the bases (the basis store's
  // offsets), per-point weights, S Z and the coarse Cholesky factors
  c->bdd_nc = 0;
  {
    std::vector<int> cidx(nu, -1);
    for (int s = 0; s < ns; ++s) {
      bool floating = true;
      for (int q = 0; q < 4; ++q) floating = floating && c->subs[s].side_type[q] != SIDE_DIRICHLET;
      if (floating) cidx[s] = c->bdd_nc++;
    }
    c->bdd_cidx = cidx;
  }
  d.bdd_pinv = cv.take<double>(nPhi);
  d.bdd_spinv = cv.take<double>((size_t)Rs * Rs + 2);
  d.bdd_wy = cv.take<double>((size_t)P * c->NY);
  d.bdd_sz = cv.take<double>((size_t)P * std::max(c->bdd_nc, 1) * c->n_lambda);
  d.bdd_L = cv.take<double>((size_t)P * std::max(c->bdd_nc * c->bdd_nc, 1));
  d.bdd_cidx = cv.take<int>(nu);
  c->minv_ld = 0; c->max_if_dof = 0;
  for (const HostIface& f : c->ifaces) { c->minv_ld += (int64_t)f.n_dof * f.n_dof; c->max_if_dof = std::max(c->max_if_dof, f.n_dof); }
  d.minv = cv.take<float>((size_t)P * std::max<int64_t>(c->minv_ld, 1));
  d.if_off = cv.take<int>(std::max<size_t>(c->ifaces.size(), 1));
  d.if_n = cv.take<int>(std::max<size_t>(c->ifaces.size(), 1));
  d.if_moff = cv.take<int>(std::max<size_t>(c->ifaces.size(), 1));
  d.dof_if = cv.take<int>((size_t)std::max<int64_t>(c->n_lambda, 1));
  d.rflag = cv.take<int>(P);
  d.pstat = cv.take<int>(P);
  d.active = cv.take<int>(32);   // flags and counts; [4, 32) the persistent CG's barrier, counters, clocks
  d.pcg_part = cv.take<int>(kPcgMaxGrid + 1);
  d.s_gdof = cv.take<int64_t>(std::max(Rs, 1));
  d.ybase = cv.take<int64_t>(nu + 1);
  d.dim_off = cv.take<int>(ns);
  d.loc_off = cv.take<int64_t>(ns);
  d.cell_off = cv.take<int64_t>(ns);
  d.face_off = cv.take<int64_t>(ns);
  // moments: Darcy p, Darcy flux, Stokes u, Stokes p
  int64_t np_ = 0, nf_ = 0;
  for (const HostSub& S : c->subs) {
    np_ += (int64_t)S.nx * S.ny;
    nf_ += (int64_t)S.ny * (S.nx + 1) + (int64_t)(S.ny + 1) * S.nx;
  }
  c->mom_len[0] = np_; c->mom_len[1] = nf_; c->mom_len[2] = St.n_u; c->mom_len[3] = St.n_p;
  int64_t mo = 0;
  for (int f = 0; f < 4; ++f) { c->mom_off[f] = mo; mo += c->mom_len[f]; }
  // Darcy accumulators and per-chunk partials; Stokes coefficient moments
  const int64_t len_d = np_ + nf_;
  int row_tiles = 0;
  {
    int max_ny = 1, max_nx = 1;
    for (const HostSub& S : c->subs) { max_ny = std::max(max_ny, S.ny); max_nx = std::max(max_nx, S.nx); }
    const int rt = std::max(1, std::min(max_ny, 512 / max_nx));
    row_tiles = ns * ((max_ny + rt - 1) / rt);
  }
  // point chunks of the per-point Darcy moments: about 4 CTAs per SM over the
  // row tiles of one subdomain (every CTA walks all subdomains)
  c->mom_chunks = std::max(1, std::min(64, (4 * 152 * ns + row_tiles - 1) / std::max(row_tiles, 1)));
  d.mom = cv.take<double>((size_t)3 * len_d);
  d.mom_w = cv.take<double>(2);
  d.mom_part = cv.take<double>((size_t)2 * (c->mom_chunks + 1) * len_d);   // + the large-group slot
  c->mom_work_cap = (int)((int64_t)ns * ((std::max<int64_t>(max_pts, 1) + 7) / 8 + c->max_tiles + 1));
  d.mom_work = cv.take<int4>((size_t)c->mom_work_cap);
  {
    int maxC = 1;
    for (const HostSub& S : c->subs) maxC = std::max(maxC, (int)S.dofs.size() + 1);
    c->gmom_stride = 1 + 2 * (int64_t)maxC + (int64_t)maxC * maxC;
  }
  d.gmom = cv.take<double>((size_t)std::max<int64_t>(n_loc_tot, 1) * c->gmom_stride);
  d.gmom_part = cv.take<double>((size_t)std::max<int64_t>(n_loc_tot, 1) * 16 * c->gmom_stride);
  d.st_c0 = cv.take<double>(Rs + 1);
  d.st_m = cv.take<double>(Rs + 1);
  d.st_M = cv.take<double>((size_t)(Rs + 1) * (Rs + 1));
  d.st_part = cv.take<double>((size_t)kStokesChunks * ((Rs + 1) + (size_t)(Rs + 1) * (Rs + 1)));
  d.fin = cv.take<double>((size_t)2 * std::max(std::max(np_, nf_), (int64_t)std::max(St.n_u, St.n_p)));
  return cv.used + 256;
}

}  // namespace

// ============================================================================
extern "C" {

sfb_status sfb_create(const sfb_problem* prob, void* stream, sfb_ctx** out) {
  if (!prob || !out) return SFB_ERR_ARG;
  *out = nullptr;
  sfb_ctx* c = new (std::nothrow) sfb_ctx();
  if (!c) return SFB_ERR_ARG;
  const int px = prob->px, py = prob->py;
  if (px < 1 || py < 1 || !prob->darcy_nx || !prob->darcy_ny || !prob->mortar_sd ||
      (px > 1 && !prob->mortar_dd_v) || (py > 1 && !prob->mortar_dd_h) ||
      (prob->mortar_degree != 1 && prob->mortar_degree != 2) || prob->stokes_sx < 1 ||
      prob->stokes_sy < 1 || !(prob->nu_s > 0) || !(prob->nu_d > 0)) {
    delete c;
    return SFB_ERR_ARG;
  }
  c->prob = *prob;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->nx.assign(prob->darcy_nx, prob->darcy_nx + px * py);
  c->ny.assign(prob->darcy_ny, prob->darcy_ny + px * py);
  c->msd.assign(prob->mortar_sd, prob->mortar_sd + px);
  if (px > 1) c->mdv.assign(prob->mortar_dd_v, prob->mortar_dd_v + py * (px - 1));
  if (py > 1) c->mdh.assign(prob->mortar_dd_h, prob->mortar_dd_h + (py - 1) * px);
  if (prob->source) c->source.assign(prob->source, prob->source + px * py);
  for (int v : c->msd) if (v < 1) { delete c; return SFB_ERR_ARG; }
  for (int v : c->mdv) if (v < 1) { delete c; return SFB_ERR_ARG; }
  for (int v : c->mdh) if (v < 1) { delete c; return SFB_ERR_ARG; }
  c->prob.darcy_nx = c->nx.data();
  c->prob.darcy_ny = c->ny.data();
  c->prob.mortar_sd = c->msd.data();
  c->prob.mortar_dd_v = c->mdv.empty() ? nullptr : c->mdv.data();
  c->prob.mortar_dd_h = c->mdh.empty() ? nullptr : c->mdh.data();
  c->prob.source = c->source.empty() ? nullptr : c->source.data();
  sfb_status s = build_geometry(c);
  if (s != SFB_OK) {
    delete c;
    return s;
  }
  stokes_assemble_host(c);
  noalloc_preload();
  *out = c;
  return SFB_OK;
}

void sfb_destroy(sfb_ctx* c) { delete c; }

const char* sfb_last_error(const sfb_ctx* c) { return c ? c->err.c_str() : "null context"; }

sfb_status sfb_set_stream(sfb_ctx* c, void* stream) {
  if (!c) return SFB_ERR_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return SFB_OK;
}

sfb_status sfb_sizes(const sfb_ctx* c, int64_t* n_lambda, int32_t* n_darcy) {
  if (!c) return SFB_ERR_ARG;
  if (n_lambda) *n_lambda = c->n_lambda;
  if (n_darcy) *n_darcy = (int32_t)c->subs.size();
  return SFB_OK;
}

sfb_status sfb_subdomain_dofs(const sfb_ctx* c, int32_t sub, int32_t* n_dof, int64_t* gd) {
  if (!c || !n_dof || sub < -1 || sub >= (int)c->subs.size()) return SFB_ERR_ARG;
  const std::vector<int64_t>& v = sub < 0 ? c->stokes.dofs : c->subs[sub].dofs;
  *n_dof = (int32_t)v.size();
  if (gd) std::copy(v.begin(), v.end(), gd);
  return SFB_OK;
}

sfb_status sfb_field_size(const sfb_ctx* c, int32_t field, int64_t* n) {
  if (!c || !n || field < 0 || field > 3) return SFB_ERR_ARG;
  int64_t np_ = 0, nf_ = 0;
  for (const HostSub& S : c->subs) {
    np_ += (int64_t)S.nx * S.ny;
    nf_ += (int64_t)S.ny * (S.nx + 1) + (int64_t)(S.ny + 1) * S.nx;
  }
  const int64_t v[4] = {np_, nf_, (int64_t)c->stokes.n_u, (int64_t)c->stokes.n_p};
  *n = v[field];
  return SFB_OK;
}

sfb_status sfb_kl_setup_regions(sfb_ctx* c, const sfb_kl_region* regions, int32_t n_regions, const double* rects,
                                const int32_t* region_of, double* eig) {
  if (!c) return SFB_ERR_ARG;
  const int ns = (int)c->subs.size();
  if (!regions || !rects || !region_of || n_regions < 1 || n_regions > ns)
    return fail(c, SFB_ERR_ARG, "KL regions: 1..n_darcy regions with rectangles and a region per subdomain");
  std::vector<int> members(n_regions, 0);
  for (int s = 0; s < ns; ++s) {
    const int r = region_of[s];
    if (r < 0 || r >= n_regions) return fail(c, SFB_ERR_ARG, "KL regions: subdomain without a valid region");
    const double* R = rects + 4 * r;
    const HostSub& S = c->subs[s];
    const double tol = 1e-12 * std::max(1.0, std::max(std::fabs(R[1] - R[0]), std::fabs(R[3] - R[2])));
    if (!(R[1] > R[0]) || !(R[3] > R[2]) || S.x0 < R[0] - tol || S.x1 > R[1] + tol || S.y0 < R[2] - tol ||
        S.y1 > R[3] + tol)
      return fail(c, SFB_ERR_ARG, "KL regions: subdomain " + std::to_string(s) + " is not inside its region");
    ++members[r];
  }
  for (int r = 0; r < n_regions; ++r)
    if (!members[r]) return fail(c, SFB_ERR_ARG, "KL regions: region " + std::to_string(r) + " has no subdomain");
  // per region: the kept 2-D modes (eigenvalue, x index, y index) and the 1-D data
  struct RegionModes {
    std::vector<std::tuple<double, int, int>> modes;
    std::vector<double> omx, omy;
    std::vector<int> parx, pary;
  };
  std::vector<RegionModes> rm(n_regions);
  int64_t w = 0;
  for (int q = 0; q < n_regions; ++q) {
    const sfb_kl_region& r = regions[q];
    if (r.n_term < 1 || r.n_term > 64 || !(r.sigma2 >= 0) || !(r.eta1 > 0) || !(r.eta2 > 0))
      return fail(c, SFB_ERR_ARG, "bad KL region");
    const bool tensor_set = r.n_modes_x > 0 || r.n_modes_y > 0;
    if (tensor_set && (r.n_modes_x < 1 || r.n_modes_y < 1 || r.n_modes_x * r.n_modes_y != r.n_term))
      return fail(c, SFB_ERR_ARG, "KL region: n_modes_x * n_modes_y must equal n_term");
    const double Lx = rects[4 * q + 1] - rects[4 * q], Ly = rects[4 * q + 3] - rects[4 * q + 2];
    // candidate 1-D modes per direction: all n_term of each (largest
    // products), or exactly n_modes_x and n_modes_y (tensor set)
    const int na = tensor_set ? r.n_modes_x : r.n_term, nb = tensor_set ? r.n_modes_y : r.n_term;
    std::vector<double> lx, ly;
    kl_1d_host(Lx, r.eta1, na, rm[q].omx, lx, rm[q].parx);
    kl_1d_host(Ly, r.eta2, nb, rm[q].omy, ly, rm[q].pary);
    // by decreasing eigenvalue, ties broken by (a + b, a); the first n_term
    // are kept (all of them for a tensor set)
    std::vector<std::tuple<double, int, int>>& cand = rm[q].modes;
    for (int a = 0; a < na; ++a)
      for (int b = 0; b < nb; ++b) cand.emplace_back(r.sigma2 * lx[a] * ly[b], a, b);
    std::stable_sort(cand.begin(), cand.end(), [](const auto& p, const auto& q2) {
      if (std::get<0>(p) != std::get<0>(q2)) return std::get<0>(p) > std::get<0>(q2);
      const int sp = std::get<1>(p) + std::get<2>(p), sq = std::get<1>(q2) + std::get<2>(q2);
      if (sp != sq) return sp < sq;
      return std::get<1>(p) < std::get<1>(q2);
    });
    cand.resize(r.n_term);
    for (int j = 0; j < r.n_term; ++j)
      if (eig) eig[w++] = std::get<0>(cand[j]);
  }
  // every subdomain evaluates its region's modes at its own cell centres, in
  // the region's centred coordinates
  for (int s = 0; s < ns; ++s) {
    const int q = region_of[s];
    const sfb_kl_region& r = regions[q];
    const double* R = rects + 4 * q;
    const double Lx = R[1] - R[0], Ly = R[3] - R[2], cx = 0.5 * (R[0] + R[1]), cy = 0.5 * (R[2] + R[3]);
    HostSub& S = c->subs[s];
    S.n_term = r.n_term; S.sigma2 = r.sigma2; S.eta1 = r.eta1; S.eta2 = r.eta2; S.mean_y = r.mean_y;
    S.lam.assign(r.n_term, 0.0); S.slam.assign(r.n_term, 0.0);
    S.fx.assign((size_t)r.n_term * S.nx, 0.0); S.fy.assign((size_t)r.n_term * S.ny, 0.0);
    for (int j = 0; j < r.n_term; ++j) {
      const auto& md = rm[q].modes[j];
      const int a = std::get<1>(md), b = std::get<2>(md);
      S.lam[j] = std::get<0>(md);
      S.slam[j] = std::sqrt(S.lam[j]);
      for (int i = 0; i < S.nx; ++i)
        S.fx[(size_t)j * S.nx + i] =
            kl_1d_eval_host(S.x0 + (i + 0.5) * S.hx - cx, Lx, rm[q].omx[a], rm[q].parx[a]);
      for (int i = 0; i < S.ny; ++i)
        S.fy[(size_t)j * S.ny + i] =
            kl_1d_eval_host(S.y0 + (i + 0.5) * S.hy - cy, Ly, rm[q].omy[b], rm[q].pary[b]);
    }
  }
  c->region_of.assign(region_of, region_of + ns);
  c->n_regions = n_regions;
  c->kl_done = true;
  c->coll_done = false;
  c->basis_done = false;
  if (c->ws) c->ws_stale = true;   // its layout and tables describe the old set-up
  return SFB_OK;
}

sfb_status sfb_kl_setup(sfb_ctx* c, const sfb_kl_region* regions, int32_t n_regions, double* eig) {
  if (!c) return SFB_ERR_ARG;
  if (!regions || n_regions != (int)c->subs.size()) return fail(c, SFB_ERR_ARG, "one KL region per Darcy subdomain");
  // one region per subdomain, on the subdomain's own rectangle
  std::vector<double> rects(4 * (size_t)n_regions);
  std::vector<int32_t> region_of(n_regions);
  for (int s = 0; s < n_regions; ++s) {
    const HostSub& S = c->subs[s];
    rects[4 * s] = S.x0; rects[4 * s + 1] = S.x1; rects[4 * s + 2] = S.y0; rects[4 * s + 3] = S.y1;
    region_of[s] = s;
  }
  return sfb_kl_setup_regions(c, regions, n_regions, rects.data(), region_of.data(), eig);
}

sfb_status sfb_collocation_setup(sfb_ctx* c, const sfb_collocation* spec, int64_t* n_pts_out) {
  if (!c || !spec) return SFB_ERR_ARG;
  if (!c->kl_done) return fail(c, SFB_ERR_STATE, "sfb_kl_setup must come first");
  const int ns = (int)c->subs.size();
  // region r's stochastic dimensions follow those of regions 0..r-1 (Section
  // 2.1); a subdomain takes its region's
  int n_dim = 0;
  std::vector<int> reg_off(c->n_regions, 0);
  for (int r = 0; r < c->n_regions; ++r) {
    int s0 = 0;
    while (c->region_of[s0] != r) ++s0;
    reg_off[r] = n_dim;
    n_dim += c->subs[s0].n_term;
  }
  c->dim_off.assign(ns, 0);
  for (int s = 0; s < ns; ++s) c->dim_off[s] = reg_off[c->region_of[s]];
  std::vector<int> rule;
  if (spec->kind == 1 && spec->n_rule > 0) {
    if (!spec->rule) return fail(c, SFB_ERR_ARG, "rule missing");
    rule.assign(spec->rule, spec->rule + spec->n_rule);
  }
  // points per global dimension of a tensor grid (Section 4.1: isotropic m,
  // or the anisotropic multi-index m_dim)
  if (spec->local_tensor < 0 || spec->local_tensor > 2) return fail(c, SFB_ERR_ARG, "local_tensor must be 0, 1 or 2");
  std::vector<int> ms;
  if (spec->kind == 0) {
    if (spec->m_dim) ms.assign(spec->m_dim, spec->m_dim + n_dim);
    else ms.assign(n_dim, spec->m);
    double npts = 1.0;
    for (int m : ms) {
      if (m < 1 || m > 32) return fail(c, SFB_ERR_ARG, "bad tensor rule size");
      npts *= m;
    }
    if (npts > 5e7) return fail(c, SFB_ERR_UNSUPPORTED, "tensor grid too large");
    tensor_grid_host(ms, c->grid);
  } else if (spec->kind == 1) {
    if (spec->m_dim) return fail(c, SFB_ERR_ARG, "m_dim applies to tensor grids only");
    if (spec->lmax < 0 || spec->lmax > 6) return fail(c, SFB_ERR_ARG, "bad Smolyak level");
    smolyak_grid_host(n_dim, spec->lmax, rule, c->grid);
  } else {
    return fail(c, SFB_ERR_ARG, "unknown grid kind");
  }
  // local realizations (Section 5.4 Steps 1-2)
  c->loc_y.assign(ns, {});
  c->n_local.assign(ns, 0);
  const int64_t np_ = c->grid.n_pts();
  for (int s = 0; s < ns; ++s) {
    const int nt = c->subs[s].n_term;
    if (spec->local_tensor == 2) {
      // Method S2 (Section 5.3): one local realization per global point, no
      // reuse: the projections of all global points in order, repeats kept
      c->loc_y[s].resize((size_t)np_ * nt);
      for (int64_t l = 0; l < np_; ++l)
        for (int j = 0; j < nt; ++j) c->loc_y[s][(size_t)l * nt + j] = c->grid.y[l * n_dim + c->dim_off[s] + j];
      c->n_local[s] = (int)np_;
    } else if (spec->local_tensor) {
      // the region's own rules on a tensor grid; the largest 1-D rule of the
      // sequence on a Smolyak grid
      std::vector<int> lm;
      if (spec->kind == 0) {
        lm.assign(ms.begin() + c->dim_off[s], ms.begin() + c->dim_off[s] + nt);
      } else {
        int m = 1;
        for (int p = 0; p <= spec->lmax; ++p) m = std::max(m, rule_size_host(p, rule));
        lm.assign(nt, m);
      }
      Grid lg;
      tensor_grid_host(lm, lg);
      if (lg.n_pts() > 1000000) return fail(c, SFB_ERR_UNSUPPORTED, "local tensor grid too large");
      c->loc_y[s] = lg.y;
      c->n_local[s] = (int)lg.n_pts();
    } else {
      std::map<std::vector<int64_t>, std::vector<double>> uniq;
      for (int64_t l = 0; l < np_; ++l) {
        std::vector<int64_t> key(nt);
        std::vector<double> val(nt);
        for (int j = 0; j < nt; ++j) {
          val[j] = c->grid.y[l * n_dim + c->dim_off[s] + j];
          key[j] = qkey(val[j]);
        }
        uniq.emplace(key, val);
      }
      c->loc_y[s].clear();
      for (auto& kv : uniq) c->loc_y[s].insert(c->loc_y[s].end(), kv.second.begin(), kv.second.end());
      c->n_local[s] = (int)uniq.size();
    }
  }
  c->coll_done = true;
  c->basis_done = false;
  if (c->ws) c->ws_stale = true;   // its layout and tables describe the old set-up
  if (n_pts_out) *n_pts_out = np_;
  return SFB_OK;
}

sfb_status sfb_collocation_points(const sfb_ctx* c, double* y_out, double* w_out) {
  if (!c) return SFB_ERR_ARG;
  if (!c->coll_done) return SFB_ERR_STATE;
  if (y_out) std::copy(c->grid.y.begin(), c->grid.y.end(), y_out);
  if (w_out) std::copy(c->grid.w.begin(), c->grid.w.end(), w_out);
  return SFB_OK;
}

sfb_status sfb_kl_tables(const sfb_ctx* c, int32_t sub, double* sqrt_lambda, double* fx, double* fy) {
  if (!c || sub < 0 || sub >= (int)c->subs.size()) return SFB_ERR_ARG;
  if (!c->kl_done) return SFB_ERR_STATE;
  const HostSub& S = c->subs[sub];
  if (sqrt_lambda) std::copy(S.slam.begin(), S.slam.end(), sqrt_lambda);
  if (fx) std::copy(S.fx.begin(), S.fx.end(), fx);
  if (fy) std::copy(S.fy.begin(), S.fy.end(), fy);
  return SFB_OK;
}

sfb_status sfb_local_points(const sfb_ctx* c, int32_t region, int32_t* n_local, double* y_out) {
  if (!c || region < 0 || region >= (int)c->subs.size()) return SFB_ERR_ARG;
  if (!c->coll_done) return SFB_ERR_STATE;
  if (n_local) *n_local = c->n_local[region];
  if (y_out) std::copy(c->loc_y[region].begin(), c->loc_y[region].end(), y_out);
  return SFB_OK;
}

sfb_status sfb_workspace_size(const sfb_ctx* cc, int32_t prec, int64_t max_pts, size_t* bytes) {
  sfb_ctx* c = const_cast<sfb_ctx*>(cc);
  if (!c || !bytes || prec < 0 || prec > 2 || max_pts < 0) return SFB_ERR_ARG;
  if (!c->coll_done) return fail(c, SFB_ERR_STATE, "collocation set-up must come first");
  Carver cv;
  Dev saved = c->dev;
  *bytes = layout(c, cv, prec == SFB_FP64 ? SFB_FP64 : SFB_MIXED, max_pts);
  c->dev = saved;
  c->ws_prec = prec == SFB_FP64 ? SFB_FP64 : SFB_MIXED;
  c->ws_pts = max_pts;
  return SFB_OK;
}

sfb_status sfb_set_workspace(sfb_ctx* c, void* ptr, size_t bytes) {
  if (!c) return SFB_ERR_ARG;
  if (!ptr || ((uintptr_t)ptr & 255)) return fail(c, SFB_ERR_ARG, "workspace must be 256-byte aligned");
  if (!c->coll_done || c->ws_prec < 0)
    return fail(c, SFB_ERR_STATE, "sfb_workspace_size must come first");
  Carver cv0;
  Dev saved = c->dev;
  const size_t need = layout(c, cv0, c->ws_prec, c->ws_pts);
  c->dev = saved;
  if (bytes < need) return fail(c, SFB_ERR_WORKSPACE, "workspace smaller than sfb_workspace_size()");
  c->ws = reinterpret_cast<char*>(ptr);
  c->ws_bytes = bytes;
  c->ws_stale = false;
  // captured basis graphs hold the old workspace's addresses
  for (int q = 0; q < 3; ++q)
    if (c->bgraph[q]) {
      cudaGraphExecDestroy(c->bgraph[q]);
      c->bgraph[q] = nullptr;
    }
  c->basis_done = false;
  c->basis_prec = -1;
  c->n_solved = 0;
  c->mom_shift_set = false;
  c->gmaps_ws = nullptr;   // the tensor maps point into the workspace: encode them again
  Carver cv;
  cv.base = c->ws;
  layout(c, cv, c->ws_prec, c->ws_pts);
  return sfb_moments_reset(c);
}


}  // extern "C"

namespace {

// Uploads the set-up tables once per workspace (synchronous; they are small).
sfb_status upload_tables(sfb_ctx* c) {
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  const int ns = (int)c->subs.size();
  std::vector<SubDev> sd(ns);
  std::vector<double> proj, kl, yloc;
  std::vector<int> info;
  std::vector<int64_t> gdof;
  int64_t item0 = 0;
  c->max_nx = 0; c->max_cols = 0; c->max_R = 0;
  for (int s = 0; s < ns; ++s) {
    const HostSub& S = c->subs[s];
    SubDev& D = sd[s];
    D.nx = S.nx; D.ny = S.ny; D.R = (int)S.dofs.size(); D.n_term = S.n_term; D.n_local = c->n_local[s];
    D.x0 = S.x0; D.y0 = S.y0; D.hx = S.hx; D.hy = S.hy; D.nu = c->prob.nu_d; D.source = S.source;
    D.mean_y = S.mean_y;
    for (int q = 0; q < 4; ++q) {
      D.side_type[q] = S.side_type[q];
      D.side_val[q] = S.side_val[q];
      D.proj_off[q] = (int64_t)proj.size();
      proj.insert(proj.end(), S.proj[q].begin(), S.proj[q].end());
    }
    D.dofinfo_off = (int64_t)info.size();
    info.insert(info.end(), S.dofinfo.begin(), S.dofinfo.end());
    D.kl_off = (int64_t)kl.size();
    kl.insert(kl.end(), S.slam.begin(), S.slam.end());
    kl.insert(kl.end(), S.fx.begin(), S.fx.end());
    kl.insert(kl.end(), S.fy.begin(), S.fy.end());
    D.yloc_off = (int64_t)yloc.size();
    yloc.insert(yloc.end(), c->loc_y[s].begin(), c->loc_y[s].end());
    D.gdof_off = (int64_t)gdof.size();
    gdof.insert(gdof.end(), S.dofs.begin(), S.dofs.end());
    D.item0 = item0;
    item0 += c->n_local[s];
    c->max_nx = std::max(c->max_nx, S.nx);
    c->max_cols = std::max(c->max_cols, D.R + 1);
    c->max_R = std::max(c->max_R, D.R);
  }
  // items in decreasing cost: nx^3 ny (factor) + nx^2 ny (R+1) (solves)
  std::vector<int> order(c->n_items), isub(c->n_items), ik(c->n_items);
  std::vector<double> cost(c->n_items);
  for (int s = 0, id = 0; s < ns; ++s)
    for (int k = 0; k < c->n_local[s]; ++k, ++id) {
      const double nx = sd[s].nx, ny = sd[s].ny;
      cost[id] = nx * nx * nx * ny + nx * nx * ny * (sd[s].R + 1);
      isub[id] = s; ik[id] = k;
    }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int> item_sub(c->n_items), item_k(c->n_items);
  for (int64_t i = 0; i < c->n_items; ++i) { item_sub[i] = isub[order[i]]; item_k[i] = ik[order[i]]; }
  // size classes of the item list (wide grids first, since cost grows as nx^3)
  c->n_wide = 0; c->wide_nx = c->wide_cols = c->narrow_nx = c->narrow_cols = 0;
  for (int64_t i = 0; i < c->n_items; ++i) {
    const SubDev& D = sd[item_sub[i]];
    if (D.nx > 64) {
      c->n_wide = i + 1;
      c->wide_nx = std::max(c->wide_nx, D.nx);
      c->wide_cols = std::max(c->wide_cols, D.R + 1);
    } else {
      c->narrow_nx = std::max(c->narrow_nx, D.nx);
      c->narrow_cols = std::max(c->narrow_cols, D.R + 1);
    }
  }
  for (int64_t i = c->n_wide; i < c->n_items; ++i)
    if (sd[item_sub[i]].nx > 64) return fail(c, SFB_ERR_ARG, "basis items out of size-class order");
  // column chunks of the split launch shapes, class by class in item order
  std::vector<int> ch_item, ch_c0, ch_cnt;
  for (int q = 0; q < 2; ++q) {
    const int64_t i0 = q == 0 ? 0 : c->n_wide, i1 = q == 0 ? c->n_wide : c->n_items;
    c->chunk_start[q] = (int64_t)ch_item.size();
    for (int64_t i = i0; i < i1; ++i) {
      const int C = sd[item_sub[i]].R + 1, nch = chunk_count(C), base = chunk_base(C);
      for (int k = 0; k < nch; ++k) {
        ch_item.push_back((int)(i - i0));
        ch_c0.push_back(k * base);
        ch_cnt.push_back(k + 1 < nch ? base : C - base * (nch - 1));
      }
    }
    c->chunk_n[q] = (int64_t)ch_item.size() - c->chunk_start[q];
  }
  if ((int64_t)ch_item.size() != c->n_chunks) return fail(c, SFB_ERR_ARG, "column chunk count mismatch");
  c->h_chunk_item = ch_item;
  c->item_id.resize(c->n_items);
  for (int64_t i = 0; i < c->n_items; ++i) c->item_id[i] = sd[item_sub[i]].item0 + item_k[i];
  // interface-solve maps
  std::vector<int> ldof(4 * c->n_lambda, 0);
  std::vector<int> fill(c->n_lambda, 0);
  auto put = [&](int64_t g, int unit, int loc) {
    const int f = fill[g]++;
    if (f < 2) { ldof[4 * g + 2 * f] = unit; ldof[4 * g + 2 * f + 1] = loc; }
  };
  for (int s = 0; s < ns; ++s)
    for (size_t a = 0; a < c->subs[s].dofs.size(); ++a) put(c->subs[s].dofs[a], s, (int)a);
  for (size_t a = 0; a < c->stokes.dofs.size(); ++a) put(c->stokes.dofs[a], ns, (int)a);
  for (int64_t g = 0; g < c->n_lambda; ++g)
    if (fill[g] != 2) return fail(c, SFB_ERR_ARG, "a mortar DOF is not shared by exactly two subdomains");
  std::vector<int> if_off, if_n, if_moff, dof_if(c->n_lambda, 0);
  {
    int mo = 0;
    for (size_t e = 0; e < c->ifaces.size(); ++e) {
      const HostIface& f = c->ifaces[e];
      if_off.push_back((int)f.off);
      if_n.push_back(f.n_dof);
      if_moff.push_back(mo);
      mo += f.n_dof * f.n_dof;
      for (int i = 0; i < f.n_dof; ++i) dof_if[f.off + i] = (int)e;
    }
  }
  std::vector<int> yoff(2 * c->n_lambda);
  for (int64_t g = 0; g < c->n_lambda; ++g)
    for (int f = 0; f < 2; ++f) yoff[2 * g + f] = (int)(c->ybase[ldof[4 * g + 2 * f]] + ldof[4 * g + 2 * f + 1]);
  std::vector<int> dim_off(c->dim_off.begin(), c->dim_off.end());
  std::vector<int64_t> loc_off(ns, 0), cell_off(ns, 0), face_off(ns, 0);
  for (int s = 1; s < ns; ++s) {
    loc_off[s] = loc_off[s - 1] + c->n_local[s - 1];
    cell_off[s] = cell_off[s - 1] + (int64_t)sd[s - 1].nx * sd[s - 1].ny;
    face_off[s] = face_off[s - 1] + (int64_t)sd[s - 1].ny * (sd[s - 1].nx + 1) + (int64_t)(sd[s - 1].ny + 1) * sd[s - 1].nx;
  }
  std::vector<int> htab, hcap;
  std::vector<int64_t> hoff;
  build_hash_tables(c, htab, hoff, hcap);
#define UP(dst, vec) SFB_CUDA(cudaMemcpyAsync(dst, (vec).data(), sizeof((vec)[0]) * (vec).size(), cudaMemcpyHostToDevice, st), "upload")
  UP(d.subs, sd); UP(d.proj, proj); UP(d.dofinfo, info); UP(d.kl, kl); UP(d.yloc, yloc); UP(d.gdof, gdof);
  UP(d.item_sub, item_sub); UP(d.item_k, item_k); UP(d.off, c->offs);
  if (!ch_item.empty()) { UP(d.chunk_item, ch_item); UP(d.chunk_c0, ch_c0); UP(d.chunk_cnt, ch_cnt); }
  UP(d.s_gdof, c->stokes.dofs); UP(d.ybase, c->ybase); UP(d.dim_off, dim_off); UP(d.loc_off, loc_off);
  UP(d.cell_off, cell_off); UP(d.face_off, face_off); UP(d.ldof, ldof); UP(d.yoff, yoff);
  UP(d.if_off, if_off); UP(d.if_n, if_n); UP(d.if_moff, if_moff); UP(d.dof_if, dof_if); UP(d.hash, htab); UP(d.hash_off, hoff);
  UP(d.hash_cap, hcap); UP(d.bdd_cidx, c->bdd_cidx);
#undef UP
  SFB_CUDA(cudaStreamSynchronize(st), "upload");
  return SFB_OK;
}

// The basis build's autotuner. For each non-empty size class with more than
// one launch shape, every shape that keeps at least one CTA resident at the
// class's largest grid and column count runs the class's own items alone on
// the context stream: once untimed, then twice timed by CUDA events. The
// shape with the shorter of its two times is kept for later builds of this
// precision. The trial launches write the same outputs as the build that
// follows, which overwrites them and clears the per-item status first.
// A launch shape exists for the precision and size class, runs at least one
// CTA per SM at the class's largest grid and column count, and (tensor-core
// form) has its tensor maps.
bool shape_fits(int fp64, int wide, int v, int max_nx, int max_cols, bool have_maps) {
  BasisShape sd;
  if (!basis_shape_desc(fp64, wide, v, &sd) || (sd.tcgen05 && !have_maps)) return false;
  int ctas = 0;
  const cudaError_t e = basis_shape_ctas(fp64, wide, v, max_nx, max_cols, &ctas);
  if (e != cudaSuccess) cudaGetLastError();
  return e == cudaSuccess && ctas >= 1;
}

// A split shape's class as a pipeline: its items in G groups of decreasing
// cost (option "basis_pipe_groups", 1 to kPipeGroups); the factor launches of
// the groups run one after another on the class's stream, and each group's
// solve launch (its items' column chunks) on one of two further streams once
// that group's factor is done, so that factors, solves and the tails of both
// may overlap. Ordering is by stream events only: no kernel waits on another.
// On the precision workload (648 items of 64 x 64 cells) one group, all
// factors and then all chunks, built in 11.3 ms against 12.6 ms for two
// groups and 13.2 ms for four: a solve launch fills every SM, so the next
// group's factor did not run beside it. Adds its launches to *nk.
cudaError_t launch_class_pipeline(sfb_ctx* c, const BasisArgs& A, int q, int shape, int nx, int cols, int refine,
                                  cudaStream_t sa, int* nk) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    if (!c->pipe_stream[q][k]) e = cudaStreamCreateWithFlags(&c->pipe_stream[q][k], cudaStreamNonBlocking);
  for (cudaEvent_t& x : c->pipe_ev[q])
    if (e == cudaSuccess && !x) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  const int G = std::max(1, std::min<int>(c->opt_pipe_groups, A.n_items));
  cudaEvent_t* ev = c->pipe_ev[q];
  e = cudaEventRecord(ev[G], sa);   // fork
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c->pipe_stream[q][k], ev[G], 0);
  const int* chi = c->h_chunk_item.data() + c->chunk_start[q];
  int ch0 = 0;
  for (int g = 0; g < G && e == cudaSuccess; ++g) {
    const int i0 = (int)((int64_t)g * A.n_items / G), i1 = (int)((int64_t)(g + 1) * A.n_items / G);
    BasisArgs f = A;
    f.item_sub = A.item_sub + i0;
    f.item_k = A.item_k + i0;
    f.n_items = i1 - i0;
    e = launch_basis_part(f, q == 0, shape, 1, nx, cols, refine, sa);
    if (e == cudaSuccess) e = cudaEventRecord(ev[g], sa);
    int ch1 = ch0;
    while (ch1 < A.n_chunks && chi[ch1] < i1) ++ch1;
    BasisArgs v = A;
    v.chunk_item = A.chunk_item + ch0;
    v.chunk_c0 = A.chunk_c0 + ch0;
    v.chunk_cnt = A.chunk_cnt + ch0;
    v.n_chunks = ch1 - ch0;
    v.chunk_slot0 = A.chunk_slot0 + ch0;
    cudaStream_t sb = c->pipe_stream[q][g & 1];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, ev[g], 0);
    if (e == cudaSuccess) e = launch_basis_part(v, q == 0, shape, 2, nx, cols, refine, sb);
    *nk += 2;
    ch0 = ch1;
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {   // join
    e = cudaEventRecord(ev[G + 1 + k], c->pipe_stream[q][k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sa, ev[G + 1 + k], 0);
  }
  return e;
}

sfb_status autotune_basis(sfb_ctx* c, int prec, const BasisArgs* cls, const int* cls_nx, const int* cls_cols,
                          int refine) {
  const int fp64 = prec == SFB_FP64 ? 1 : 0;
  const int ns = basis_shape_count(fp64);
  cudaStream_t st = c->stream;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
    for (int v = 0; v < 4; ++v) c->btune_ms[prec][q][v] = 0.0;
    c->bshape[prec][q] = 0;
    if (cls[q].n_items == 0) continue;
    // the shapes of this class that fit at its sizes; one alone is not timed
    std::vector<int> fit;
    for (int v = 0; v < ns && v < 4; ++v)
      if (shape_fits(fp64, q == 0, v, cls_nx[q], cls_cols[q], cls[q].gmaps != nullptr)) fit.push_back(v);
    if (fit.size() == 1) c->bshape[prec][q] = fit[0];
    if (fit.size() < 2) continue;
    int best = -1;
    for (int v : fit) {
      if (e != cudaSuccess) break;
      float ms_min = 0.f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        if (rep > 0) e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) {
          int nk = 0;
          if (basis_shape_split(fp64, q == 0, v)) {
            e = launch_class_pipeline(c, cls[q], q, v, cls_nx[q], cls_cols[q], refine, st, &nk);
          } else {
            e = launch_basis_shape(cls[q], fp64, q == 0, v, cls_nx[q], cls_cols[q], refine, st);
            nk = 1;
          }
          c->launches += nk;
        }
        if (rep == 0 || e != cudaSuccess) continue;
        e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && (rep == 1 || ms < ms_min)) ms_min = ms;
      }
      if (e != cudaSuccess) break;
      c->btune_ms[prec][q][v] = ms_min;
      if (best < 0 || ms_min < c->btune_ms[prec][q][best]) best = v;
    }
    if (best >= 0) c->bshape[prec][q] = best;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return cuda_fail(c, e, "basis autotuner");
  c->btuned[prec] = true;
  return SFB_OK;
}

// Tensor maps of every item's block inverses for the tensor-core basis kernel:
// the item's hi and lo arrays, [2][ny][np][np] FP32, as one row-major 2-D
// tensor of np columns and 2 ny np rows, read in boxes of 4 columns by np
// rows (one K-chunk of the product's A operand, which the copy lays down in
// the core-matrix layout). Encoded once per workspace with the driver's
// cuTensorMapEncodeTiled (looked up through the runtime, so the library does
// not link the driver); false when the driver cannot encode them, and the
// tensor-core launch shape is then skipped.
bool encode_gmaps(sfb_ctx* c) {
  if (c->gmaps_ws == c->ws) return c->gmaps_ok;
  c->gmaps_ws = c->ws;
  c->gmaps_ok = false;
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  std::vector<CUtensorMap> maps((size_t)c->n_items);
  int64_t id = 0;
  for (int s = 0; s < (int)c->subs.size(); ++s) {
    const HostSub& H = c->subs[s];
    const cuuint64_t np = (cuuint64_t)((H.nx + kPanel - 1) / kPanel * kPanel);
    for (int k = 0; k < c->n_local[s]; ++k, ++id) {
      float* base = reinterpret_cast<float*>(c->dev.G) + c->offs[id].g;
      const cuuint64_t dims[2] = {np, 2 * (cuuint64_t)H.ny * np};
      const cuuint64_t strides[1] = {np * 4};
      const cuuint32_t box[2] = {4, (cuuint32_t)np};
      const cuuint32_t es[2] = {1, 1};
      const CUresult r = enc(&maps[id], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  if (cudaMemcpyAsync(c->dev.gmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->gmaps_ok = true;
  return true;
}

bool host_or_device_copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st) == cudaSuccess;
}

}  // namespace

extern "C" {

sfb_status sfb_build_stochastic_basis(sfb_ctx* c, int32_t prec, sfb_basis_stats* stats) {
  if (!c) return SFB_ERR_ARG;
  if (prec < 0 || prec > SFB_FACTOR_FP64) return fail(c, SFB_ERR_ARG, "bad precision");
  if (!c->ws) return fail(c, SFB_ERR_WORKSPACE, "no workspace set");
  if (c->ws_stale)
    return fail(c, SFB_ERR_STATE, "set-up changed after sfb_set_workspace: call sfb_workspace_size and "
                                  "sfb_set_workspace again");
  if ((prec == SFB_FP64 || prec == SFB_FACTOR_FP64) && c->ws_prec != SFB_FP64)
    return fail(c, SFB_ERR_WORKSPACE, "workspace was sized for the FP32 factor; FP64 needs more");
  // Method S1's set-up: the FP64 kernel with the particular right-hand side
  // only, launched plainly with the FP64 build's launch shapes
  const bool factor_only = prec == SFB_FACTOR_FP64;
  if (factor_only) prec = SFB_FP64;
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  if (c->basis_prec < 0) {
    sfb_status s = upload_tables(c);
    if (s != SFB_OK) return s;
    cudaError_t e = stokes_solve_device(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "Stokes basis");
    int sst = 0;
    SFB_CUDA(cudaMemcpyAsync(&sst, d.s_status, sizeof(int), cudaMemcpyDeviceToHost, st), "Stokes status");
    SFB_CUDA(cudaStreamSynchronize(st), "Stokes basis");
    if (sst) return fail(c, SFB_ERR_NOT_SPD, "zero pivot in the Stokes factorization");
    c->basis_prec = 99;  // tables and Stokes basis present
    c->bdd_stokes_ready = false;
  }
  const int n = (int)c->n_items;
  BasisArgs a;
  a.subs = d.subs; a.proj = d.proj; a.dofinfo = d.dofinfo; a.kl = d.kl; a.yloc = d.yloc;
  a.item_sub = d.item_sub; a.item_k = d.item_k; a.off = d.off; a.n_items = n;
  a.X = d.X; a.T = d.T; a.G = d.G; a.Z = d.Z; a.S = d.S; a.DL = d.DL; a.phi = d.phi; a.phi32 = d.phi32; a.D = d.D;
  a.status = d.status; a.resid = d.resid; a.corr1 = d.corr1; a.errest = d.errest; a.nref = d.nref;
  a.cycles = d.cycles;
  a.max_refine = c->opt_refine_max;
  a.refine_tol = c->opt_refine_tol;
  a.particular_only = factor_only ? 1 : 0;
  if (prec != SFB_FP64 && encode_gmaps(c)) a.gmaps = d.gmaps;
  // size classes: [0] grids wider than 64 cells (the first n_wide items), [1] the rest
  const int fp64 = prec == SFB_FP64 ? 1 : 0;
  const int refine = prec == SFB_MIXED ? a.max_refine : 0;
  a.n_items_all = n;
  BasisArgs cls[2] = {a, a};
  cls[0].n_items = (int)c->n_wide;
  cls[1].item_sub = a.item_sub + c->n_wide;
  cls[1].item_k = a.item_k + c->n_wide;
  cls[1].n_items = n - (int)c->n_wide;
  for (int q = 0; q < 2; ++q) {
    cls[q].chunk_item = d.chunk_item + c->chunk_start[q];
    cls[q].chunk_c0 = d.chunk_c0 + c->chunk_start[q];
    cls[q].chunk_cnt = d.chunk_cnt + c->chunk_start[q];
    cls[q].n_chunks = (int)c->chunk_n[q];
    cls[q].chunk_slot0 = (int)c->chunk_start[q];
  }
  const int cls_nx[2] = {c->wide_nx, c->narrow_nx}, cls_cols[2] = {c->wide_cols, c->narrow_cols};
  if (c->opt_basis_autotune && !c->btuned[prec] && !factor_only) {
    sfb_status s = autotune_basis(c, prec, cls, cls_nx, cls_cols, refine);
    if (s != SFB_OK) return s;
  }
  SFB_CUDA(cudaMemsetAsync(d.status, 0, sizeof(int) * n, st), "memset");
  const int64_t nu_st = n + c->n_chunks;   // statistics slots: items, then chunks
  SFB_CUDA(cudaMemsetAsync(d.resid, 0, sizeof(double) * nu_st, st), "memset");
  SFB_CUDA(cudaMemsetAsync(d.corr1, 0, sizeof(double) * nu_st, st), "memset");
  SFB_CUDA(cudaMemsetAsync(d.errest, 0, sizeof(double) * nu_st, st), "memset");
  SFB_CUDA(cudaMemsetAsync(d.nref, 0, sizeof(int) * nu_st, st), "memset");
  SFB_CUDA(cudaMemsetAsync(d.cycles, 0, sizeof(long long) * kCycSlots * nu_st, st), "memset");
  int shp[2] = {c->bshape[prec][0], c->bshape[prec][1]};
  // a shape this class lacks or that does not fit (or the tensor-core one
  // without maps): the first shape that fits
  for (int q = 0; q < 2; ++q) {
    if (cls[q].n_items == 0 || shape_fits(fp64, q == 0, shp[q], cls_nx[q], cls_cols[q], a.gmaps != nullptr)) continue;
    shp[q] = 0;
    for (int v = 0; v < basis_shape_count(fp64); ++v)
      if (shape_fits(fp64, q == 0, v, cls_nx[q], cls_cols[q], a.gmaps != nullptr)) { shp[q] = v; break; }
  }
  const bool two = cls[0].n_items > 0 && cls[1].n_items > 0;
  if (two) {
    if (!c->side) SFB_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "stream");
    if (!c->fork) SFB_CUDA(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "event");
    if (!c->join) SFB_CUDA(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming), "event");
  }
  // One launch per size class (a pipeline for a split shape): wide grids on
  // the main stream, narrow grids concurrently on a side stream joined back
  // before the epilogue.
  auto run_class = [&](int q, cudaStream_t sq, int* nk) -> cudaError_t {
    if (basis_shape_split(fp64, q == 0, shp[q]))
      return launch_class_pipeline(c, cls[q], q, shp[q], cls_nx[q], cls_cols[q], refine, sq, nk);
    *nk += 1;
    return launch_basis_shape(cls[q], fp64, q == 0, shp[q], cls_nx[q], cls_cols[q], refine, sq);
  };
  // The persistent form: one launch over every item of both classes (FP32
  // factor, not Method S1's set-up); the autotuner times it against the
  // per-class launches above (option "basis_persistent": -1 the autotuner
  // decides, 0 never, 1 always).
  BasisArgs pa = a;
  pa.n_items = n;
  pa.chunk_item = d.chunk_item;
  pa.chunk_c0 = d.chunk_c0;
  pa.chunk_cnt = d.chunk_cnt;
  pa.n_chunks = (int)c->n_chunks;
  pa.chunk_slot0 = 0;
  const int all_nx = std::max(cls_nx[0], cls_nx[1]), all_cols = std::max(cls_cols[0], cls_cols[1]);
  int pctas = 0;
  const bool can_persist = !fp64 && !factor_only && n > 0 && all_nx <= 128 &&
                           launch_basis_persistent(pa, d.persist_counter, d.persist_flags, (int)c->n_wide,
                                                   (int)c->chunk_n[0], all_nx, all_cols, refine, st, &pctas) ==
                               cudaSuccess &&
                           pctas >= 1;
  cudaGetLastError();
  auto issue_persistent = [&](cudaStream_t s0, int* nk) -> cudaError_t {
    *nk = 1;
    return launch_basis_persistent(pa, d.persist_counter, d.persist_flags, (int)c->n_wide, (int)c->chunk_n[0], all_nx,
                                   all_cols, refine, s0, nullptr);
  };
  auto issue_classes = [&](cudaStream_t s0, int* nk) -> cudaError_t {
    *nk = 0;
    if (!two) return run_class(cls[0].n_items > 0 ? 0 : 1, s0, nk);
    cudaError_t e = cudaEventRecord(c->fork, s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
    if (e == cudaSuccess) e = run_class(0, s0, nk);
    if (e == cudaSuccess) e = run_class(1, c->side, nk);
    if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, c->join, 0);
    return e;
  };
  bool persist = can_persist && c->opt_basis_persistent == 1;
  if (can_persist && c->opt_basis_persistent == -1 && c->opt_basis_autotune) {
    if (!c->bpersist_tuned[prec]) {
      // one untimed and two timed builds of each form; the shorter time wins
      cudaEvent_t t0 = nullptr, t1 = nullptr;
      cudaError_t e = cudaEventCreate(&t0);
      if (e == cudaSuccess) e = cudaEventCreate(&t1);
      float best[2] = {0.f, 0.f};
      for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
          int nk = 0;
          e = cudaEventRecord(t0, st);
          if (e == cudaSuccess) e = form == 0 ? issue_classes(st, &nk) : issue_persistent(st, &nk);
          c->launches += nk;
          if (e == cudaSuccess) e = cudaEventRecord(t1, st);
          if (e == cudaSuccess) e = cudaEventSynchronize(t1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
          if (e == cudaSuccess && rep > 0 && (rep == 1 || ms < best[form])) best[form] = ms;
        }
      }
      if (t0) cudaEventDestroy(t0);
      if (t1) cudaEventDestroy(t1);
      if (e != cudaSuccess) return cuda_fail(c, e, "basis autotuner (persistent form)");
      c->bpersist_ms[prec][0] = best[0];
      c->bpersist_ms[prec][1] = best[1];
      c->bpersist[prec] = best[1] < best[0];
      c->bpersist_tuned[prec] = true;
    }
    persist = c->bpersist[prec];
  }
  auto issue = [&](cudaStream_t s0, int* nk) -> cudaError_t {
    return persist ? issue_persistent(s0, nk) : issue_classes(s0, nk);
  };
  // The launches of all size classes as one CUDA graph, captured on a private
  // stream (the context stream may be the legacy default stream, which cannot
  // capture) and replayed on the context stream while the workspace, the
  // refinement options and the launch shapes stay the same. A context stream
  // that is itself being captured (the caller's graph) gets the plain launches.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SFB_CUDA(cudaStreamIsCapturing(st, &cap), "capture status");
  const bool graph = c->opt_basis_graph && cap == cudaStreamCaptureStatusNone && !factor_only;
  if (graph) {
    sfb_ctx::GraphKey key;
    key.ws = c->ws;
    key.refine = refine;
    key.refine_tol = a.refine_tol;
    key.shape[0] = shp[0];
    key.shape[1] = shp[1];
    key.persist = persist ? 1 : 0;
    key.groups = c->opt_pipe_groups;
    if (c->bgraph[prec] && !(c->bkey[prec] == key)) {
      cudaGraphExecDestroy(c->bgraph[prec]);
      c->bgraph[prec] = nullptr;
    }
    if (!c->bgraph[prec]) {
      if (!c->gcap) SFB_CUDA(cudaStreamCreateWithFlags(&c->gcap, cudaStreamNonBlocking), "stream");
      cudaGraph_t g = nullptr;
      int nk = 0;
      cudaError_t e = cudaStreamBeginCapture(c->gcap, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        const cudaError_t el = issue(c->gcap, &nk);
        const cudaError_t ec = cudaStreamEndCapture(c->gcap, &g);
        e = el != cudaSuccess ? el : ec;
      }
      cudaGraphExec_t ex = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "basis graph capture");
      c->bgraph[prec] = ex;
      c->bkey[prec] = key;
      c->bgraph_kernels[prec] = nk;
    }
  }
  // timing events, released on every return
  struct Events {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  cudaEvent_t &e0 = evs.e[0], &e1 = evs.e[1], &ek = evs.e[2];
  SFB_CUDA(cudaEventCreate(&e0), "event");
  SFB_CUDA(cudaEventCreate(&e1), "event");
  SFB_CUDA(cudaEventCreate(&ek), "event");
  SFB_CUDA(cudaEventRecord(e0, st), "event");
  cudaError_t e = cudaSuccess;
  if (graph) {
    e = cudaGraphLaunch(c->bgraph[prec], st);
    c->launches += c->bgraph_kernels[prec];
  } else {
    int nk = 0;
    e = issue(st, &nk);
    c->launches += nk;
  }
  c->last_build_graph = graph;
  if (e != cudaSuccess) return cuda_fail(c, e, "basis kernel");
  SFB_CUDA(cudaEventRecord(ek, st), "event");
  e = launch_flux_epilogue(a, c->max_R, st);
  c->launches += 1;
  if (e != cudaSuccess) return cuda_fail(c, e, "flux epilogue");
  SFB_CUDA(cudaEventRecord(e1, st), "event");
  std::vector<int> status(n), nref(nu_st);
  std::vector<double> resid(nu_st), corr(nu_st), est(nu_st);
  std::vector<long long> cyc(kCycSlots * (size_t)nu_st);
  SFB_CUDA(cudaMemcpyAsync(status.data(), d.status, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaMemcpyAsync(nref.data(), d.nref, sizeof(int) * nu_st, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaMemcpyAsync(resid.data(), d.resid, sizeof(double) * nu_st, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaMemcpyAsync(corr.data(), d.corr1, sizeof(double) * nu_st, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaMemcpyAsync(est.data(), d.errest, sizeof(double) * nu_st, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaMemcpyAsync(cyc.data(), d.cycles, sizeof(long long) * kCycSlots * nu_st, cudaMemcpyDeviceToHost, st), "stats");
  SFB_CUDA(cudaStreamSynchronize(st), "basis build");
  // a split class's refinement statistics come per chunk: fold them into the
  // chunk's item (largest residual, correction, estimate and step count;
  // the chunks' clocks summed)
  for (int q = 0; q < 2; ++q) {
    if (cls[q].n_items == 0 || !(persist || basis_shape_split(fp64, q == 0, shp[q]))) continue;
    const int64_t i0 = q == 0 ? 0 : c->n_wide;
    std::vector<char> seen(n, 0);
    for (int64_t k = 0; k < c->chunk_n[q]; ++k) {
      const int64_t slot = n + c->chunk_start[q] + k;
      const int64_t id = c->item_id[i0 + c->h_chunk_item[(size_t)(c->chunk_start[q] + k)]];
      if (!seen[id]) { nref[id] = 0; resid[id] = corr[id] = est[id] = 0.0; seen[id] = 1; }
      nref[id] = std::max(nref[id], nref[slot]);
      resid[id] = std::max(resid[id], resid[slot]);
      corr[id] = std::max(corr[id], corr[slot]);
      est[id] = std::max(est[id], est[slot]);
      for (int e = 2; e < kCycSlots; ++e) cyc[kCycSlots * (size_t)id + e] += cyc[kCycSlots * (size_t)slot + e];
    }
  }
  float ms = 0.f, kms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventElapsedTime(&kms, e0, ek);
  int any = 0, n_nc = 0;
  for (int i = 0; i < n; ++i) { any |= status[i]; n_nc += (status[i] & ST_NOT_CONVERGED) != 0; }
  if (stats) {
    stats->n_items = n;
    int64_t fr = 0;
    for (int s = 0; s < (int)c->subs.size(); ++s) fr += (int64_t)c->subs[s].dofs.size() * c->n_local[s];
    stats->n_flux_responses = factor_only ? 0 : fr;
    stats->max_refine_steps = n ? *std::max_element(nref.begin(), nref.end()) : 0;
    double nref_sum = 0.0;
    for (int i = 0; i < n; ++i) nref_sum += nref[i];
    stats->mean_refine_steps = n ? nref_sum / n : 0.0;
    stats->n_not_converged = n_nc;
    stats->max_rel_residual = n ? *std::max_element(resid.begin(), resid.end()) : 0.0;
    stats->max_first_correction = n ? *std::max_element(corr.begin(), corr.end()) : 0.0;
    stats->max_error_estimate = n ? *std::max_element(est.begin(), est.end()) : 0.0;
    for (int q = 0; q < kCycSlots; ++q) {
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += (double)cyc[kCycSlots * (size_t)i + q];
      stats->phase_cycles[q] = n ? acc / n : 0.0;
    }
    stats->ms = ms;
    stats->kernel_ms = kms;
    double f32 = 0.0, f64 = 0.0;
    int64_t id = 0;
    for (int s = 0; s < (int)c->subs.size(); ++s) {
      const HostSub& H = c->subs[s];
      const double nx = H.nx, ny = H.ny, C = factor_only ? 1.0 : (double)H.dofs.size() + 1.0;
      const double fac = 7.0 / 3.0 * nx * nx * nx * ny, sol = 6.0 * nx * nx * ny * C, pass = 11.0 * nx * ny * C;
      for (int k = 0; k < c->n_local[s]; ++k, ++id) {
        if (prec == SFB_FP64) {
          f64 += fac + sol;
        } else {
          f32 += fac + (1.0 + nref[id]) * sol;
          f64 += nref[id] * pass;
        }
      }
    }
    stats->flops_fp32 = f32;
    stats->flops_fp64 = f64;
    for (int q = 0; q < 2; ++q) {
      stats->launch_shape[q] = cls[q].n_items > 0 ? shp[q] : -1;
      for (int v = 0; v < 4; ++v) stats->tune_ms[q][v] = c->btune_ms[prec][q][v];
    }
    stats->graph = graph ? 1 : 0;
    stats->persistent = persist ? 1 : 0;
  }
  c->basis_done = true;
  c->basis_prec = factor_only ? SFB_FACTOR_FP64 : prec;
  c->bdd_items_ready = false;   // the balancing preconditioner's pseudo-inverses follow the bases
  if (any & ST_NONFINITE) return fail(c, SFB_ERR_NONFINITE, "non-finite permeability or solution");
  if (any & ST_NOT_SPD) return fail(c, SFB_ERR_NOT_SPD, "non-positive pivot in a block factorization");
  if (any & ST_TIMEOUT) return fail(c, SFB_ERR_TIMEOUT, "a bulk copy did not complete within the wait limit");
  if (any & ST_NOT_CONVERGED) return fail(c, SFB_ERR_NOT_CONVERGED, "iterative refinement stopped above tolerance");
  return SFB_OK;
}

sfb_status sfb_basis_launch_shape(int32_t prec, int32_t wide, int32_t shape, int32_t* threads,
                                  int32_t* ctas_per_sm, int32_t* g_buffers, int32_t* tcgen05, int32_t* split) {
  if (prec < 0 || prec > 2 || (wide != 0 && wide != 1)) return SFB_ERR_ARG;
  BasisShape d;
  if (!basis_shape_desc(prec == SFB_FP64, wide, shape, &d)) return SFB_ERR_ARG;
  if (threads) *threads = d.threads;
  if (ctas_per_sm) *ctas_per_sm = d.min_ctas;
  if (g_buffers) *g_buffers = d.g_buffers;
  if (tcgen05) *tcgen05 = d.tcgen05;
  if (split) *split = d.split;
  return SFB_OK;
}

sfb_status sfb_get_basis(sfb_ctx* c, int32_t sub, int32_t k, double* phi, double* g, double* x) {
  if (!c) return SFB_ERR_ARG;
  if (!c->basis_done) return fail(c, SFB_ERR_STATE, "no basis built");
  cudaStream_t st = c->stream;
  if (sub == -1) {
    const int Rs = (int)c->stokes.dofs.size();
    if (k != 0 || x) return fail(c, SFB_ERR_ARG, "Stokes basis: k = 0, x = NULL");
    if (phi) SFB_CUDA(cudaMemcpyAsync(phi, c->dev.s_phi, sizeof(double) * Rs * Rs, cudaMemcpyDefault, st), "copy");
    if (g) SFB_CUDA(cudaMemcpyAsync(g, c->dev.s_phi + Rs * Rs, sizeof(double) * Rs, cudaMemcpyDefault, st), "copy");
    SFB_CUDA(cudaStreamSynchronize(st), "copy");
    return SFB_OK;
  }
  if (sub < 0 || sub >= (int)c->subs.size() || k < 0 || k >= c->n_local[sub])
    return fail(c, SFB_ERR_ARG, "no such basis item");
  int64_t id = 0;
  for (int s = 0; s < sub; ++s) id += c->n_local[s];
  id += k;
  const ItemOff& o = c->offs[id];
  const HostSub& S = c->subs[sub];
  const int R = (int)S.dofs.size();
  if (phi && c->basis_prec == SFB_FACTOR_FP64)
    return fail(c, SFB_ERR_STATE, "the factor-only build forms no flux basis: phi must be NULL");
  if (phi) SFB_CUDA(cudaMemcpyAsync(phi, c->dev.phi + o.phi, sizeof(double) * R * R, cudaMemcpyDefault, st), "copy");
  if (g) SFB_CUDA(cudaMemcpyAsync(g, c->dev.phi + o.phi + (int64_t)R * R, sizeof(double) * R, cudaMemcpyDefault, st), "copy");
  if (x) SFB_CUDA(cudaMemcpyAsync(x, c->dev.X + o.x, sizeof(double) * (size_t)S.nx * S.ny * (R + 1),
                                  cudaMemcpyDefault, st), "copy");  // [R+1][n_cells]
  SFB_CUDA(cudaStreamSynchronize(st), "copy");
  return SFB_OK;
}

sfb_status sfb_interface_solve_batch(sfb_ctx* c, const double* y, const double* w, int64_t n_pts, int32_t krylov,
                                     double rtol, int32_t max_it, double* lambda_out, int32_t* iters_out) {
  if (!c) return SFB_ERR_ARG;
  if (!c->basis_done) return fail(c, SFB_ERR_STATE, "sfb_build_stochastic_basis must come first");
  if (n_pts < 0 || krylov < SFB_CG || krylov > SFB_CG_DTN || !(rtol > 0) || max_it < 1)
    return fail(c, SFB_ERR_ARG, "bad interface solve arguments");
  if (krylov == SFB_CG_DTN && c->basis_prec != SFB_FP64 && c->basis_prec != SFB_FACTOR_FP64)
    return fail(c, SFB_ERR_STATE, "SFB_CG_DTN needs the FP64 block factors (an SFB_FP64 or SFB_FACTOR_FP64 build)");
  if (krylov != SFB_CG_DTN && c->basis_prec == SFB_FACTOR_FP64)
    return fail(c, SFB_ERR_STATE, "the factor-only build forms no flux basis: only SFB_CG_DTN solves from it");
  if (c->opt_cg_precond == 3 && krylov != SFB_CG && krylov != SFB_CG_DTN)
    return fail(c, SFB_ERR_ARG, "the balancing preconditioner (cg_precond 3) runs with SFB_CG");
  if (c->opt_cg_precond == 3 && krylov == SFB_CG && c->bdd_nc > 16)
    return fail(c, SFB_ERR_UNSUPPORTED, "the balancing preconditioner takes at most 16 floating subdomains");
  if (krylov == SFB_CG_DTN) {
    int mnx = 1, mny = 1, mR = 1;
    for (const HostSub& H : c->subs) {
      mnx = std::max(mnx, H.nx);
      mny = std::max(mny, H.ny);
      mR = std::max(mR, (int)H.dofs.size());
    }
    if (dtn_smem_bytes(mnx, mny, mR) > 227 * 1024)
      return fail(c, SFB_ERR_UNSUPPORTED, "SFB_CG_DTN keeps a subdomain's forward sweep in shared memory: grid too large");
  }
  if (n_pts == 0) return SFB_OK;  // an empty batch changes nothing
  if (!y || !w) return fail(c, SFB_ERR_ARG, "bad interface solve arguments");
  if (n_pts > c->ws_pts) return fail(c, SFB_ERR_WORKSPACE, "batch larger than the workspace was sized for");
  Dev& d = c->dev;
  cudaStream_t st = c->stream;
  const int nd = c->grid.n_dim;
  if (!host_or_device_copy(d.y, y, sizeof(double) * n_pts * nd, st) ||
      !host_or_device_copy(d.w, w, sizeof(double) * n_pts, st))
    return fail(c, SFB_ERR_CUDA, "copy of the points");
  int n_failed = 0;
  sfb_status s = iface_solve_device(c, n_pts, rtol, max_it, krylov, &n_failed);
  if (s != SFB_OK) return s;
  s = moments_accumulate_device(c, n_pts);
  if (s != SFB_OK) return s;
  if (lambda_out)
    SFB_CUDA(cudaMemcpyAsync(lambda_out, d.lam, sizeof(double) * n_pts * c->n_lambda, cudaMemcpyDefault, st),
             "copy lambda");
  if (iters_out)
    SFB_CUDA(cudaMemcpyAsync(iters_out, d.pstat, sizeof(int) * n_pts, cudaMemcpyDefault, st), "copy iters");
  int mflags = 0;
  SFB_CUDA(cudaMemcpyAsync(&mflags, d.active + 2, sizeof(int), cudaMemcpyDeviceToHost, st), "copy flags");
  SFB_CUDA(cudaStreamSynchronize(st), "interface solve");
  if (mflags & (4 | 8 | 16))
    return fail(c, SFB_ERR_CUDA, "moments: malformed point-by-point work list (flags " + std::to_string(mflags) + ")");
  c->n_solved += n_pts;
  if (n_failed) return fail(c, SFB_ERR_NOT_CONVERGED, std::to_string(n_failed) + " points did not converge");
  return SFB_OK;
}

sfb_status sfb_moments(sfb_ctx* c, int32_t field, double* mean_out, double* var_out) {
  if (!c || field < 0 || field > 3) return SFB_ERR_ARG;
  if (c->n_solved == 0) return fail(c, SFB_ERR_STATE, "no point solved since the last reset");
  const int64_t n = c->mom_len[field];
  sfb_status s = moments_finalize_device(c, field, c->dev.fin, c->dev.fin + n);
  if (s != SFB_OK) return s;
  if (mean_out) SFB_CUDA(cudaMemcpyAsync(mean_out, c->dev.fin, sizeof(double) * n, cudaMemcpyDefault, c->stream), "copy");
  if (var_out) SFB_CUDA(cudaMemcpyAsync(var_out, c->dev.fin + n, sizeof(double) * n, cudaMemcpyDefault, c->stream), "copy");
  SFB_CUDA(cudaStreamSynchronize(c->stream), "moments");
  return SFB_OK;
}

sfb_status sfb_launch_count(const sfb_ctx* c, int64_t* n) {
  if (!c || !n) return SFB_ERR_ARG;
  *n = c->launches;
  return SFB_OK;
}

sfb_status sfb_solve_timings(sfb_ctx* c, double* ms_out, int32_t* cg_iterations) {
  if (!c || !ms_out) return SFB_ERR_ARG;
  if (c->n_solved == 0 || !c->ev[5]) return fail(c, SFB_ERR_STATE, "no interface solve yet");
  SFB_CUDA(cudaEventSynchronize(c->ev[5]), "timings");
  float t[5];
  for (int q = 0; q < 5; ++q) SFB_CUDA(cudaEventElapsedTime(&t[q], c->ev[q], c->ev[q + 1]), "timings");
  ms_out[0] = t[0];          // index conversion and grouping
  ms_out[1] = t[1];          // CG iterations
  ms_out[2] = t[2];          // status bookkeeping
  ms_out[3] = t[3];          // Darcy moments
  ms_out[4] = t[4];          // Stokes moments and weights
  if (cg_iterations) *cg_iterations = c->cg_iters_run;
  return SFB_OK;
}

sfb_status sfb_cg_phase_cycles(const sfb_ctx* c, double* cycles_out) {
  if (!c || !cycles_out) return SFB_ERR_ARG;
  for (int k = 0; k < 6; ++k) cycles_out[k] = c->pcg_cycles[k];
  return SFB_OK;
}

sfb_status sfb_set_option(sfb_ctx* c, const char* name, double value) {
  if (!c || !name) return SFB_ERR_ARG;
  const std::string n(name);
  if (n == "refine_tol") {
    if (!(value > 0 && value < 1)) return fail(c, SFB_ERR_ARG, "refine_tol must lie in (0, 1)");
    c->opt_refine_tol = value;
  } else if (n == "refine_max") {
    if (!(value >= 1 && value <= 50)) return fail(c, SFB_ERR_ARG, "refine_max must lie in [1, 50]");
    c->opt_refine_max = (int)value;
  } else if (n == "moments_group_factor") {
    if (!(value >= 0 && value <= 1e6)) return fail(c, SFB_ERR_ARG, "moments_group_factor must lie in [0, 1e6]");
    c->opt_big_factor = value;
  } else if (n == "cg_check_every") {
    if (!(value >= 1 && value <= 1000)) return fail(c, SFB_ERR_ARG, "cg_check_every must lie in [1, 1000]");
    c->opt_cg_chunk = (int)value;
  } else if (n == "cg_precond") {
    if (!(value == 0 || value == 1 || value == 2 || value == 3)) return fail(c, SFB_ERR_ARG, "cg_precond must be 0, 1, 2 or 3");
    c->opt_cg_precond = (int)value;
  } else if (n == "moments_double_float") {
    if (!(value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "moments_double_float must be 0 or 1");
    c->opt_mom_df = (int)value;
  } else if (n == "cg_test_barrier_timeout") {
    if (!(value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "cg_test_barrier_timeout must be 0 or 1");
    c->test_barrier_skip = (int)value;
  } else if (n == "cg_persistent") {
    if (!(value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "cg_persistent must be 0 or 1");
    c->opt_cg_persistent = (int)value;
  } else if (n == "basis_autotune") {
    if (!(value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "basis_autotune must be 0 or 1");
    c->opt_basis_autotune = (int)value;
    for (int p = 0; p < 3; ++p) {
      c->btuned[p] = false;
      c->bpersist_tuned[p] = false;
      c->bshape[p][0] = c->bshape[p][1] = 0;
    }
  } else if (n == "basis_shape") {
    if (!(value >= 0 && value < 4 && value == (int)value)) return fail(c, SFB_ERR_ARG, "basis_shape must be 0..3");
    const int v = (int)value;
    if (v >= basis_shape_count(0) && v >= basis_shape_count(1))
      return fail(c, SFB_ERR_ARG, "no precision has launch shape " + std::to_string(v));
    c->opt_basis_autotune = 0;
    for (int p = 0; p < 3; ++p) {
      for (int q = 0; q < 2; ++q) {
        BasisShape sd;
        c->bshape[p][q] = basis_shape_desc(p == SFB_FP64, q == 0, v, &sd) ? v : 0;
      }
      c->btuned[p] = true;
    }
  } else if (n == "basis_pipe_groups") {
    if (!(value >= 1 && value <= sfb_ctx::kPipeGroups && value == (int)value))
      return fail(c, SFB_ERR_ARG, "basis_pipe_groups must be 1.." + std::to_string(sfb_ctx::kPipeGroups));
    c->opt_pipe_groups = (int)value;
  } else if (n == "basis_persistent") {
    if (!(value == -1 || value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "basis_persistent must be -1, 0 or 1");
    c->opt_basis_persistent = (int)value;
    for (int p = 0; p < 3; ++p) c->bpersist_tuned[p] = false;
  } else if (n == "basis_graph") {
    if (!(value == 0 || value == 1)) return fail(c, SFB_ERR_ARG, "basis_graph must be 0 or 1");
    c->opt_basis_graph = (int)value;
  } else if (n == "gmres_restart") {
    if (!(value >= 1 && value <= kGmresMax && value == (int)value))
      return fail(c, SFB_ERR_ARG, "gmres_restart must be an integer in 1.." + std::to_string(kGmresMax));
    c->opt_gmres_m = (int)value;
  } else if (n == "cg_replace_ratio") {
    if (!(value >= 1e-4 && value < 1)) return fail(c, SFB_ERR_ARG, "cg_replace_ratio must lie in [1e-4, 1)");
    c->opt_cg_replace = value;
  } else {
    return fail(c, SFB_ERR_ARG, "unknown option " + n);
  }
  return SFB_OK;
}

sfb_status sfb_moments_reset(sfb_ctx* c) {
  if (!c) return SFB_ERR_ARG;
  if (!c->ws) return fail(c, SFB_ERR_WORKSPACE, "no workspace set");
  const int64_t len_d = c->mom_len[0] + c->mom_len[1];
  const int64_t Cs = (int64_t)c->stokes.dofs.size() + 1;
  SFB_CUDA(cudaMemsetAsync(c->dev.mom, 0, sizeof(double) * 3 * len_d, c->stream), "memset");
  SFB_CUDA(cudaMemsetAsync(c->dev.mom_w, 0, sizeof(double) * 2, c->stream), "memset");
  SFB_CUDA(cudaMemsetAsync(c->dev.st_c0, 0, sizeof(double) * Cs, c->stream), "memset");
  SFB_CUDA(cudaMemsetAsync(c->dev.st_m, 0, sizeof(double) * Cs, c->stream), "memset");
  SFB_CUDA(cudaMemsetAsync(c->dev.st_M, 0, sizeof(double) * Cs * Cs, c->stream), "memset");
  c->mom_shift_set = false;
  c->n_solved = 0;
  return SFB_OK;
}

}  // extern "C"
