// The opaque context behind sfb_ctx* and the device workspace layout.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/sfb.h"
#include "host_setup.h"
#include "sfb_internal.h"

namespace sfb {

// Bump allocator over the caller's workspace: a dry run (base == nullptr)
// measures, a second run hands out 256-byte aligned slices.
struct Carver {
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += count * sizeof(T);
    return p;
  }
};

struct StokesHost {
  int sx = 0, sy = 0;
  double x0 = 0, x1 = 0, y0 = 0, y1 = 0, hx = 0, hy = 0;
  int NX = 0, NY = 0, n_nodes = 0, n_u = 0, n_p = 0;
  std::vector<int64_t> dofs;       // Stokes-Darcy mortar DOFs (global)
  std::vector<int> free_index;     // full DOF (u then p) -> free index or -1
  std::vector<int> free_to_full;   // free index -> full DOF
  int n_free = 0;
  // assembled system on free DOFs as unique (row, col, value) triplets
  std::vector<int> tr_row, tr_col;
  std::vector<double> tr_val;
  std::vector<double> rhs;         // [n_free][R_s + 1]
  std::vector<double> dir_val;     // full velocity vector of Dirichlet values
  std::vector<double> nb;          // [n_bottom_nodes][R_s]: <xi_l, phi_node . n>
  std::vector<int> nb_node;        // bottom node ids
  // the free system is ordered node by node along the shorter lattice
  // direction (u_x, u_y and the vertex pressure of a node together), which
  // makes it banded: kl sub- and ku super-diagonals; the triplets are sorted
  // by row, row r's entries at [row_ptr[r], row_ptr[r + 1])
  int kl = 0, ku = 0;
  std::vector<int> row_ptr;
};

struct Dev {
  // set-up tables
  SubDev* subs = nullptr;
  double* proj = nullptr;
  int* dofinfo = nullptr;
  double* kl = nullptr;
  double* yloc = nullptr;
  int64_t* gdof = nullptr;
  int* item_sub = nullptr;
  int* item_k = nullptr;
  ItemOff* off = nullptr;
  // basis store
  double* X = nullptr;
  double* T = nullptr;
  void* G = nullptr;
  void* Z = nullptr;
  void* gmaps = nullptr;     // per item: tensor map (128 bytes) of its block inverses, tensor-core form
  double* phi = nullptr;
  float* phi32 = nullptr;    // FP32 copy of phi for the FP32 interface products
  double* D = nullptr;
  void* S = nullptr;
  void* DL = nullptr;
  double* errest = nullptr;
  long long* cycles = nullptr;
  int* status = nullptr;
  double* resid = nullptr;
  double* corr1 = nullptr;
  int* nref = nullptr;
  int* chunk_item = nullptr;  // split launch shapes: per column chunk its class-local item,
  int* chunk_c0 = nullptr;    // first column and column count (wide class first)
  int* chunk_cnt = nullptr;
  int* persist_counter = nullptr;   // the persistent basis launch's task counter
  int* persist_flags = nullptr;     // ... and its per-item "factor done" flags
  // Stokes
  double* s_mat = nullptr;
  double* s_pl = nullptr;    // the band LU's panel multipliers in final row order
  int* s_piv = nullptr;
  double* s_rhs = nullptr;
  double* s_b = nullptr;     // the Stokes right-hand sides, kept for the refinement residual
  double* s_res = nullptr;   // residual, then correction, of the refinement pass
  int* s_row_ptr = nullptr;
  double* s_U = nullptr;     // [n_u][Cs]
  double* s_P = nullptr;     // [n_p][Cs]
  double* s_phi = nullptr;   // [Rs][Rs] then g [Rs]
  float* s_phi32 = nullptr;  // FP32 copy of s_phi
  double* s_dir = nullptr;
  double* s_nb = nullptr;
  int* s_nb_node = nullptr;
  int* s_free_to_full = nullptr;
  int* s_tr_row = nullptr;
  int* s_tr_col = nullptr;
  double* s_tr_val = nullptr;
  int* s_status = nullptr;
  // interface solve (sized for max_pts)
  double* y = nullptr;
  double* w = nullptr;
  int* kmap = nullptr;        // [n_pts][n_sub]
  int* hash = nullptr;        // per region open-addressing tables
  int64_t* hash_off = nullptr;
  int* hash_cap = nullptr;
  int* grp_count = nullptr;   // per subdomain [n_local]
  int* grp_start = nullptr;
  int* grp_pts = nullptr;     // per subdomain [n_pts] points sorted by group
  int* tiles = nullptr;       // per subdomain [max_tiles][3]
  int* n_tiles = nullptr;     // per subdomain (+ Stokes)
  int* ldof = nullptr;        // per global DOF: 2 (unit, local) pairs
  int* yoff = nullptr;        // per global DOF: its 2 offsets into a point's Y row
  double* lam = nullptr;
  double* r = nullptr;
  double* p = nullptr;
  double* Y = nullptr;        // [n_pts][NY]
  double* rr = nullptr;
  double* gn = nullptr;
  double* rlast = nullptr;
  double* dinv = nullptr;
  double* gmV = nullptr;      // GMRES Krylov basis [kGmresMax + 1][n_pts][n_lambda]
  double* gmS = nullptr;      // GMRES per-point state [n_pts][kGmresState]
  double* bdd_pinv = nullptr;  // balancing preconditioner: pseudo-inverses of the Darcy bases (phi offsets)
  double* bdd_spinv = nullptr; // ... and of the Stokes basis
  double* bdd_wy = nullptr;    // per point, in Y's layout: each unit's stiffness share at its DOFs
  double* bdd_sz = nullptr;    // per point: S Z [n_c][n_lambda]
  double* bdd_L = nullptr;     // per point: Cholesky factor of S_0 = Z^T S Z
  int* bdd_cidx = nullptr;     // per unit: its coarse vector or -1
  int* gmJ = nullptr;         // GMRES steps of the current cycle per point     // Jacobi preconditioner of the interface CG, per point
  float* minv = nullptr;      // interface block-Jacobi inverses, per point [minv_ld]
  int* if_off = nullptr;      // per interface: first global DOF, DOF count, offset of its block
  int* if_n = nullptr;
  int* if_moff = nullptr;
  int* dof_if = nullptr;      // per global DOF: its interface
  int* rflag = nullptr;
  int* pstat = nullptr;       // per point: iterations (>0 converged, <0 active/failed)
  int* active = nullptr;
  int* pcg_part = nullptr;    // persistent CG: per-CTA ranges of resident tiles
  int64_t* s_gdof = nullptr;  // Stokes local -> global mortar DOF
  int64_t* ybase = nullptr;   // per unit offset into a point's Y row
  int* dim_off = nullptr;     // per subdomain: its KL region's first stochastic dimension
  int64_t* loc_off = nullptr; // per region offset into grp_count / grp_start
  int64_t* cell_off = nullptr;// per subdomain first cell in the Darcy pressure field
  int64_t* face_off = nullptr;// per subdomain first face in the Darcy flux field
  double* fin = nullptr;      // [2][max field length] finalised mean / variance
  // moments
  double* mom = nullptr;      // Darcy entries: shift, S1, S2
  double* mom_w = nullptr;
  double* mom_part = nullptr; // [chunks][2][Darcy entries] partial sums of a batch
  int4* mom_work = nullptr;   // point-by-point moment sub-tiles (subdomain, tile, first point)
  double* st_c0 = nullptr;    // Stokes: coefficients of the shift point
  double* st_m = nullptr;     // Stokes: sum w (c - c0)
  double* st_M = nullptr;     // Stokes: sum w (c - c0)(c - c0)^T
  double* st_part = nullptr;  // Stokes: per point chunk partials of st_m, st_M
  double* gmom = nullptr;     // per group: W | cbar | m | M (large groups)
  double* gmom_part = nullptr;// per group and point chunk: partial moments
};

}  // namespace sfb

struct sfb_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  // problem
  sfb_problem prob{};
  std::vector<int32_t> nx, ny, msd, mdv, mdh;
  std::vector<double> source;
  std::vector<sfb::HostSub> subs;
  std::vector<sfb::HostIface> ifaces;
  int64_t n_lambda = 0;
  sfb::StokesHost stokes;
  // state
  bool kl_done = false, coll_done = false, basis_done = false;
  bool ws_stale = false;   // a set-up call came after the workspace was set
  int basis_prec = -1;
  int64_t n_solved = 0;
  int64_t launches = 0;   // kernels launched by this context
  // collocation
  sfb::Grid grid;
  std::vector<std::vector<double>> loc_y;  // per region [n_local][nt]
  std::vector<int> n_local;
  std::vector<int> dim_off;                // kappa(i, 0) of each subdomain's KL region
  std::vector<int> region_of;              // KL region of each Darcy subdomain
  int n_regions = 0;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int ws_prec = -1;
  int64_t ws_pts = 0;
  sfb::Dev dev;
  int64_t n_items = 0;
  int64_t n_chunks = 0;                 // column chunks of all items (split launch shapes)
  int64_t chunk_start[2] = {0, 0}, chunk_n[2] = {0, 0};   // per size class (wide, narrow)
  std::vector<int> h_chunk_item;        // host copy of the chunks' class-local items
  std::vector<int64_t> item_id;         // item id of each item in build order
  int max_nx = 0, max_cols = 0, max_R = 0;
  // basis items come in decreasing cost; the first n_wide have nx > 64 and run
  // with the wide-grid kernel variant, the rest with the narrow one
  int64_t n_wide = 0;
  int wide_nx = 0, wide_cols = 0, narrow_nx = 0, narrow_cols = 0;
  cudaStream_t side = nullptr;          // second stream for the narrow items
  cudaEvent_t fork = nullptr, join = nullptr;
  // split launch shapes: per size class two streams for the solve launches of
  // alternate item groups, and the events that order each group's solves
  // after its factor (see sfb_build_stochastic_basis)
  static constexpr int kPipeGroups = 4;   // at most (option "basis_pipe_groups")
  cudaStream_t pipe_stream[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t pipe_ev[2][kPipeGroups + 3] = {};
  cudaStream_t gcap = nullptr;          // private stream on which the basis graph is captured
  std::vector<sfb::ItemOff> offs;
  std::vector<int64_t> ybase;              // per unit (Darcy subs, then Stokes) offset into Y
  int64_t NY = 0;
  int max_tiles = 0;
  int64_t mom_len[4] = {0, 0, 0, 0};
  int64_t mom_off[4] = {0, 0, 0, 0};
  bool mom_shift_set = false;
  int mom_chunks = 1;
  int mom_work_cap = 0;       // entries of dev.mom_work
  int64_t minv_ld = 0;        // sum over interfaces of (DOF count)^2
  int max_if_dof = 0;         // largest interface DOF count
  int64_t gmom_stride = 1;
  // options (sfb_set_option)
  double opt_refine_tol = 1e-11;
  int opt_refine_max = 8;
  int opt_cg_chunk = 8;
  int opt_cg_persistent = 1;    // interface CG in one cooperative launch (0: one launch per step)
  int opt_cg_precond = 2;       // interface CG preconditioner: 0 none, 1 Jacobi, 2 interface blocks
  double opt_cg_replace = 0.1;  // mixed CG: FP64 residual once the recursive one drops by this factor
  int opt_gmres_m = sfb::kGmresMax;   // GMRES restart length
  int opt_mom_df = 1;           // mixed form: moment contractions in double-float (0: FP64)
  double opt_big_factor = 1.0;   // groups above this many times (R+1) points use coefficient moments
  int opt_basis_graph = 1;      // basis launches of every size class replayed as one CUDA graph
  int opt_basis_autotune = 1;   // time the launch shapes of each size class on the first build
  // basis build: launch shape per precision (sfb_precision) and size class
  // ([0] grids wider than 64 cells, [1] the rest), the autotuner's timings of
  // each candidate (ms, 0 = not timed), and the captured graph per precision
  int bshape[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  bool btuned[3] = {false, false, false};
  // the persistent basis launch: option (-1 autotuned, 0 off, 1 on), the
  // autotuner's choice and timings (per-class launches, persistent launch)
  int opt_basis_persistent = -1;
  int opt_pipe_groups = 1;
  bool bpersist[3] = {false, false, false}, bpersist_tuned[3] = {false, false, false};
  double bpersist_ms[3][2] = {};
  double btune_ms[3][2][4] = {};
  struct GraphKey {
    const char* ws = nullptr;
    int refine = 0;
    double refine_tol = 0.0;
    int shape[2] = {0, 0};
    int persist = 0;
    int groups = 0;
    bool operator==(const GraphKey& o) const {
      return ws == o.ws && refine == o.refine && refine_tol == o.refine_tol && shape[0] == o.shape[0] &&
             shape[1] == o.shape[1] && persist == o.persist && groups == o.groups;
    }
  };
  cudaGraphExec_t bgraph[3] = {nullptr, nullptr, nullptr};
  GraphKey bkey[3];
  int bgraph_kernels[3] = {0, 0, 0};
  bool last_build_graph = false;
  // tensor maps of the block inverses (tensor-core basis kernel): encoded for
  // the workspace at gmaps_ws; gmaps_ok false when the driver cannot encode them
  const char* gmaps_ws = nullptr;
  bool gmaps_ok = false;
  // device-time phase markers of the last interface solve (CUDA events)
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int cg_iters_run = 0;
  bool cg_persistent_run = false;
  int test_barrier_skip = 0;   // test hook of the next one-launch CG (see cg_test_barrier_timeout)
  int pcg_grid = 1;
  std::vector<int> pcg_starts;   // host copy of the last resident partition
  int pcg_mode = 0;   // last persistent CG: bit 0 resident tiles, bit 1 two streaming buffers
  double pcg_cycles[6] = {0, 0, 0, 0, 0, 0};   // per CTA, last persistent CG
  bool last_dtn = false;
  // balancing preconditioner: coarse vectors (floating Darcy subdomains),
  // each unit's coarse index, and whether the pseudo-inverses are current
  int bdd_nc = 0;
  std::vector<int> bdd_cidx;
  bool bdd_items_ready = false, bdd_stokes_ready = false;   // the last batch was solved by Method S1 (its moments recover by subdomain solves)
  ~sfb_ctx() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t g : bgraph)
      if (g) cudaGraphExecDestroy(g);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
    for (auto& q : pipe_stream)
      for (cudaStream_t x : q)
        if (x) cudaStreamDestroy(x);
    for (auto& q : pipe_ev)
      for (cudaEvent_t x : q)
        if (x) cudaEventDestroy(x);
    if (gcap) cudaStreamDestroy(gcap);
  }
};

namespace sfb {
// Method S1 (s1.cu): the subdomain-solve form of the Darcy units' products,
// the recovery of the Darcy entries, and their moments.
size_t dtn_smem_bytes(int max_nx, int max_ny, int max_R);
cudaError_t launch_dtn(sfb_ctx* c, const double* vin, int64_t p0, int64_t cnt, int recovery, double* field,
                       cudaStream_t st);
cudaError_t launch_s1_moments(sfb_ctx* c, const double* field, int64_t p0, int64_t cnt, int first,
                              cudaStream_t st);
}  // namespace sfb
