// Host assembly of the deterministic Stokes subdomain system: Taylor-Hood
// P2-P1 triangles (two per rectangle, split along the SW-NE diagonal) for
// 2 nu (D u, D v) - (div v, p) - (div u, q) with the BJS term
// nu alpha / sqrt(K_l) u.tau v.tau on the interface (Eqs. 2.2-2.4, 2.10,
// weak form of Section 3.2, K_l = 1 so the basis is deterministic) and the
// normal-stress mortar load -<lambda, v.n> (Eqs. 5.1-5.2). Element integrals
// are exact: gradients of P2 shapes are linear in the barycentric
// coordinates, and int_T lambda_m lambda_n = |T| (1 + delta_mn) / 12.
// The factorization and solves of this system run on the GPU (stokes.cu).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sfb_ctx.h"

namespace sfb {

namespace {

struct Trip {
  int64_t key;
  double val;
};

}  // namespace

void stokes_assemble_host(sfb_ctx* c) {
  StokesHost& S = c->stokes;
  const sfb_problem& P = c->prob;
  S.sx = P.stokes_sx; S.sy = P.stokes_sy;
  S.x0 = P.stokes_box[0]; S.x1 = P.stokes_box[1]; S.y0 = P.stokes_box[2]; S.y1 = P.stokes_box[3];
  S.hx = (S.x1 - S.x0) / S.sx; S.hy = (S.y1 - S.y0) / S.sy;
  S.NX = 2 * S.sx + 1; S.NY = 2 * S.sy + 1;
  S.n_nodes = S.NX * S.NY;
  S.n_u = 2 * S.n_nodes;
  S.n_p = (S.sx + 1) * (S.sy + 1);
  const int nn = S.n_nodes, n_full = S.n_u + S.n_p;
  const double nu = P.nu_s;
  auto node = [&](int i, int j) { return j * S.NX + i; };

  // Dirichlet data: parabolic inflow on the left edge, no slip on the top.
  std::vector<char> dir(S.n_u, 0);
  S.dir_val.assign(S.n_u, 0.0);
  for (int j = 0; j < S.NY; ++j) {
    const int n = node(0, j);
    const double s = (double)j / (S.NY - 1);
    dir[n] = dir[nn + n] = 1;
    S.dir_val[n] = P.u_in * 4.0 * s * (1.0 - s);
  }
  for (int i = 0; i < S.NX; ++i) {
    const int n = node(i, S.NY - 1);
    dir[n] = dir[nn + n] = 1;
    S.dir_val[n] = S.dir_val[nn + n] = 0.0;
  }
  S.free_index.assign(n_full, -1);
  S.free_to_full.clear();
  for (int d = 0; d < n_full; ++d)
    if (d >= S.n_u || !dir[d]) { S.free_index[d] = (int)S.free_to_full.size(); S.free_to_full.push_back(d); }
  S.n_free = (int)S.free_to_full.size();

  const int Rs = (int)S.dofs.size(), Cs = Rs + 1;
  S.rhs.assign((size_t)S.n_free * Cs, 0.0);
  std::vector<Trip> trips;
  trips.reserve((size_t)S.sx * S.sy * 2 * (144 + 72 + 72));
  auto add = [&](int r, int col, double v) {
    if (v == 0.0) return;
    const int fr = S.free_index[r];
    if (fr < 0) return;  // Dirichlet row
    const int fc = S.free_index[col];
    if (fc >= 0) trips.push_back({(int64_t)fr * S.n_free + fc, v});
    else S.rhs[(size_t)fr * Cs + Rs] -= v * S.dir_val[col];  // lift Dirichlet data
  };

  for (int J = 0; J < S.sy; ++J)
    for (int I = 0; I < S.sx; ++I)
      for (int tri = 0; tri < 2; ++tri) {
        const int i = 2 * I, j = 2 * J;
        int nodes[6], pv[3];
        double vx[3], vy[3];
        const double xs = S.x0 + I * S.hx, ys = S.y0 + J * S.hy;
        const int psw = J * (S.sx + 1) + I, pse = psw + 1, pnw = psw + S.sx + 1, pne = pnw + 1;
        if (tri == 0) {  // SW, SE, NE
          const int v[3] = {node(i, j), node(i + 2, j), node(i + 2, j + 2)};
          const int m[3] = {node(i + 1, j), node(i + 2, j + 1), node(i + 1, j + 1)};
          for (int q = 0; q < 3; ++q) { nodes[q] = v[q]; nodes[3 + q] = m[q]; }
          pv[0] = psw; pv[1] = pse; pv[2] = pne;
          vx[0] = xs; vy[0] = ys; vx[1] = xs + S.hx; vy[1] = ys; vx[2] = xs + S.hx; vy[2] = ys + S.hy;
        } else {         // SW, NE, NW
          const int v[3] = {node(i, j), node(i + 2, j + 2), node(i, j + 2)};
          const int m[3] = {node(i + 1, j + 1), node(i + 1, j + 2), node(i, j + 1)};
          for (int q = 0; q < 3; ++q) { nodes[q] = v[q]; nodes[3 + q] = m[q]; }
          pv[0] = psw; pv[1] = pne; pv[2] = pnw;
          vx[0] = xs; vy[0] = ys; vx[1] = xs + S.hx; vy[1] = ys + S.hy; vx[2] = xs; vy[2] = ys + S.hy;
        }
        const double det = (vx[1] - vx[0]) * (vy[2] - vy[0]) - (vx[2] - vx[0]) * (vy[1] - vy[0]);
        const double area = 0.5 * std::fabs(det);
        double gl[3][2] = {{(vy[1] - vy[2]) / det, (vx[2] - vx[1]) / det},
                           {(vy[2] - vy[0]) / det, (vx[0] - vx[2]) / det},
                           {(vy[0] - vy[1]) / det, (vx[1] - vx[0]) / det}};
        // grad phi_a = sum_m lambda_m G[a][m] (using sum_m lambda_m = 1)
        double G[6][3][2];
        std::memset(G, 0, sizeof(G));
        for (int a = 0; a < 3; ++a)
          for (int m = 0; m < 3; ++m)
            for (int d = 0; d < 2; ++d) G[a][m][d] = (m == a ? 4.0 : 0.0) * gl[a][d] - gl[a][d];
        const int ed[3][2] = {{0, 1}, {1, 2}, {2, 0}};
        for (int e = 0; e < 3; ++e) {
          const int p = ed[e][0], q = ed[e][1];
          for (int d = 0; d < 2; ++d) { G[3 + e][q][d] += 4.0 * gl[p][d]; G[3 + e][p][d] += 4.0 * gl[q][d]; }
        }
        auto mm = [&](int m, int n) { return area * (m == n ? 2.0 : 1.0) / 12.0; };
        // stiffness: nu [2 ux_x vx_x + 2 uy_y vy_y + (ux_y + uy_x)(vx_y + vy_x)]
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b < 6; ++b) {
            double kxx = 0, kyy = 0, kxy = 0, kyx = 0;  // int d_x phi_a d_x phi_b etc.
            for (int m = 0; m < 3; ++m)
              for (int n = 0; n < 3; ++n) {
                const double w = mm(m, n);
                kxx += w * G[a][m][0] * G[b][n][0];
                kyy += w * G[a][m][1] * G[b][n][1];
                kxy += w * G[a][m][0] * G[b][n][1];
                kyx += w * G[a][m][1] * G[b][n][0];
              }
            // rows: test a (component cv), cols: trial b (component cu)
            add(nodes[a], nodes[b], nu * (2.0 * kxx + kyy));
            add(nn + nodes[a], nn + nodes[b], nu * (2.0 * kyy + kxx));
            add(nodes[a], nn + nodes[b], nu * kyx);   // v_x,y * u_y,x
            add(nn + nodes[a], nodes[b], nu * kxy);   // v_y,x * u_x,y
          }
        // divergence: b(v, q) = -(div v, q), both (v, p) and (u, q) blocks
        for (int k = 0; k < 3; ++k)
          for (int a = 0; a < 6; ++a) {
            double bx = 0, by = 0;
            for (int m = 0; m < 3; ++m) { bx += mm(k, m) * G[a][m][0]; by += mm(k, m) * G[a][m][1]; }
            const int prow = S.n_u + pv[k];
            add(prow, nodes[a], -bx);
            add(prow, nn + nodes[a], -by);
            add(nodes[a], prow, -bx);
            add(nn + nodes[a], prow, -by);
          }
      }
  // BJS on the bottom (interface) edges: nu alpha / sqrt(K_l) u_x v_x, K_l = 1.
  {
    const double coef = P.nu_s * P.alpha;
    const double m1[3][3] = {{4, 2, -1}, {2, 16, 2}, {-1, 2, 4}};
    for (int I = 0; I < S.sx; ++I) {
      const int ids[3] = {node(2 * I, 0), node(2 * I + 1, 0), node(2 * I + 2, 0)};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) add(ids[a], ids[b], coef * S.hx * m1[a][b] / 30.0);
    }
  }
  // merge duplicate triplets
  std::sort(trips.begin(), trips.end(), [](const Trip& a, const Trip& b) { return a.key < b.key; });
  S.tr_row.clear(); S.tr_col.clear(); S.tr_val.clear();
  for (size_t t = 0; t < trips.size();) {
    const int64_t key = trips[t].key;
    double v = 0.0;
    while (t < trips.size() && trips[t].key == key) v += trips[t++].val;
    S.tr_row.push_back((int)(key / S.n_free));
    S.tr_col.push_back((int)(key % S.n_free));
    S.tr_val.push_back(v);
  }
  // normal-stress mortar load: N[(y, node), l] = <xi_l, phi_node . n>, n = (0, -1)
  S.nb_node.clear();
  for (int i = 0; i < S.NX; ++i) S.nb_node.push_back(node(i, 0));
  S.nb.assign((size_t)S.NX * Rs, 0.0);
  std::vector<double> tmp;
  for (int I = 0; I < S.sx; ++I) {
    const double xa = S.x0 + I * S.hx, xb = xa + S.hx;
    for (int q = 0; q < 3; ++q) {
      const int bi = 2 * I + q;
      for (const HostIface& itf : c->ifaces) {
        if (itf.kind != 0) continue;
        tmp.assign(itf.n_dof, 0.0);
        mortar_times_p2(itf, xa, xb, q, tmp.data());
        for (int a = 0; a < itf.n_dof; ++a) {
          const int64_t gd = itf.off + a;
          const int l = (int)(std::lower_bound(S.dofs.begin(), S.dofs.end(), gd) - S.dofs.begin());
          S.nb[(size_t)bi * Rs + l] -= tmp[a];
        }
      }
    }
  }
  // basis right-hand sides: -N[:, j] on free u_y rows of bottom nodes
  for (int bi = 0; bi < S.NX; ++bi) {
    const int fr = S.free_index[nn + S.nb_node[bi]];
    if (fr < 0) continue;
    for (int l = 0; l < Rs; ++l) S.rhs[(size_t)fr * Cs + l] = -S.nb[(size_t)bi * Rs + l];
  }
  // Band ordering of the free unknowns: by P2-lattice node along the shorter
  // lattice direction, the two velocity components and (at vertices) the
  // pressure of a node together. A triangle couples nodes of two neighbouring
  // lattice lines, so the bandwidth is about six lattice lines' worth of
  // unknowns instead of the whole system.
  const bool by_column = S.NY < S.NX;
  auto key_of = [&](int d) -> int64_t {
    int i, j, comp;
    if (d < S.n_u) {
      comp = d / nn;
      i = (d % nn) % S.NX;
      j = (d % nn) / S.NX;
    } else {
      const int q = d - S.n_u;
      comp = 2;
      i = 2 * (q % (S.sx + 1));
      j = 2 * (q / (S.sx + 1));
    }
    const int64_t line = by_column ? (int64_t)i * S.NY + j : (int64_t)j * S.NX + i;
    return line * 3 + comp;
  };
  std::vector<int> order(S.n_free);
  for (int f = 0; f < S.n_free; ++f) order[f] = f;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return key_of(S.free_to_full[a]) < key_of(S.free_to_full[b]); });
  std::vector<int> pos(S.n_free);
  for (int b = 0; b < S.n_free; ++b) pos[order[b]] = b;
  std::vector<int> f2f(S.n_free);
  for (int b = 0; b < S.n_free; ++b) f2f[b] = S.free_to_full[order[b]];
  S.free_to_full.swap(f2f);
  for (int d = 0; d < n_full; ++d)
    if (S.free_index[d] >= 0) S.free_index[d] = pos[S.free_index[d]];
  std::vector<double> rhs2(S.rhs.size());
  for (int f = 0; f < S.n_free; ++f)
    std::copy(S.rhs.begin() + (size_t)f * Cs, S.rhs.begin() + (size_t)(f + 1) * Cs, rhs2.begin() + (size_t)pos[f] * Cs);
  S.rhs.swap(rhs2);
  S.kl = S.ku = 0;
  std::vector<Trip> bt(S.tr_val.size());
  for (size_t t = 0; t < S.tr_val.size(); ++t) {
    const int r = pos[S.tr_row[t]], q = pos[S.tr_col[t]];
    bt[t] = {(int64_t)r * S.n_free + q, S.tr_val[t]};
    S.kl = std::max(S.kl, r - q);
    S.ku = std::max(S.ku, q - r);
  }
  // row-major order (the refinement residual runs row by row)
  std::sort(bt.begin(), bt.end(), [](const Trip& a, const Trip& b) { return a.key < b.key; });
  S.row_ptr.assign((size_t)S.n_free + 1, 0);
  for (size_t t = 0; t < bt.size(); ++t) {
    S.tr_row[t] = (int)(bt[t].key / S.n_free);
    S.tr_col[t] = (int)(bt[t].key % S.n_free);
    S.tr_val[t] = bt[t].val;
    ++S.row_ptr[(size_t)S.tr_row[t] + 1];
  }
  for (int r = 0; r < S.n_free; ++r) S.row_ptr[(size_t)r + 1] += S.row_ptr[r];
}

}  // namespace sfb
