// Host-side plan of the FIND passes.
//
// Sec. 2.1-2.2 of the paper: the mesh is split recursively into clusters;
// B_C is the set of nodes of C with a neighbour outside C, S_C the private
// inner nodes (B_C1 u B_C2) \ B_C eliminated when C is formed; the complement
// cluster Cbar has boundary B_Cbar (nodes outside C next to C) and private
// inner set (B_Dbar u B_D1) \ B_Cbar (D the parent, D1 the sibling).  The
// neighbour graph is that of A: the stencil bonds plus the dense coupling of
// all nodes within each contact column (the lead self-energies).
//
// Split rule (the paper's figures are missing; this is the reading taken):
// bisect the longer side, ties split y, the first half gets floor(len/2),
// until both sides are <= leaf.
#include "plan.hpp"

#include <algorithm>
#include <cstdio>
#include <functional>

namespace findgb {

int64_t bond_count(int nx, int ny, int stencil) {
  int64_t c = (int64_t)(ny - 1) * nx + (int64_t)ny * (nx - 1);
  if (stencil == 9) c += 2 * (int64_t)(ny - 1) * (nx - 1);
  return c;
}

namespace {

struct Mesh {
  int nx, ny, stencil;
  int node(int x, int y) const { return y * nx + x; }
};

bool inside(const Cluster& c, int node, int nx) {
  int x = node % nx, y = node / nx;
  return x >= c.x0 && x < c.x1 && y >= c.y0 && y < c.y1;
}

// Visit every graph neighbour j of node i (stencil bonds; contact cliques are
// handled separately because they are dense).
template <class F>
void stencil_neighbours(const Mesh& m, int i, F&& f) {
  int x = i % m.nx, y = i / m.nx;
  static const int d5[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
  static const int d9[4][2] = {{1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
  for (auto& d : d5) {
    int x2 = x + d[0], y2 = y + d[1];
    if (x2 >= 0 && x2 < m.nx && y2 >= 0 && y2 < m.ny) f(m.node(x2, y2));
  }
  if (m.stencil == 9)
    for (auto& d : d9) {
      int x2 = x + d[0], y2 = y + d[1];
      if (x2 >= 0 && x2 < m.nx && y2 >= 0 && y2 < m.ny) f(m.node(x2, y2));
    }
}

}  // namespace

int build_plan(int nx, int ny, int stencil, int leaf, Plan& p, std::string& err) {
  if (nx < 1 || ny < 2) { err = "need nx >= 1 and ny >= 2"; return 1; }
  if (stencil != 5 && stencil != 9) { err = "stencil must be 5 or 9"; return 1; }
  if (leaf < 1) { err = "leaf must be >= 1"; return 1; }
  if ((int64_t)nx * ny > (int64_t)1 << 30) { err = "mesh too large"; return 1; }
  p = Plan();
  p.nx = nx; p.ny = ny; p.stencil = stencil; p.leaf = leaf;
  const Mesh m{nx, ny, stencil};
  const int n = nx * ny;

  // ---- tree
  std::function<int(int, int, int, int, int, int)> make = [&](int x0, int x1, int y0, int y1,
                                                              int parent, int depth) -> int {
    int id = (int)p.cl.size();
    p.cl.push_back(Cluster{x0, x1, y0, y1, parent, {-1, -1}, depth, 0});
    int wx = x1 - x0, wy = y1 - y0;
    if (wx <= leaf && wy <= leaf) return id;
    int a, b;
    if (wy >= wx) {
      int h = wy / 2;
      a = make(x0, x1, y0, y0 + h, id, depth + 1);
      b = make(x0, x1, y0 + h, y1, id, depth + 1);
    } else {
      int h = wx / 2;
      a = make(x0, x0 + h, y0, y1, id, depth + 1);
      b = make(x0 + h, x1, y0, y1, id, depth + 1);
    }
    p.cl[id].child[0] = a;
    p.cl[id].child[1] = b;
    p.cl[id].height = 1 + std::max(p.cl[a].height, p.cl[b].height);
    return id;
  };
  make(0, nx, 0, ny, -1, 0);
  const int ncl = (int)p.cl.size();

  // ---- boundary sets B_C and B_Cbar
  p.B.assign(ncl, {});
  p.Bb.assign(ncl, {});
  std::vector<int> stamp(n, -1);
  for (int g = 0; g < ncl; ++g) {
    const Cluster& c = p.cl[g];
    std::vector<int>& B = p.B[g];
    std::vector<int>& Bb = p.Bb[g];
    for (int y = c.y0; y < c.y1; ++y)
      for (int x = c.x0; x < c.x1; ++x) {
        int i = m.node(x, y);
        bool bnd = false;
        stencil_neighbours(m, i, [&](int j) {
          if (!inside(c, j, nx)) {
            bnd = true;
            if (stamp[j] != g) { stamp[j] = g; Bb.push_back(j); }
          }
        });
        // dense lead coupling inside each contact column
        bool contact = (y == 0 || y == ny - 1);
        if (contact && (c.x0 > 0 || c.x1 < nx)) bnd = true;
        if (bnd) B.push_back(i);
      }
    for (int col : {0, ny - 1}) {
      if (col < c.y0 || col >= c.y1) continue;
      for (int x = 0; x < nx; ++x) {
        if (x >= c.x0 && x < c.x1) continue;
        int j = m.node(x, col);
        if (stamp[j] != g) { stamp[j] = g; Bb.push_back(j); }
      }
    }
    std::sort(B.begin(), B.end());
    std::sort(Bb.begin(), Bb.end());
  }

  // ---- matrix ids: U_C for every non-root basic cluster, U_Cbar for every
  // non-root complement cluster
  p.up_mat.assign(ncl, -1);
  p.dn_mat.assign(ncl, -1);
  auto add_mat = [&](int dim) {
    int id = (int)p.mat_dim.size();
    p.mat_dim.push_back(dim);
    p.mat_off.push_back(p.mat_elems);
    p.mat_elems += (int64_t)dim * dim;
    return id;
  };
  for (int g = 1; g < ncl; ++g) p.up_mat[g] = add_mat((int)p.B[g].size());
  for (int g = 1; g < ncl; ++g) p.dn_mat[g] = add_mat((int)p.Bb[g].size());

  // ---- gather tables
  std::vector<int> mark(n, 0);
  int mark_gen = 0;
  // Appends positions for the merged list (src, idx already attached) ordered
  // [S, B]: S = merged nodes not in keep (merged order), then keep (sorted).
  auto emit_elim = [&](const std::vector<Pos>& merged, const std::vector<int>& keep, ElimOp& op) {
    ++mark_gen;
    for (int j : keep) mark[j] = mark_gen;
    op.pos = (int64_t)p.pos.size();
    int s = 0;
    for (const Pos& q : merged)
      if (mark[q.node] != mark_gen) { p.pos.push_back(q); ++s; }
    // keep in sorted order; find each in merged
    ++mark_gen;
    std::vector<int> where;  // node -> index in merged, via a temporary map
    for (size_t k = 0; k < merged.size(); ++k) { stamp[merged[k].node] = (int)k; mark[merged[k].node] = mark_gen; }
    for (int j : keep) {
      if (mark[j] != mark_gen) return false;  // keep not a subset of merged
      p.pos.push_back(merged[stamp[j]]);
    }
    op.n = (int)merged.size();
    op.s = s;
    op.b = (int)keep.size();
    return true;
  };

  auto flops_elim = [](double s, double b, bool lesser) {
    // Sec. 4, Eqs. (14)-(15): U costs s^3/3 + s^2 b + s b^2, R costs s^2 b + 3 s b^2
    // complex multiply-adds; 8 real flops each.
    double u = s * s * s / 3.0 + s * s * b + s * b * b;
    double r = s * s * b + 3.0 * s * b * b;
    return 8.0 * (lesser ? u + r : u);
  };

  int maxh = p.cl[0].height;
  p.up_levels.assign(maxh + 1, {});
  int maxd = 0;
  for (auto& c : p.cl) maxd = std::max(maxd, c.depth);
  p.dn_levels.assign(maxd, {});

  for (int g = 1; g < ncl; ++g) {  // upward ops (the root is not eliminated)
    const Cluster& c = p.cl[g];
    std::vector<Pos> merged;
    ElimOp op{};
    op.cluster = g;
    op.dst = p.up_mat[g];
    op.src1 = op.src2 = -1;
    if (c.child[0] < 0) {
      for (int y = c.y0; y < c.y1; ++y)
        for (int x = c.x0; x < c.x1; ++x) merged.push_back(Pos{m.node(x, y), 0, 0});
    } else {
      int a = c.child[0], b = c.child[1];
      op.src1 = p.up_mat[a];
      op.src2 = p.up_mat[b];
      for (size_t k = 0; k < p.B[a].size(); ++k) merged.push_back(Pos{p.B[a][k], 1, (int)k});
      for (size_t k = 0; k < p.B[b].size(); ++k) merged.push_back(Pos{p.B[b][k], 2, (int)k});
    }
    if (!emit_elim(merged, p.B[g], op)) { err = "internal: B_C not inside merged set"; return 2; }
    p.up_levels[c.height].push_back(op);
  }
  for (int g = 1; g < ncl; ++g) {  // downward ops
    const Cluster& c = p.cl[g];
    int d = c.parent;
    int d1 = p.cl[d].child[0] == g ? p.cl[d].child[1] : p.cl[d].child[0];
    std::vector<Pos> merged;
    ElimOp op{};
    op.cluster = g;
    op.dst = p.dn_mat[g];
    op.src1 = (d == 0) ? -1 : p.dn_mat[d];
    op.src2 = p.up_mat[d1];
    if (d != 0)
      for (size_t k = 0; k < p.Bb[d].size(); ++k) merged.push_back(Pos{p.Bb[d][k], 1, (int)k});
    for (size_t k = 0; k < p.B[d1].size(); ++k) merged.push_back(Pos{p.B[d1][k], 2, (int)k});
    if (!emit_elim(merged, p.Bb[g], op)) { err = "internal: B_Cbar not inside merged set"; return 2; }
    p.dn_levels[c.depth - 1].push_back(op);
  }
  // drop empty levels (a degenerate tree has none)
  p.up_levels.erase(std::remove_if(p.up_levels.begin(), p.up_levels.end(),
                                   [](const std::vector<ElimOp>& v) { return v.empty(); }),
                    p.up_levels.end());
  p.dn_levels.erase(std::remove_if(p.dn_levels.begin(), p.dn_levels.end(),
                                   [](const std::vector<ElimOp>& v) { return v.empty(); }),
                    p.dn_levels.end());

  // ---- leaf extraction ops and their bond tables
  p.n_bonds = (int)bond_count(nx, ny, stencil);
  const int oy = 0, ox = (ny - 1) * nx, odp = ox + ny * (nx - 1), odm = odp + (ny - 1) * (nx - 1);
  std::vector<int> posK(n, -1);
  for (int g = 0; g < ncl; ++g) {
    const Cluster& c = p.cl[g];
    if (c.child[0] >= 0) continue;
    ++p.n_leaves;
    LeafOp op{};
    op.cluster = g;
    op.src = (g == 0) ? -1 : p.dn_mat[g];
    op.x0 = c.x0; op.y0 = c.y0; op.wx = c.x1 - c.x0;
    op.pos = (int64_t)p.pos.size();
    int k = 0;
    if (g != 0)
      for (size_t q = 0; q < p.Bb[g].size(); ++q) {
        p.pos.push_back(Pos{p.Bb[g][q], 1, (int)q});
        posK[p.Bb[g][q]] = k++;
      }
    op.nb = k;
    for (int y = c.y0; y < c.y1; ++y)
      for (int x = c.x0; x < c.x1; ++x) {
        p.pos.push_back(Pos{m.node(x, y), 0, 0});
        posK[m.node(x, y)] = k++;
      }
    op.n = k;
    op.c = k - op.nb;
    op.bond = (int64_t)p.bonds.size();
    auto add_bond = [&](int bond, int i, int j, int kind) {
      if (posK[j] < 0) { err = "internal: bond target outside the bordered leaf"; return false; }
      p.bonds.push_back(LeafBond{bond, posK[i], posK[j], kind});
      return true;
    };
    for (int y = c.y0; y < c.y1; ++y)
      for (int x = c.x0; x < c.x1; ++x) {
        int i = m.node(x, y);
        bool ok = true;
        if (y < ny - 1) ok &= add_bond(oy + y * nx + x, i, m.node(x, y + 1), 0);
        if (x < nx - 1) ok &= add_bond(ox + y * (nx - 1) + x, i, m.node(x + 1, y), 0);
        if (stencil == 9 && y < ny - 1) {
          if (x < nx - 1) ok &= add_bond(odp + y * (nx - 1) + x, i, m.node(x + 1, y + 1), 1);
          if (x >= 1) ok &= add_bond(odm + y * (nx - 1) + (x - 1), i, m.node(x - 1, y + 1), 1);
        }
        if (!ok) return 2;
      }
    op.nbond = (int)((int64_t)p.bonds.size() - op.bond);
    for (int q = 0; q < op.n; ++q) posK[p.pos[op.pos + q].node] = -1;
    p.leaf_ops.push_back(op);
  }

  // ---- sizes and the flop model
  for (auto& lv : p.up_levels)
    for (auto& op : lv) {
      p.max_s = std::max(p.max_s, op.s);
      p.max_b = std::max(p.max_b, op.b);
      p.flops_diag += flops_elim(op.s, op.b, false);
      p.flops_lesser += flops_elim(op.s, op.b, true);
    }
  for (auto& lv : p.dn_levels)
    for (auto& op : lv) {
      p.max_s = std::max(p.max_s, op.s);
      p.max_b = std::max(p.max_b, op.b);
      p.flops_diag += flops_elim(op.s, op.b, false);
      p.flops_lesser += flops_elim(op.s, op.b, true);
    }
  for (auto& op : p.leaf_ops) {
    p.max_kn = std::max(p.max_kn, op.n);
    // Eq. (8): eliminate Bbar onto C (s = nb, b = c) and invert the c x c
    // result; Eq. (5)/(7): the same elimination of Sigma, then G R G^H.
    double c = op.c;
    p.flops_diag += flops_elim(op.nb, c, false) + 8.0 * c * c * c;
    p.flops_lesser += flops_elim(op.nb, c, true) + 8.0 * 3.0 * c * c * c;
  }
  return 0;
}

}  // namespace findgb
