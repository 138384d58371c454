// Host-side plan of the FIND passes: cluster tree, boundary / private-inner
// sets, gather tables of every elimination, level grouping and the flop model.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace findgb {

struct Cluster {
  int x0, x1, y0, y1;  // half-open rectangle of mesh nodes
  int parent;          // -1 for the root
  int child[2];        // -1 for a leaf
  int depth;           // root = 0
  int height;          // leaf = 0
};

// One row/column of an assembled block M: which mesh node it stands for and
// where its entries come from.  src 0: the original A / Sigma< (computed from
// the mesh); src 1 / 2: the first / second source matrix of the op, at row
// and column `idx` of that matrix.
struct Pos {
  int node;
  int src;
  int idx;
};

// One elimination (an upward merge, a leaf's own elimination, or a downward
// complement merge): assemble M over n positions ordered [S, B], eliminate
// the s private inner positions, keep the b boundary positions.
struct ElimOp {
  int cluster;
  int dst;         // matrix id receiving U (and R)
  int src1, src2;  // matrix ids of the source blocks, -1 if absent
  int n, s, b;
  int64_t pos;     // first entry in Plan::pos
};

// One leaf extraction: the bordered system over [Bbar, C].
struct LeafOp {
  int cluster;
  int src;           // matrix id of U_Cbar (-1 when the leaf is the root)
  int n, nb, c;      // n = nb + c
  int x0, y0, wx;    // leaf rectangle origin and width (C is row-major in it)
  int64_t pos;
  int64_t bond;      // first entry in Plan::bonds
  int nbond;
};

// A bond current produced by a leaf: the bond's output index, the positions
// of its source (in C) and target (in C or Bbar) in the leaf's bordered
// system, and the hopping kind (0: nearest, t; 1: diagonal, tp).
struct LeafBond {
  int bond;
  int pi, pj;
  int kind;
};

struct Plan {
  int nx = 0, ny = 0, stencil = 5, leaf = 8;
  std::vector<Cluster> cl;
  std::vector<std::vector<int>> B, Bb;  // B_C (inside C) and B_Cbar (outside C)
  std::vector<int> up_mat, dn_mat;       // cluster -> matrix id of U_C / U_Cbar
  std::vector<int> mat_dim;
  std::vector<int64_t> mat_off;          // complex elements, per energy
  int64_t mat_elems = 0;
  std::vector<Pos> pos;
  std::vector<std::vector<ElimOp>> up_levels;  // by height
  std::vector<std::vector<ElimOp>> dn_levels;  // by depth 1, 2, ...
  std::vector<LeafOp> leaf_ops;
  std::vector<LeafBond> bonds;
  int n_bonds = 0;
  int n_leaves = 0;
  int max_s = 0, max_b = 0, max_kn = 0;
  double flops_diag = 0, flops_lesser = 0;  // real flops per energy
};

int64_t bond_count(int nx, int ny, int stencil);

// Returns 0 on success; on failure fills err.
int build_plan(int nx, int ny, int stencil, int leaf, Plan& p, std::string& err);

}  // namespace findgb
